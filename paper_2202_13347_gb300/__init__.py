"""GB300 (sm_103a) implementation of the SFOC descriptor and Fast-NCC_SFOC
matching of arXiv 2202.13347 (fine registration: Sec. 2 and Sec. 3.2).

The work runs in the CUDA library ``libsfoc_gb300.so`` built from
``csrc/`` (C ABI in ``include/sfoc.h``); ``binding`` marshals torch tensors
into it.  Importing the binding fails if the library is not built.
"""
from .build import build, LIB  # noqa: F401


def load():
    """Returns the binding module with the library loaded (raises if absent)."""
    from . import binding as b
    b.lib()
    return b
