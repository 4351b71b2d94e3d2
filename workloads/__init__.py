"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  Holds no arithmetic of the matching method."""
from .gen import (Pair, inverting_pair_512, sar_pair_2048, mixed_batch, speckle_pair_10000, tiny_pair, template_half,
                  margin_for, optical_like, shift_image, scale01, piecewise_inverting_map,
                  gamma_speckle, radiometric, block_points, planted_model, apply_model,
                  planted_correspondences, ransac_samples, add_noise)

__all__ = ["Pair", "inverting_pair_512", "sar_pair_2048", "mixed_batch", "speckle_pair_10000", "tiny_pair", "template_half",
           "margin_for", "optical_like", "shift_image", "scale01", "piecewise_inverting_map",
           "gamma_speckle", "radiometric", "block_points", "planted_model", "apply_model",
           "planted_correspondences", "ransac_samples", "add_noise"]
