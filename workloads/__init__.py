"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  Holds no arithmetic of the matching method."""
from .gen import (Pair, config1, config2, config4, config5, tiny_pair, template_half,
                  margin_for, optical_like, shift_image, scale01, piecewise_inverting_map,
                  gamma_speckle, radiometric, block_points, planted_model, apply_model,
                  planted_correspondences, ransac_samples, add_noise)

__all__ = ["Pair", "config1", "config2", "config4", "config5", "tiny_pair", "template_half",
           "margin_for", "optical_like", "shift_image", "scale01", "piecewise_inverting_map",
           "gamma_speckle", "radiometric", "block_points", "planted_model", "apply_model",
           "planted_correspondences", "ransac_samples", "add_noise"]
