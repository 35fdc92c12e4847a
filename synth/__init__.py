"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark."""
from .generator import (Pair, batch_sizes, config_pair, default_counts,  # noqa: F401
                        ground_truth_affine, make_pair,
                        pair_seed, rotate_bilinear, scene, serving_sizes, smooth_sizes)
