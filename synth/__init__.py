"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark."""
from .generator import (Pair, batch_sizes, config_pair, default_counts, make_pair,  # noqa: F401
                        pair_seed, rotate_bilinear, scene, serving_sizes, smooth_sizes)
