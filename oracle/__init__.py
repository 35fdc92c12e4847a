"""FP64 CPU oracle of the RIFT2 feature pipeline.  Test infrastructure only: imported by
the tests, the smoke check and the benchmark's CPU baseline, never by the CUDA path."""
from .rift2_oracle import *  # noqa: F401,F403
from .rift2_oracle import DEFAULT, Features, Params  # noqa: F401
