"""FP64 CPU oracle of the uplink receiver hot path.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import this package; the library's product path never does, and this package imports
nothing of the library (it shares no code with the CUDA kernels).
"""
from . import phy_oracle  # noqa: F401
