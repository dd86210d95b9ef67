"""CPU FP64 oracle of the HyperNetVec V-cycle.

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg; never by the library."""
from .hnv_oracle import *  # noqa: F401,F403
