"""FP64 CPU oracle for LocalPower.  TEST INFRASTRUCTURE ONLY: imported by the
tests, the smoke check and the benchmark's CPU-baseline leg, never by the product."""
from .fp64 import *  # noqa: F401,F403
