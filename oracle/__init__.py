"""Serial CPU oracle of the swap-sweep method (plain C behind ctypes).

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
CPU-baseline leg may import this package.  The product library never calls
it and shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
