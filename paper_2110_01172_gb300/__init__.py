"""GB300-native (sm_103a) multi-dimensional DCT library.

Implements the three-stage DCT of arXiv 2110.01172 (reorder, real FFT,
twiddle-and-combine, and the mirror-image inverse) in hand-written CUDA
kernels behind the C ABI of include/gbdct.h.  ``binding`` is the Python
argument-marshalling layer over that ABI; ``inputs`` draws the seeded
synthetic workloads.
"""

__version__ = "0.1.0"

from .binding import (Plan, MultiPlan, dct2, idct2, dct3, idct3, dst2, idst2, idct_idxst, idxst_idct,  # noqa: F401,E402
                      PoissonSolver, load, GbdctError)
