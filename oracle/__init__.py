"""FP64 CPU oracle for the multi-dimensional DCT family (test infrastructure).

This package is test infrastructure, not part of the library.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the GPU library never does, and this package imports nothing from
the GPU library.

Every function is a plain, slow, obviously-correct restatement of a definition
from arXiv 2110.01172 ("A New Acceleration Paradigm for Discrete Cosine
Transform and Other Fourier-Related Transforms"), evaluated as separable dense
direct sums in float64.  None of them uses an FFT.
"""

from .dct_oracle import (  # noqa: F401
    dct2_matrix,
    dct3_inverse_matrix,
    dst2_matrix,
    dst2_inverse_matrix,
    idxst_matrix,
    dct2_1d,
    idct_1d,
    idxst_1d,
    dct2_2d,
    idct2_2d,
    dst2_2d,
    idst2_2d,
    idct_idxst,
    idxst_idct,
    dct2_3d,
    idct2_3d,
    dct2_3d_entries,
    idct2_3d_entries,
    dct2_2d_entries,
    idct2_2d_entries,
    poisson_solve,
    compress_threshold,
)
