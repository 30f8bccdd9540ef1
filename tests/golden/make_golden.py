"""Write the small text fixtures under tests/golden/ from the FP64 oracle only.

Run from the repository root:  python tests/golden/make_golden.py

Fixtures (each a whitespace-separated text matrix with a '#' header that
states its source):

* dct2d_4x4.txt  - 2D DCT-II (Section II-A, Eq. 2d-dct-definition) of the
  4x4 integer ramp x[n1, n2] = 4 n1 + n2, the input size of the paper's
  worked example (Section III-C, Fig. 4; the figure's values are not
  recoverable, so the expected values come from the oracle).
* idct2d_4x4.txt - the exact inverse (Eq. 1b per axis, times 2/N) applied to
  the same integer ramp.
* dct2d_2x8.txt  - 2D DCT-II of a 2x8 +-1 checkerboard.
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def ramp(n1, n2):
    return (np.arange(n1)[:, None] * n2 + np.arange(n2)[None, :]).astype(np.float64)


def checker(n1, n2):
    return ((-1.0) ** (np.arange(n1)[:, None] + np.arange(n2)[None, :])).astype(np.float64)


def write(name, header, arr):
    path = os.path.join(HERE, name)
    np.savetxt(path, arr, fmt="%.17g", header=header)
    print("wrote", path)


def main():
    write("dct2d_4x4.txt",
          "oracle dct2_2d of x[n1,n2]=4*n1+n2 (Section II-A Eq. 2d-dct-definition; "
          "4x4 as in Section III-C Fig. 4)", oracle.dct2_2d(ramp(4, 4)))
    write("idct2d_4x4.txt",
          "oracle idct2_2d of x[n1,n2]=4*n1+n2 (Eq. 1b per axis times 2/N)",
          oracle.idct2_2d(ramp(4, 4)))
    write("dct2d_2x8.txt",
          "oracle dct2_2d of the 2x8 checkerboard (-1)^(n1+n2) (Eq. 2d-dct-definition)",
          oracle.dct2_2d(checker(2, 8)))


if __name__ == "__main__":
    main()
