"""The cuFFT comparison baselines (B1 three-stage, B2 row-column) against the
FP64 oracle (needs a GB300).  They are not part of the library; bench.py
times them beside it, and this test makes their numbers meaningful."""

import ctypes
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2110_01172_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sys.path.insert(0, ROOT)
    import bench
    return bench.load_baselines()


@pytest.mark.parametrize("shape", [(2, 2), (64, 128), (256, 256), (512, 64)])
def test_b1_and_b2_match_the_oracle(lib, shape):
    n1, n2 = shape
    x = inputs.uniform(shape, seed=80)
    xd = torch.from_numpy(x).cuda()
    X, Y, back = torch.empty_like(xd), torch.empty_like(xd), torch.empty_like(xd)
    h1, h2 = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.gbdct_b1_create(ctypes.byref(h1), n1, n2) == 0
    assert lib.gbdct_b2_create(ctypes.byref(h2), n1, n2) == 0
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.gbdct_b1_forward(h1, p(xd), p(X), s) == 0
    assert lib.gbdct_b2_forward(h2, p(xd), p(Y), s) == 0
    assert lib.gbdct_b1_inverse(h1, p(X), p(back), s) == 0
    torch.cuda.synchronize()
    ref = oracle.dct2_2d(x)
    for got in (X, Y):
        g = got.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= 1e-5
        assert np.abs(g - ref).max() <= 1e-4 * np.abs(ref).max()
    b = back.cpu().numpy().astype(np.float64)
    assert np.abs(b - x).max() <= 1e-4 * np.abs(x).max()
    lib.gbdct_b1_destroy(h1)
    lib.gbdct_b2_destroy(h2)
