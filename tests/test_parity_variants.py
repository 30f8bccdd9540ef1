"""GPU parity of the DST-II and IDXST kinds against the FP64 oracle.

DST-II is not defined in the paper; the oracle's sine analogue is pinned on
the CPU by DST-II(x)_k = DCT-II((-1)^n x)_{N-1-k} and scipy.  IDCT_IDXST and
IDXST_IDCT follow Section V-B, Eq. (idxst), with the 2/N-scaled IDCT.
"""

import numpy as np
import pytest

import oracle
from paper_2110_01172_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2, MAX_ABS = 1e-5, 1e-4


def check(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= REL_L2 and mx <= MAX_ABS, (err, mx)


SHAPES = [(2, 2), (8, 16), (16, 4), (64, 32), (128, 256), (2048, 2048)]


@pytest.mark.parametrize("shape", SHAPES)
def test_dst2_forward_and_inverse(shape):
    from paper_2110_01172_gb300 import Plan
    x = inputs.uniform(shape, seed=41)
    plan = Plan(shape, "dst2")
    S = plan.forward(torch.from_numpy(x).cuda())
    y = plan.inverse(S)
    torch.cuda.synchronize()
    Sh = S.cpu().numpy()
    check(Sh, oracle.dst2_2d(x))
    check(y.cpu().numpy(), oracle.idst2_2d(Sh))


@pytest.mark.parametrize("kind", ["idct_idxst", "idxst_idct"])
@pytest.mark.parametrize("shape", SHAPES + [(1024, 4096)])
def test_idxst_kinds(kind, shape):
    from paper_2110_01172_gb300 import Plan, binding
    x = inputs.uniform(shape, seed=43)
    plan = Plan(shape, kind)
    y = plan.inverse(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    n1, n2 = shape
    if n1 * n2 <= 2048 * 2048:
        ref = oracle.idct_idxst(x) if kind == "idct_idxst" else oracle.idxst_idct(x)
        check(y.cpu().numpy(), ref)
    else:  # sampled entries of the separable sum
        yh = y.cpu().numpy()
        d1 = oracle.dct3_inverse_matrix(n1) if kind == "idct_idxst" else oracle.idxst_matrix(n1)
        d2 = oracle.idxst_matrix(n2) if kind == "idct_idxst" else oracle.dct3_inverse_matrix(n2)
        rng = np.random.default_rng(1)
        for i, j in zip(rng.integers(0, n1, 12), rng.integers(0, n2, 12)):
            ref = d1[i] @ x.astype(np.float64) @ d2[j]
            assert abs(yh[i, j] - ref) <= MAX_ABS * np.abs(yh).max()
    buf = torch.zeros(shape, device="cuda")
    assert plan.forward_ptr(buf.data_ptr(), buf.data_ptr()) == binding.ERR_UNSUPPORTED
