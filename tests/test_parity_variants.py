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


FOLD_SHAPES = [(256, 256), (512, 256), (256, 1024), (1024, 512), (256, 16384), (2048, 512), (512, 2048)]
LAUNCHES = {"fs2": 3, "tp": 2, "pair": 4}


@pytest.mark.parametrize("family", ["fs2", "tp", "pair"])
@pytest.mark.parametrize("shape", FOLD_SHAPES)
def test_kinds_folded_and_mapped_paths(family, shape):
    """fs2 and tp fold each kind's index/sign maps into their first loads and
    last stores; pair runs the map kernels around the DCT-II.  All against the
    oracle, for every kind, forward and inverse where defined."""
    from paper_2110_01172_gb300 import Plan
    if family == "pair" and max(shape) > 8192:
        pytest.skip("pair supports sides up to 8192")
    if family == "tp" and not (shape[0] >= 128 and shape[1] <= 8192):
        pytest.skip("tp supports N1 >= 128, N2 <= 8192")
    x = inputs.uniform(shape, seed=44)
    xd = torch.from_numpy(x).cuda()
    p = Plan(shape, "dst2", family=family)
    assert p.family == family
    assert p.launches_per_exec == LAUNCHES[family]
    S = p.forward(xd)
    back = p.inverse(S)
    torch.cuda.synchronize()
    Sh = S.cpu().numpy()
    check(Sh, oracle.dst2_2d(x))
    check(back.cpu().numpy(), oracle.idst2_2d(Sh))
    for kind, ref in (("idct_idxst", oracle.idct_idxst), ("idxst_idct", oracle.idxst_idct)):
        q = Plan(shape, kind, family=family)
        y = q.inverse(xd)
        torch.cuda.synchronize()
        check(y.cpu().numpy(), ref(x))


def test_folded_kinds_batched_and_in_place():
    from paper_2110_01172_gb300 import Plan
    shape = (512, 1024)
    xs = np.stack([inputs.uniform(shape, seed=45 + i) for i in range(3)])
    p = Plan(shape, "dst2", batch=3)
    assert p.family == "tp"            # the default family folds the maps in
    xd = torch.from_numpy(xs).cuda()
    S = p.forward(xd)
    torch.cuda.synchronize()
    for i in range(3):
        check(S[i].cpu().numpy(), oracle.dst2_2d(xs[i]))
    p.inverse(S, out=S)
    torch.cuda.synchronize()
    for i in range(3):
        check(S[i].cpu().numpy(), xs[i])
    q = Plan(shape, "idxst_idct", batch=3)
    y = xd.clone()
    q.inverse(y, out=y)
    torch.cuda.synchronize()
    for i in range(3):
        check(y[i].cpu().numpy(), oracle.idxst_idct(xs[i]))
