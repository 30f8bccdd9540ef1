"""GPU parity of the 3D DCT-II / inverse (Section III-D) against the FP64 oracle.

A 3D plan runs the 2D transform of every axis-0 slice (a batched 2D plan) and
a 1D pass along axis 0.  Full comparisons at sizes the oracle finishes in
seconds (every axis-0 length class from 2 to 4096, the 2D slice families seq,
pair and fs2); 128^3 and 256^3 on sampled entries computed one by one, plus
the round trip over the whole array.  Same acceptance as 2D: relative L2
<= 1e-5 and max abs <= 1e-4 max|X|.
"""

import numpy as np
import pytest

import oracle
from paper_2110_01172_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS = 1e-4


def check(got, ref, rel=REL_L2, mabs=MAX_ABS):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    mx = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert err <= rel and mx <= mabs, f"rel-L2 {err:.3e}, max-abs/max {mx:.3e}"


def _plan(shape, batch=1):
    from paper_2110_01172_gb300 import Plan
    return Plan(shape, "dct2", batch=batch)


@pytest.mark.parametrize("shape", [(2, 2, 2), (2, 4, 8), (4, 8, 16), (16, 16, 16), (8, 32, 64),
                                   (64, 16, 32), (128, 16, 8), (32, 256, 256), (1024, 4, 16),
                                   (4096, 2, 4), (512, 64, 2)])
def test_3d_full_oracle(shape):
    x = inputs.uniform(shape, seed=40)
    plan = _plan(shape)
    X = plan.forward(torch.from_numpy(x).cuda())
    y = plan.inverse(X)
    torch.cuda.synchronize()
    Xh = X.cpu().numpy()
    check(Xh, oracle.dct2_3d(x))
    check(y.cpu().numpy(), oracle.idct2_3d(Xh))
    from paper_2110_01172_gb300 import binding
    assert plan.check_device_error() == binding.OK


def _sample3(shape, count, seed):
    rng = np.random.default_rng(seed)
    idx = [list(rng.integers(0, n, count)) for n in shape]
    corners = [[0, n - 1, n // 2, 1] for n in shape]
    return tuple(np.array(i + c) for i, c in zip(idx, corners))


@pytest.mark.parametrize("shape", [(128, 128, 128), (256, 256, 256)])
def test_3d_sampled_entries_and_round_trip(shape):
    x = inputs.uniform(shape, seed=0)
    plan = _plan(shape)
    X = plan.forward(torch.from_numpy(x).cuda())
    y = plan.inverse(X)
    torch.cuda.synchronize()
    Xh, yh = X.cpu().numpy(), y.cpu().numpy()
    k = _sample3(shape, 24, seed=shape[0])
    ref = oracle.dct2_3d_entries(x, *k)
    got = Xh[k].astype(np.float64)
    assert np.abs(got - ref).max() <= MAX_ABS * np.abs(Xh).max()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= REL_L2
    j = _sample3(shape, 8, seed=shape[0] + 1)
    ref_inv = oracle.idct2_3d_entries(Xh, *j)
    assert np.abs(yh[j] - ref_inv).max() <= MAX_ABS * np.abs(yh).max()
    check(yh, x.astype(np.float64))


def test_3d_batched_matches_per_transform_oracle():
    shape, b = (8, 16, 32), 3
    xs = np.stack([inputs.uniform(shape, seed=50 + i) for i in range(b)])
    plan = _plan(shape, batch=b)
    X = plan.forward(torch.from_numpy(xs).cuda())
    y = plan.inverse(X)
    torch.cuda.synchronize()
    for i in range(b):
        check(X[i].cpu().numpy(), oracle.dct2_3d(xs[i]))
        check(y[i].cpu().numpy(), xs[i].astype(np.float64))


def test_3d_in_place_and_module_functions():
    from paper_2110_01172_gb300 import dct3, idct3
    shape = (32, 64, 16)
    x = inputs.uniform(shape, seed=60)
    ref = oracle.dct2_3d(x)
    xd = torch.from_numpy(x).cuda()
    out = dct3(xd)
    plan = _plan(shape)
    plan.forward(xd, out=xd)
    torch.cuda.synchronize()
    check(out.cpu().numpy(), ref)
    assert torch.equal(out, xd)
    back = idct3(out)
    plan.inverse(xd, out=xd)
    torch.cuda.synchronize()
    assert torch.equal(back, xd)
    check(xd.cpu().numpy(), x.astype(np.float64))


def test_3d_single_steps_compose_to_the_full_transform():
    shape = (64, 256, 256)
    plan = _plan(shape)
    assert plan.launches_per_exec >= 3
    x = torch.from_numpy(inputs.uniform(shape, seed=61)).cuda()
    full = plan.forward(x)
    stepped = torch.empty_like(x)
    for k in range(plan.launches_per_exec):
        assert plan.step_name(False, k)
        plan.step(False, k, x, stepped)
    torch.cuda.synchronize()
    assert torch.equal(full, stepped)
    back = torch.empty_like(x)
    for k in range(plan.launches_per_exec):
        plan.step(True, k, full, back)
    torch.cuda.synchronize()
    assert torch.equal(back, plan.inverse(full))
