"""Continuous-batching Poisson server: host logic on CPU, results on the GPU."""

import numpy as np
import pytest

from paper_2110_01172_gb300 import inputs
from paper_2110_01172_gb300.serving import AdmissionController, request_bytes


def test_admission_controller_budget():
    ac = AdmissionController(100)
    assert ac.try_reserve(60)
    assert not ac.try_reserve(50)      # would exceed the budget: rejected, nothing reserved
    assert ac.reserved == 60
    ac.release(60)
    assert ac.try_reserve(100)
    assert not ac.try_reserve(1)


def test_request_bytes_grows_with_area():
    # 40 bytes per element (plans, staging, denominators, the four arrays) on
    # top of a fixed margin for the graph
    assert request_bytes((128, 128)) - request_bytes((64, 64)) >= 40 * (128 * 128 - 64 * 64)
    assert request_bytes((2048, 2048)) > 160 * 2 ** 20


def test_arrivals_and_shapes_are_seeded():
    a = inputs.poisson_arrivals(50, 1000.0, seed=3)
    assert np.all(np.diff(a) >= 0) and a[0] == 0.0
    assert np.allclose(a, inputs.poisson_arrivals(50, 1000.0, seed=3))
    shapes = inputs.serving_shapes(100, seed=1)
    assert all(64 <= s <= 2048 and (s & (s - 1)) == 0 for sh in shapes for s in sh)


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    torch = pytest.importorskip("torch")
    from paper_2110_01172_gb300.serving import PoissonServer, make_requests, serve_plain
    reqs = make_requests(24, rate_per_s=20000.0, seed=5, lo=64, hi=512)
    server = PoissonServer(slots=6, keep_outputs=True)
    mixed = server.serve(reqs)
    alone = serve_plain(reqs, keep_outputs=True)
    assert [r.rid for r in mixed] == [r.rid for r in alone] == list(range(24))
    for m, a in zip(mixed, alone):
        for x, y in zip(m.outputs, a.outputs):
            assert torch.equal(x, y)   # bitwise: the kernels and plan choice depend only on the shape


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(64, 64), (128, 2048), (256, 256), (2048, 2048)])
def test_admission_charge_covers_what_a_resident_solve_holds(shape):
    """request_bytes (what admission reserves) is at least the measured device
    bytes of a resident solve: solver workspaces and tables, the four arrays
    and what the CUDA-graph capture allocates in its private pool."""
    torch = pytest.importorskip("torch")
    from paper_2110_01172_gb300.serving import _Resources
    res = _Resources(shape, torch.device("cuda", 0), graph=True)
    assert 0 < res.device_bytes <= request_bytes(shape)
    res.close()


@pytest.mark.gpu
def test_server_matches_oracle_on_a_few_requests():
    pytest.importorskip("torch")
    import oracle
    from paper_2110_01172_gb300.serving import PoissonServer, make_requests
    reqs = make_requests(5, rate_per_s=5000.0, seed=9, lo=64, hi=256)
    res = PoissonServer(slots=3, keep_outputs=True).serve(reqs)
    for r, q in zip(res, reqs):
        ref = oracle.poisson_solve(q.rho.numpy())
        for got, want in zip(r.outputs, ref):
            got = got.numpy().astype(np.float64)
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5
