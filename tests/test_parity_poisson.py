"""GPU parity of the spectral Poisson solve (Algorithm 4) against the oracle.

The oracle's solve is itself pinned on the CPU by finite differences of the
continuous cosine series (field = minus the gradient of the potential, minus
the Laplacian = density minus its mean).
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


@pytest.mark.parametrize("shape", [(16, 16), (64, 128), (256, 256), (512, 1024), (2048, 2048)])
def test_poisson_solve_matches_oracle(shape):
    from paper_2110_01172_gb300 import PoissonSolver
    rho = inputs.density_blobs(shape, seed=7, n_blobs=300)
    solver = PoissonSolver(shape)
    psi, xi0, xi1 = solver.solve(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    rpsi, rxi0, rxi1 = oracle.poisson_solve(rho)
    check(psi.cpu().numpy(), rpsi)
    check(xi0.cpu().numpy(), rxi0)
    check(xi1.cpu().numpy(), rxi1)
    assert solver.workspace_bytes > 0
    solver.close()
