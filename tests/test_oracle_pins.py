"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test checks the oracle against something it does not share code with:
brute-force scalar sums written with ``math.cos``, closed forms (constant
input, cosine basis images), invariants (round trip, Parseval under the
orthonormal weights), library routines in special cases (``scipy.fft``), the
identities that define IDXST and relate DST-II to DCT-II, and FFT-based
restatements of the paper's own Algorithms 1 and 2.  A plausible slip in the
oracle (a dropped weight, a wrong sign or index, a transposed operand, a
missing 2/N) fails at least one of them.
"""

import math

import numpy as np
import pytest
import scipy.fft

import oracle
from paper_2110_01172_gb300 import inputs

SMALL_SHAPES = [(1, 1), (1, 5), (2, 3), (3, 2), (4, 4), (5, 6), (7, 3), (8, 8), (6, 1)]


def _brute_dct2d(x):
    """Quadruple loop of Eq. (2d-dct-definition) with math.cos, no tables."""
    n1, n2 = x.shape
    out = np.zeros((n1, n2))
    for k1 in range(n1):
        for k2 in range(n2):
            acc = 0.0
            for a in range(n1):
                for b in range(n2):
                    acc += (float(x[a, b]) * math.cos(math.pi / n1 * (a + 0.5) * k1)
                            * math.cos(math.pi / n2 * (b + 0.5) * k2))
            out[k1, k2] = acc
    return out


def _brute_idct2d(X):
    """Quadruple loop of Eq. (1b) per axis times (2/N1)(2/N2)."""
    n1, n2 = X.shape
    out = np.zeros((n1, n2))
    for a in range(n1):
        for b in range(n2):
            acc = 0.0
            for k1 in range(n1):
                w1 = 0.5 if k1 == 0 else 1.0
                for k2 in range(n2):
                    w2 = 0.5 if k2 == 0 else 1.0
                    acc += (w1 * w2 * float(X[k1, k2])
                            * math.cos(math.pi / n1 * k1 * (a + 0.5))
                            * math.cos(math.pi / n2 * k2 * (b + 0.5)))
            out[a, b] = acc * (2.0 / n1) * (2.0 / n2)
    return out


@pytest.mark.parametrize("shape", SMALL_SHAPES)
def test_dct2d_matches_bruteforce(shape):
    x = inputs.uniform(shape, seed=11)
    ref = _brute_dct2d(x)
    got = oracle.dct2_2d(x)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("shape", SMALL_SHAPES)
def test_idct2d_matches_bruteforce(shape):
    X = inputs.uniform(shape, seed=12)
    ref = _brute_idct2d(X)
    got = oracle.idct2_2d(X)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("shape", [(4, 4), (8, 16), (5, 7), (32, 2)])
def test_constant_input_gives_dc_only(shape):
    c = 0.75
    X = oracle.dct2_2d(np.full(shape, c))
    assert X[0, 0] == pytest.approx(c * shape[0] * shape[1], rel=1e-14)
    rest = X.copy()
    rest[0, 0] = 0.0
    assert np.abs(rest).max() < 1e-12


@pytest.mark.parametrize("shape,p,q", [((8, 8), 3, 5), ((16, 4), 0, 2), ((6, 10), 5, 0),
                                       ((4, 4), 0, 0), ((7, 9), 6, 8)])
def test_cosine_basis_gives_single_delta(shape, p, q):
    n1, n2 = shape
    a = np.arange(n1)[:, None]
    b = np.arange(n2)[None, :]
    x = np.cos(np.pi * p * (2 * a + 1) / (2 * n1)) * np.cos(np.pi * q * (2 * b + 1) / (2 * n2))
    X = oracle.dct2_2d(x)
    amp = (n1 / 2) * (n2 / 2) * (2 if p == 0 else 1) * (2 if q == 0 else 1)
    expect = np.zeros(shape)
    expect[p, q] = amp
    np.testing.assert_allclose(X, expect, atol=1e-11 * amp)


@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (3, 5), (16, 8), (31, 64), (128, 128)])
def test_round_trip(shape):
    x = inputs.uniform(shape, seed=3).astype(np.float64)
    np.testing.assert_allclose(oracle.idct2_2d(oracle.dct2_2d(x)), x, atol=1e-12)
    np.testing.assert_allclose(oracle.dct2_2d(oracle.idct2_2d(x)), x, atol=1e-11 * max(shape) ** 2)


@pytest.mark.parametrize("shape", [(4, 4), (9, 6), (64, 32)])
def test_parseval_orthonormal(shape):
    n1, n2 = shape
    x = inputs.uniform(shape, seed=4).astype(np.float64)
    X = oracle.dct2_2d(x)
    w1 = np.full(n1, np.sqrt(2.0 / n1))
    w1[0] = np.sqrt(1.0 / n1)
    w2 = np.full(n2, np.sqrt(2.0 / n2))
    w2[0] = np.sqrt(1.0 / n2)
    Xo = X * w1[:, None] * w2[None, :]
    assert np.linalg.norm(Xo) == pytest.approx(np.linalg.norm(x), rel=1e-13)


@pytest.mark.parametrize("shape", [(8, 8), (5, 12), (256, 256), (64, 128)])
def test_matches_scipy_dctn_special_case(shape):
    # scipy's unnormalised type-2 DCT is 2 sum x cos(...) per axis: 4x ours in 2D.
    x = inputs.uniform(shape, seed=5).astype(np.float64)
    X = oracle.dct2_2d(x)
    np.testing.assert_allclose(scipy.fft.dctn(x, type=2), 4.0 * X, atol=1e-10 * np.abs(X).max())
    # scipy's type-3 DCT is x_0 + 2 sum_{k>=1} x_k cos(...): (N/2)... per axis.
    Y = oracle.idct2_2d(x)
    np.testing.assert_allclose(scipy.fft.dctn(x, type=3) / (shape[0] * shape[1]), Y, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 13, 64])
def test_dst2_identity_and_scipy(n):
    x = inputs.uniform((n,), seed=6).astype(np.float64)
    S = oracle.dst2_matrix(n) @ x
    # DST-II(x)_k = DCT-II((-1)^j x_j)_{N-1-k}
    alt = x * (-1.0) ** np.arange(n)
    np.testing.assert_allclose(S, oracle.dct2_1d(alt)[::-1], atol=1e-12 * n)
    np.testing.assert_allclose(scipy.fft.dst(x, type=2), 2.0 * S, atol=1e-12 * n)
    np.testing.assert_allclose(oracle.dst2_inverse_matrix(n) @ S, x, atol=1e-12 * n)


@pytest.mark.parametrize("shape", [(4, 4), (6, 10), (32, 16)])
def test_dst2_2d_round_trip(shape):
    x = inputs.uniform(shape, seed=7).astype(np.float64)
    np.testing.assert_allclose(oracle.idst2_2d(oracle.dst2_2d(x)), x, atol=1e-12)
    np.testing.assert_allclose(oracle.dst2_2d(x), scipy.fft.dstn(x, type=2) / 4.0, atol=1e-10)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 16, 33])
def test_idxst_definition(n):
    # Eq. (idxst): IDXST(x)_k = (-1)^k IDCT({x_{N-j}})_k with x_N = 0.
    x = inputs.uniform((n,), seed=8).astype(np.float64)
    rev = np.zeros(n)
    rev[1:] = x[::-1][:-1]          # rev[j] = x[N - j] for j >= 1, rev[0] = x_N = 0
    expect = (-1.0) ** np.arange(n) * oracle.idct_1d(rev)
    np.testing.assert_allclose(oracle.idxst_1d(x), expect, atol=1e-12 * n)


@pytest.mark.parametrize("shape", [(4, 8), (8, 4), (16, 16), (3, 5)])
def test_mixed_transforms_match_nested_1d_definitions(shape):
    # IDCT_IDXST(x) = IDCT(IDXST(x)^T)^T with 1D maps on the last axis.
    x = inputs.uniform(shape, seed=9).astype(np.float64)
    nested = oracle.idct_1d(oracle.idxst_1d(x).T).T
    np.testing.assert_allclose(oracle.idct_idxst(x), nested, atol=1e-12)
    nested2 = oracle.idxst_1d(oracle.idct_1d(x).T).T
    np.testing.assert_allclose(oracle.idxst_idct(x), nested2, atol=1e-12)


# ---------------------------------------------------------------------------
# The paper's algorithms restated with numpy.fft pin the oracle's scalings
# ---------------------------------------------------------------------------

def _alg1_variants(x):
    """The four 1D DCT-via-RFFT algorithms of Algorithm 1 (as printed)."""
    n = x.shape[0]
    j = np.arange(n)
    ph = np.exp(-1j * np.pi * j / (2 * n))
    # 4N-point: x at odd positions, mirrored in the upper half, zeros at even.
    x4 = np.zeros(4 * n)
    x4[1:2 * n:2] = x
    x4[2 * n + 1::2] = x[::-1]
    y4 = np.fft.rfft(x4)[:n].real
    # mirrored 2N-point.
    y2m = (ph * np.fft.rfft(np.concatenate([x, x[::-1]]))[:n]).real
    # zero-padded 2N-point.
    y2p = 2 * (ph * np.fft.rfft(np.concatenate([x, np.zeros(n)]))[:n]).real
    # N-point with the even/odd reorder of Eq. (n_pre) and Eq. (n_post).
    v = np.empty(n)
    half = (n - 1) // 2
    v[:half + 1] = x[0::2][:half + 1]
    v[half + 1:] = x[2 * n - 2 * np.arange(half + 1, n) - 1]
    yn = 2 * (ph * np.fft.fft(v)).real
    # Hermitian form of Eq. (n_post_update): upper half from conj X(N - j).
    F = np.fft.fft(v)
    yh = np.empty(n)
    for k in range(n):
        if k <= math.ceil((n - 1) / 2):
            yh[k] = 2 * (ph[k] * F[k]).real
        else:
            yh[k] = 2 * (ph[k] * np.conj(F[n - k])).real
    return y4, y2m, y2p, yn, yh


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 15, 64])
def test_algorithm1_variants_equal_twice_eq1a(n):
    # Every Algorithm 1 variant, as printed, returns 2x Eq. (1a); the oracle
    # follows Eq. (1a), the definition the benchmark configuration fixes.
    x = inputs.uniform((n,), seed=10).astype(np.float64)
    ref = oracle.dct2_1d(x)
    for y in _alg1_variants(x):
        np.testing.assert_allclose(y / 2.0, ref, atol=1e-12 * max(1, n))


def _reorder_2d(x):
    """Eq. (2d_dct_pre): v(n1, n2) = x(s1(n1), s2(n2))."""
    n1, n2 = x.shape

    def sigma(n, N):
        return 2 * n if n <= (N - 1) // 2 else 2 * N - 2 * n - 1

    i1 = np.array([sigma(a, n1) for a in range(n1)])
    i2 = np.array([sigma(b, n2) for b in range(n2)])
    return x[np.ix_(i1, i2)], i1, i2


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (4, 4), (5, 6), (7, 3), (8, 16), (16, 2)])
def test_algorithm2_three_stage_reading(shape):
    """Algorithm 2 with the reading used by the GPU path equals the oracle.

    Reading: y = (1/2) Re(b (a X(n1,n2) + conj(a) X((N1-n1) mod N1, n2))), i.e.
    factor 1/2 instead of the printed 2 and a periodic index instead of
    X(N1, .) = 0.  The printed form (factor 2, X(N1, .) = 0) gives 4x the
    definition for n1 >= 1 and 2x on row 0; both facts are asserted.
    """
    n1, n2 = shape
    x = inputs.uniform(shape, seed=13).astype(np.float64)
    v, _, _ = _reorder_2d(x)
    V = np.fft.fft2(v)
    k1 = np.arange(n1)[:, None]
    k2 = np.arange(n2)[None, :]
    a = np.exp(-1j * np.pi * k1 / (2 * n1))
    b = np.exp(-1j * np.pi * k2 / (2 * n2))
    Q = V[(-np.arange(n1)) % n1, :]
    y = 0.5 * (b * (a * V + np.conj(a) * Q)).real
    ref = oracle.dct2_2d(x)
    np.testing.assert_allclose(y, ref, atol=1e-12 * max(1.0, np.abs(ref).max()))
    # The printed convention X(N1, .) = 0 with factor 2.
    Qz = np.zeros_like(V)
    Qz[1:, :] = V[n1 - np.arange(1, n1), :]
    yp = 2 * (b * (a * V + np.conj(a) * Qz)).real
    np.testing.assert_allclose(yp[1:, :], 4 * ref[1:, :], atol=1e-11 * max(1.0, np.abs(ref).max()))
    np.testing.assert_allclose(yp[0, :], 2 * ref[0, :], atol=1e-11 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (4, 4), (5, 6), (8, 16), (16, 2), (3, 7)])
def test_algorithm2_inverse_reading(shape):
    """2D IDCT of Algorithm 2 with the conjugated twiddle equals the oracle.

    Reading: V(k1,k2) = conj(a) conj(b) [C(k1,k2) - C(N1-k1,N2-k2)
    - j (C(N1-k1,k2) + C(k1,N2-k2))], C(N1,.) = C(.,N2) = 0, then the inverse
    2D DFT (with its 1/(N1 N2)) and the inverse reorder of Eq. (2d_idct_post).
    The printed twiddle e^{-j...} does not reconstruct the input; asserted too.
    """
    n1, n2 = shape
    C = inputs.uniform(shape, seed=14).astype(np.float64)
    Cp = np.zeros((n1 + 1, n2 + 1))
    Cp[:n1, :n2] = C
    k1 = np.arange(n1)[:, None]
    k2 = np.arange(n2)[None, :]
    r1 = n1 - k1
    r2 = n2 - k2
    br = Cp[k1, k2] - Cp[r1, r2] - 1j * (Cp[r1, k2] + Cp[k1, r2])
    a = np.exp(-1j * np.pi * k1 / (2 * n1))
    b = np.exp(-1j * np.pi * k2 / (2 * n2))
    v = np.fft.ifft2(np.conj(a) * np.conj(b) * br).real
    _, i1, i2 = _reorder_2d(np.zeros(shape))
    y = np.empty(shape)
    y[np.ix_(i1, i2)] = v
    ref = oracle.idct2_2d(C)
    np.testing.assert_allclose(y, ref, atol=1e-12)
    if n1 * n2 > 1:
        vp = np.fft.ifft2(a * b * br).real
        yp = np.empty(shape)
        yp[np.ix_(i1, i2)] = vp
        assert np.abs(yp - ref).max() > 1e-3


def test_hermitian_pairs_of_the_paper_examples():
    # Section II-C footnote: N=5 pairs (1,4),(2,3); N=6 pairs (1,5),(2,4),(3,3).
    for n, pairs in ((5, [(1, 4), (2, 3)]), (6, [(1, 5), (2, 4), (3, 3)])):
        F = np.fft.fft(inputs.uniform((n,), seed=n).astype(np.float64))
        for p, q in pairs:
            assert F[p] == pytest.approx(np.conj(F[q]), abs=1e-12)
        assert len(np.fft.rfft(np.zeros(n))) == math.ceil((n + 1) / 2)


# ---------------------------------------------------------------------------
# Large-size helpers, 3D and applications
# ---------------------------------------------------------------------------

def test_entries_helpers_match_full_oracle():
    x = inputs.uniform((64, 32), seed=15)
    X = oracle.dct2_2d(x)
    k1 = np.array([0, 1, 63, 17, 32])
    k2 = np.array([0, 31, 5, 16, 0])
    np.testing.assert_allclose(oracle.dct2_2d_entries(x, k1, k2), X[k1, k2], atol=1e-12)
    Y = oracle.idct2_2d(x)
    np.testing.assert_allclose(oracle.idct2_2d_entries(x, k1, k2), Y[k1, k2], atol=1e-12)


def test_dct3d_bruteforce_and_round_trip():
    x = inputs.uniform((3, 4, 2), seed=16)
    n0, n1, n2 = x.shape
    ref = np.zeros(x.shape)
    for k0 in range(n0):
        for k1 in range(n1):
            for k2 in range(n2):
                acc = 0.0
                for a in range(n0):
                    for b in range(n1):
                        for c in range(n2):
                            acc += (float(x[a, b, c]) * math.cos(math.pi / n0 * (a + 0.5) * k0)
                                    * math.cos(math.pi / n1 * (b + 0.5) * k1)
                                    * math.cos(math.pi / n2 * (c + 0.5) * k2))
                ref[k0, k1, k2] = acc
    np.testing.assert_allclose(oracle.dct2_3d(x), ref, atol=1e-12)
    y = inputs.uniform((8, 4, 16), seed=17).astype(np.float64)
    np.testing.assert_allclose(oracle.idct2_3d(oracle.dct2_3d(y)), y, atol=1e-12)


def test_3d_entries_helpers_match_brute_force_pinned_full_maps():
    """The single-entry 3D helpers against the full maps (pinned above by the
    sextuple loop and the round trip), including the corners and row N/2."""
    x = inputs.uniform((8, 4, 16), seed=18)
    X, Y = oracle.dct2_3d(x), oracle.idct2_3d(x)
    k0 = np.array([0, 7, 4, 1, 0, 3])
    k1 = np.array([0, 3, 2, 0, 1, 2])
    k2 = np.array([0, 15, 8, 1, 15, 7])
    np.testing.assert_allclose(oracle.dct2_3d_entries(x, k0, k1, k2), X[k0, k1, k2], atol=1e-11)
    np.testing.assert_allclose(oracle.idct2_3d_entries(x, k0, k1, k2), Y[k0, k1, k2], atol=1e-12)


def test_3d_separable_cosine_is_a_single_delta():
    """cos(pi p (2a+1)/2N0) cos(pi q (2b+1)/2N1) cos(pi r (2c+1)/2N2) maps to one
    nonzero coefficient (N0/2)(N1/2)(N2/2) (doubled per zero index)."""
    n0, n1, n2, p, q, r = 4, 8, 2, 3, 0, 1
    a = np.cos(np.pi * p * (2 * np.arange(n0) + 1) / (2 * n0))
    b = np.cos(np.pi * q * (2 * np.arange(n1) + 1) / (2 * n1))
    c = np.cos(np.pi * r * (2 * np.arange(n2) + 1) / (2 * n2))
    x = np.einsum("i,j,k->ijk", a, b, c)
    X = oracle.dct2_3d(x)
    want = np.zeros_like(X)
    want[p, q, r] = (n0 / 2) * (n1 / 2) * (n2 / 2) * (2 if p == 0 else 1) * (2 if q == 0 else 1) * (2 if r == 0 else 1)
    np.testing.assert_allclose(X, want, atol=1e-12)


def _cos_series(coef, t1, t2):
    """Evaluate sum_uv w c_uv cos(pi u (t1+1/2)/N1) cos(pi v (t2+1/2)/N2) off-grid.

    w = (2/N1)(2/N2) with the 1/2 weights on u = 0 and v = 0, i.e. the
    continuous extension of the inverse transform at real positions t1, t2.
    """
    n1, n2 = coef.shape
    u = np.arange(n1)
    v = np.arange(n2)
    w1 = np.where(u == 0, 0.5, 1.0) * 2.0 / n1
    w2 = np.where(v == 0, 0.5, 1.0) * 2.0 / n2
    c1 = np.cos(np.pi * np.outer(t1 + 0.5, u) / n1) * w1
    c2 = np.cos(np.pi * np.outer(t2 + 0.5, v) / n2) * w2
    return c1 @ coef @ c2.T


def test_poisson_solve_pins():
    shape = (16, 32)
    rho = inputs.density_blobs(shape, seed=1, n_blobs=20).astype(np.float64)
    psi, xi0, xi1 = oracle.poisson_solve(rho)
    n1, n2 = shape
    a = oracle.dct2_2d(rho)
    wu = np.pi * np.arange(n1) / n1
    wv = np.pi * np.arange(n2) / n2
    den = wu[:, None] ** 2 + wv[None, :] ** 2
    phi = np.where(den > 0, a / np.where(den > 0, den, 1.0), 0.0)
    t1 = np.arange(n1, dtype=np.float64)
    t2 = np.arange(n2, dtype=np.float64)
    # the potential is the cosine series of phi at the grid points
    np.testing.assert_allclose(psi, _cos_series(phi, t1, t2), atol=1e-10)
    # field = minus the derivative of the potential series (central differences)
    h = 1e-4
    d0 = (_cos_series(phi, t1 + h, t2) - _cos_series(phi, t1 - h, t2)) / (2 * h)
    d1 = (_cos_series(phi, t1, t2 + h) - _cos_series(phi, t1, t2 - h)) / (2 * h)
    scale = np.abs(xi0).max() + np.abs(xi1).max()
    np.testing.assert_allclose(xi0, -d0, atol=1e-6 * scale)
    np.testing.assert_allclose(xi1, -d1, atol=1e-6 * scale)
    # minus the Laplacian of the potential series is rho minus its mean
    lap = ((_cos_series(phi, t1 + h, t2) + _cos_series(phi, t1 - h, t2)
            + _cos_series(phi, t1, t2 + h) + _cos_series(phi, t1, t2 - h)
            - 4 * _cos_series(phi, t1, t2)) / h ** 2)
    np.testing.assert_allclose(-lap, rho - rho.mean(), atol=2e-3 * np.abs(rho).max())


def test_compress_threshold():
    b = np.array([[-2.0, 0.5], [0.1, -0.09]])
    np.testing.assert_array_equal(oracle.compress_threshold(b, 0.1), [[-2.0, 0.5], [0.1, 0.0]])
