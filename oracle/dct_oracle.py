"""FP64 direct-sum oracle for 2D/3D DCT-II, its inverse, DST-II and IDXST.

Test infrastructure only (see the package docstring): never imported by the
GPU library.  Parity is checked against these functions, so each is written as
the plain definition it follows, in float64, with no FFT, no blocking and no
fusion.  Inputs of any real dtype are up-cast to float64 first.

Angle evaluation.  A table entry cos(pi * m / (2N)) is evaluated with the
integer m reduced modulo 4N first, so every angle handed to ``numpy.cos`` lies
in [0, 2*pi) and large products (2n+1)*k cannot lose precision.

Scaling conventions (the paper is loose about constants; the readings are):

* Forward DCT-II is exactly the unnormalised sum of Section II-A, Eq. (1a) in
  1D and Eq. (2) ("2d-dct-definition") in 2D:
  X[k1,k2] = sum_{n1,n2} x[n1,n2] cos(pi k1 (2 n1 + 1) / (2 N1))
                                  cos(pi k2 (2 n2 + 1) / (2 N2)).
* The inverse is the paper's IDCT (DCT-III, Eq. (1b)) applied per axis and
  multiplied by 2/N per axis, which makes it the exact inverse of the forward
  transform (Eq. (1b) composed with Eq. (1a) alone gives N/2 times the input).
* IDXST follows Section V-B, Eq. (idxst): IDXST(x)_k = (-1)^k IDCT({x_{N-n}})_k
  with x_N = 0, using the same (2/N-scaled) IDCT.  Its closed form is
  (2/N) sum_{m=1}^{N-1} x_m sin(pi m (2k+1) / (2N)).
* DST-II is not defined in the paper; the standard unnormalised analogue
  X_k = sum_n x_n sin(pi (2n+1)(k+1) / (2N)) is used, with its exact inverse.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "dct2_matrix", "dct3_inverse_matrix", "dst2_matrix", "dst2_inverse_matrix",
    "idxst_matrix", "dct2_1d", "idct_1d", "idxst_1d", "dct2_2d", "idct2_2d",
    "dst2_2d", "idst2_2d", "idct_idxst", "idxst_idct", "dct2_3d", "idct2_3d",
    "dct2_3d_entries", "idct2_3d_entries",
    "dct2_2d_entries", "idct2_2d_entries", "poisson_solve", "compress_threshold",
]


# ---------------------------------------------------------------------------
# 1D transform matrices (rows index the output, columns the input)
# ---------------------------------------------------------------------------

def _cos_half(m: np.ndarray, n: int) -> np.ndarray:
    """cos(pi * m / (2n)) for integer m, with m reduced modulo 4n first."""
    m = np.mod(m.astype(np.int64), 4 * n)
    return np.cos(np.pi * m.astype(np.float64) / (2.0 * n))


def _sin_half(m: np.ndarray, n: int) -> np.ndarray:
    """sin(pi * m / (2n)) for integer m, with m reduced modulo 4n first."""
    m = np.mod(m.astype(np.int64), 4 * n)
    return np.sin(np.pi * m.astype(np.float64) / (2.0 * n))


def dct2_matrix(n: int) -> np.ndarray:
    """DCT-II matrix C[k, j] = cos(pi k (2j+1) / (2n)) (Section II-A, Eq. 1a)."""
    k = np.arange(n, dtype=np.int64)[:, None]
    j = np.arange(n, dtype=np.int64)[None, :]
    return _cos_half((2 * j + 1) * k, n)


def dct3_inverse_matrix(n: int) -> np.ndarray:
    """Exact inverse of ``dct2_matrix(n)``: the paper's IDCT (Eq. 1b) times 2/n.

    D[j, k] = (2/n) w_k cos(pi k (2j+1) / (2n)), w_0 = 1/2, w_k = 1 otherwise.
    Eq. 1b weights the k = 0 term by 1/2 and the others by 1; the 2/n factor
    turns IDCT(DCT(x)) = (n/2) x into the identity.
    """
    j = np.arange(n, dtype=np.int64)[:, None]
    k = np.arange(n, dtype=np.int64)[None, :]
    w = np.ones(n)
    w[0] = 0.5
    return (2.0 / n) * _cos_half((2 * j + 1) * k, n) * w[None, :]


def idxst_matrix(n: int) -> np.ndarray:
    """IDXST matrix of Section V-B, Eq. (idxst), with the 2/n-scaled IDCT.

    IDXST(x)_k = (-1)^k IDCT({x_{n-m}})_k with x_n = 0.  Substituting
    m -> n - m turns (-1)^k cos(pi (n-m)(2k+1)/(2n)) into
    sin(pi m (2k+1)/(2n)), so T[k, m] = (2/n) sin(pi m (2k+1)/(2n)) for m >= 1
    and T[k, 0] = 0 (x_0 is dropped because it lands on x_n = 0).
    """
    k = np.arange(n, dtype=np.int64)[:, None]
    m = np.arange(n, dtype=np.int64)[None, :]
    t = (2.0 / n) * _sin_half(m * (2 * k + 1), n)
    t[:, 0] = 0.0
    return t


def dst2_matrix(n: int) -> np.ndarray:
    """DST-II matrix S[k, j] = sin(pi (2j+1)(k+1) / (2n)) (not in the paper)."""
    k = np.arange(n, dtype=np.int64)[:, None]
    j = np.arange(n, dtype=np.int64)[None, :]
    return _sin_half((2 * j + 1) * (k + 1), n)


def dst2_inverse_matrix(n: int) -> np.ndarray:
    """Exact inverse of ``dst2_matrix(n)`` (a scaled DST-III).

    E[j, k] = (2/n) w_k sin(pi (2j+1)(k+1) / (2n)), w_{n-1} = 1/2, else 1:
    the rows of S are orthogonal with squared norm n/2, except the last
    (k = n-1, entries +-1) whose squared norm is n.
    """
    j = np.arange(n, dtype=np.int64)[:, None]
    k = np.arange(n, dtype=np.int64)[None, :]
    w = np.ones(n)
    w[n - 1] = 0.5
    return (2.0 / n) * _sin_half((2 * j + 1) * (k + 1), n) * w[None, :]


def _f64(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float64)


# ---------------------------------------------------------------------------
# 1D transforms along the last axis
# ---------------------------------------------------------------------------

def dct2_1d(x) -> np.ndarray:
    """Unnormalised DCT-II along the last axis (Eq. 1a)."""
    x = _f64(x)
    return x @ dct2_matrix(x.shape[-1]).T


def idct_1d(x) -> np.ndarray:
    """Exact inverse of ``dct2_1d`` along the last axis (Eq. 1b times 2/N)."""
    x = _f64(x)
    return x @ dct3_inverse_matrix(x.shape[-1]).T


def idxst_1d(x) -> np.ndarray:
    """IDXST along the last axis (Section V-B, Eq. idxst)."""
    x = _f64(x)
    return x @ idxst_matrix(x.shape[-1]).T


# ---------------------------------------------------------------------------
# 2D transforms: separable products A0 @ x @ A1^T (axis 0 = N1, axis 1 = N2)
# ---------------------------------------------------------------------------

def _sep2(a0: np.ndarray, x: np.ndarray, a1: np.ndarray) -> np.ndarray:
    return a0 @ x @ a1.T


def dct2_2d(x) -> np.ndarray:
    """2D DCT-II, Eq. (2d-dct-definition): X = C_{N1} x C_{N2}^T."""
    x = _f64(x)
    n1, n2 = x.shape
    return _sep2(dct2_matrix(n1), x, dct2_matrix(n2))


def idct2_2d(x) -> np.ndarray:
    """Exact inverse of ``dct2_2d``: per-axis IDCT (Eq. 1b) times (2/N1)(2/N2)."""
    x = _f64(x)
    n1, n2 = x.shape
    return _sep2(dct3_inverse_matrix(n1), x, dct3_inverse_matrix(n2))


def dst2_2d(x) -> np.ndarray:
    """2D DST-II (separable sine analogue of the 2D DCT-II)."""
    x = _f64(x)
    n1, n2 = x.shape
    return _sep2(dst2_matrix(n1), x, dst2_matrix(n2))


def idst2_2d(x) -> np.ndarray:
    """Exact inverse of ``dst2_2d``."""
    x = _f64(x)
    n1, n2 = x.shape
    return _sep2(dst2_inverse_matrix(n1), x, dst2_inverse_matrix(n2))


def idct_idxst(x) -> np.ndarray:
    """IDCT_IDXST of Section V-B: IDCT on axis 0 (length N1), IDXST on axis 1.

    The paper writes IDCT(IDXST(x)^T)^T with the 1D transforms acting on the
    last axis: the inner IDXST acts on axis 1, the outer IDCT (after the
    transpose) on axis 0.  The transform is separable, so the order of the
    two axes does not matter.
    """
    x = _f64(x)
    n1, n2 = x.shape
    return _sep2(dct3_inverse_matrix(n1), x, idxst_matrix(n2))


def idxst_idct(x) -> np.ndarray:
    """IDXST_IDCT of Section V-B: IDXST on axis 0 (length N1), IDCT on axis 1."""
    x = _f64(x)
    n1, n2 = x.shape
    return _sep2(idxst_matrix(n1), x, dct3_inverse_matrix(n2))


def dct2_2d_entries(x, k1, k2) -> np.ndarray:
    """Selected entries X[k1[i], k2[i]] of ``dct2_2d(x)``, one direct sum each.

    Used to check very large transforms where the full oracle is too slow:
    each entry is sum_{n1,n2} x[n1,n2] c1[n1] c2[n2] with the cosine rows of
    Eq. (2d-dct-definition).
    """
    x = _f64(x)
    n1, n2 = x.shape
    k1 = np.asarray(k1, dtype=np.int64)
    k2 = np.asarray(k2, dtype=np.int64)
    j1 = np.arange(n1, dtype=np.int64)
    j2 = np.arange(n2, dtype=np.int64)
    out = np.empty(k1.shape[0])
    for i in range(k1.shape[0]):
        c1 = _cos_half((2 * j1 + 1) * k1[i], n1)
        c2 = _cos_half((2 * j2 + 1) * k2[i], n2)
        out[i] = c1 @ x @ c2
    return out


def idct2_2d_entries(x, n1_idx, n2_idx) -> np.ndarray:
    """Selected entries of ``idct2_2d(x)``, one direct sum each."""
    x = _f64(x)
    n1, n2 = x.shape
    n1_idx = np.asarray(n1_idx, dtype=np.int64)
    n2_idx = np.asarray(n2_idx, dtype=np.int64)
    d1 = dct3_inverse_matrix(n1)
    d2 = dct3_inverse_matrix(n2)
    out = np.empty(n1_idx.shape[0])
    for i in range(n1_idx.shape[0]):
        out[i] = d1[n1_idx[i]] @ x @ d2[n2_idx[i]]
    return out


# ---------------------------------------------------------------------------
# 3D (Section III-D: separable along every axis, any order)
# ---------------------------------------------------------------------------

def dct2_3d(x) -> np.ndarray:
    """3D DCT-II: the 1D DCT-II (Eq. 1a) applied along each of the three axes."""
    x = _f64(x)
    n0, n1, n2 = x.shape
    return np.einsum("ai,bj,ck,ijk->abc", dct2_matrix(n0), dct2_matrix(n1),
                     dct2_matrix(n2), x, optimize=True)


def idct2_3d(x) -> np.ndarray:
    """Exact inverse of ``dct2_3d`` (per-axis 2/N-scaled IDCT of Eq. 1b)."""
    x = _f64(x)
    n0, n1, n2 = x.shape
    return np.einsum("ai,bj,ck,ijk->abc", dct3_inverse_matrix(n0),
                     dct3_inverse_matrix(n1), dct3_inverse_matrix(n2), x,
                     optimize=True)


def dct2_3d_entries(x, k0, k1, k2) -> np.ndarray:
    """Entries X[k0[i], k1[i], k2[i]] of ``dct2_3d(x)``, each as the triple sum
    of x against the three cosine rows (for sizes too large for the full map)."""
    x = _f64(x)
    n0, n1, n2 = x.shape
    c0, c1, c2 = dct2_matrix(n0), dct2_matrix(n1), dct2_matrix(n2)
    return np.array([np.einsum("i,j,k,ijk->", c0[a], c1[b], c2[c], x, optimize=True)
                     for a, b, c in zip(k0, k1, k2)])


def idct2_3d_entries(x, n0_idx, n1_idx, n2_idx) -> np.ndarray:
    """Entries of ``idct2_3d(x)`` at the given positions, as triple sums."""
    x = _f64(x)
    n0, n1, n2 = x.shape
    d0, d1, d2 = dct3_inverse_matrix(n0), dct3_inverse_matrix(n1), dct3_inverse_matrix(n2)
    return np.array([np.einsum("i,j,k,ijk->", d0[a], d1[b], d2[c], x, optimize=True)
                     for a, b, c in zip(n0_idx, n1_idx, n2_idx)])


# ---------------------------------------------------------------------------
# Applications (Section V)
# ---------------------------------------------------------------------------

def poisson_solve(rho):
    """Spectral Neumann Poisson solve of Section V-B, Algorithm 4.

    The paper only says "scaled electric potential a1, a2 based on a"; the
    reading used here is the grid-unit eigen-frequencies w_u = pi u / N1 and
    w_v = pi v / N2 of the cosine basis cos(pi u (n + 1/2) / N):

      a       = DCT2(rho)                                  (Algorithm 4, line 2)
      phi_uv  = a_uv / (w_u^2 + w_v^2), phi_00 = 0
      psi     = IDCT2(phi)                                 (potential)
      xi_0    = IDXST_IDCT(a_uv w_u / (w_u^2 + w_v^2))      (field along axis 0)
      xi_1    = IDCT_IDXST(a_uv w_v / (w_u^2 + w_v^2))      (field along axis 1)

    Returns (psi, xi_0, xi_1), each N1 x N2 float64.
    """
    rho = _f64(rho)
    n1, n2 = rho.shape
    a = dct2_2d(rho)
    wu = np.pi * np.arange(n1, dtype=np.float64) / n1
    wv = np.pi * np.arange(n2, dtype=np.float64) / n2
    den = wu[:, None] ** 2 + wv[None, :] ** 2
    den[0, 0] = 1.0
    inv = 1.0 / den
    inv[0, 0] = 0.0
    phi = a * inv
    psi = idct2_2d(phi)
    xi0 = idxst_idct(a * wu[:, None] * inv)
    xi1 = idct_idxst(a * wv[None, :] * inv)
    return psi, xi0, xi1


def compress_threshold(b, eps: float) -> np.ndarray:
    """Magnitude threshold f_eps of Section V-A, Eq. (image-compression)."""
    b = _f64(b)
    return np.where(np.abs(b) >= eps, b, 0.0)
