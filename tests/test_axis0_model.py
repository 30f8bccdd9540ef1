"""Data layout and arithmetic of the packed axis-0 pass of the 3D transform, on the CPU.

The pass (dct_axis0.cu, k_axis0_soa) takes a float4 of a row, four adjacent
real columns, as one point of a two-lane sequence: lane a is the complex
column (col 4q) + i (col 4q+1), lane b is (col 4q+2) + i (col 4q+3).  Along
axis 0 it applies the 1D three-stage method (Section III-A): the row reorder,
a length-N FFT of each packed column, the Hermitian split of the two real
columns with the twiddle e^{-i pi k / 2N} / 2, and for the inverse the
rebuild Z[k] = Va[k] + i Vb[k] from rows k and N-k (row N taken as zero) with
e^{+i pi k / 2N} / N, the inverse FFT and the inverse reorder.  This model
restates those steps with numpy in the kernel's lane layout and checks them
against the FP64 oracle's 1D DCT-II and its inverse along axis 0, and the
strip geometry (which float4 columns and rows a CTA touches) for the sizes
the packed form serves.
"""

import numpy as np
import pytest

import oracle


def reorder_src(n, length):
    return 2 * n if n <= (length - 1) // 2 else 2 * length - 2 * n - 1


def lanes(x):
    """(N, M) real -> (N, M/4, 2) complex: lane a = cols 4q + i 4q+1, lane b = 4q+2 + i 4q+3."""
    q = x.reshape(x.shape[0], -1, 4)
    return np.stack([q[..., 0] + 1j * q[..., 1], q[..., 2] + 1j * q[..., 3]], axis=-1)


def forward_model(x):
    n = x.shape[0]
    z = lanes(x)[[reorder_src(i, n) for i in range(n)]]
    Z = np.fft.fft(z, axis=0)
    k = np.arange(n)
    Zm = Z[(n - k) % n]
    va2 = Z + np.conj(Zm)                 # 2 Va
    vb2 = -1j * (Z - np.conj(Zm))         # 2 Vb
    w = (np.exp(-1j * np.pi * k / (2 * n)) / 2)[:, None, None]
    xa, xb = np.real(w * va2), np.real(w * vb2)
    out = np.empty_like(x)
    out[:, 0::4], out[:, 1::4] = xa[..., 0], xb[..., 0]
    out[:, 2::4], out[:, 3::4] = xa[..., 1], xb[..., 1]
    return out


def inverse_model(X):
    n = X.shape[0]
    k = np.arange(n)
    c = lanes(X)                          # lane value: (X_a, X_b) of a column pair as re / im
    m = np.concatenate([np.zeros_like(c[:1]), c[1:][::-1]])   # row N - k, row N = 0
    w = (np.exp(1j * np.pi * k / (2 * n)) / n)[:, None, None]
    va = w * (c.real - 1j * m.real)
    vb = w * (c.imag - 1j * m.imag)
    z = np.fft.ifft(va + 1j * vb, axis=0) * n
    out = np.empty_like(X)
    rows = [reorder_src(i, n) for i in range(n)]
    out[rows, 0::4], out[rows, 1::4] = z[..., 0].real, z[..., 0].imag
    out[rows, 2::4], out[rows, 3::4] = z[..., 1].real, z[..., 1].imag
    return out


@pytest.mark.parametrize("n,m", [(64, 8), (128, 16), (256, 4), (16, 32)])
def test_packed_forward_is_the_axis0_dct(n, m):
    rng = np.random.default_rng(n + m)
    x = rng.standard_normal((n, m))
    ref = oracle.dct2_1d(x.T).T             # DCT-II along axis 0
    np.testing.assert_allclose(forward_model(x), ref, atol=1e-9 * n)


@pytest.mark.parametrize("n,m", [(64, 8), (128, 16), (256, 4), (16, 32)])
def test_packed_inverse_is_the_axis0_inverse(n, m):
    rng = np.random.default_rng(3 * n + m)
    X = rng.standard_normal((n, m))
    ref = oracle.idct_1d(X.T).T
    np.testing.assert_allclose(inverse_model(X), ref, atol=1e-9 * n)
    x = rng.standard_normal((n, m))
    np.testing.assert_allclose(inverse_model(forward_model(x)), x, atol=1e-9 * n)


@pytest.mark.parametrize("n", [64, 128, 256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("m", [8, 128, 4096, 65536])
def test_packed_strip_geometry(n, m):
    """NP = 128 / (N/16) sequences per CTA (at least one), TPS = N/16 threads each;
    the packed form runs when M is a multiple of 4 NP; a CTA's threads read every
    reordered row once for each of its NP float4 columns, and the strips tile the
    M/4 float4 columns."""
    tps = n // 16
    np_ = max(1, 128 // tps)
    if m % (4 * np_):
        pytest.skip("the one-sequence form serves this shape")
    ctas = m // 4 // np_
    rows = sorted(reorder_src(g + tps * j, n) for g in range(tps) for j in range(16))
    assert rows == list(range(n))
    cols = sorted(b * np_ + p for b in range(ctas) for p in range(np_))
    assert cols == list(range(m // 4))
    smem = np_ * (n + n // 16) * 16
    assert smem <= 227 * 1024 and np_ * tps <= 512
