"""Index arithmetic and radix-2 algebra of the two-pass kernels, on the CPU.

The two-pass family (dct2d_tp_kernels.cuh) splits the length-N1 column FFT
once by decimation in time: the column pass writes E = DFT_M(v[2m]) to
workspace rows [0, M) and O = DFT_M(v[2m+1]) to rows [M, N1) (M = N1/2), and
the row pass rebuilds the column-spectrum rows its two items need from four
workspace rows.  This file restates those maps with numpy (a model of the data
flow, not of the kernels' arithmetic order) and checks them against the plain
column DFT: the item pairing covers every row once, the four rebuilt rows are
the right column-spectrum rows, the inverse pairing's E' / O' give the even and
odd halves of the inverse column DFT, every index stays inside its buffer, and
the column pass's strips tile the rows.
"""

import numpy as np
import pytest

SIZES = [128, 256, 512, 1024, 2048, 4096, 8192]


def reorder_src(n, length):
    return 2 * n if n <= (length - 1) // 2 else 2 * length - 2 * n - 1


def item_b(c, m):
    return m - c if c else m // 2


def mirror(k, n1):
    return n1 - k if k else n1 // 2


def fft_tps(length):
    return length // 16


@pytest.mark.parametrize("n1", SIZES)
def test_item_pairing_covers_every_row_once(n1):
    m = n1 // 2
    rows, ws_rows = [], []
    for c in range(n1 // 4):
        kb = item_b(c, m)
        for k in (c, kb):
            rows += [k, mirror(k, n1)]
        ws_rows += [c, m + c, kb, m + kb]
        assert all(0 <= r < n1 for r in ws_rows[-4:])
    assert sorted(rows) == list(range(n1))          # every column-spectrum row once
    assert sorted(ws_rows) == list(range(n1))       # every workspace row read (written) once


def _column_model(n1, ncol, seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n1, ncol)) + 1j * rng.standard_normal((n1, ncol))
    v = z[[reorder_src(n, n1) for n in range(n1)]]
    m = n1 // 2
    work = np.concatenate([np.fft.fft(v[0::2], axis=0), np.fft.fft(v[1::2], axis=0)])
    return v, work, np.fft.fft(v, axis=0), m


@pytest.mark.parametrize("n1", [16, 32, 512])
def test_forward_radix2_step_rebuilds_the_rows(n1):
    """(z_a, m_a, z_b, m_b) of group c = (V[c], V[mirror c], V[kb], V[mirror kb])."""
    _, work, V, m = _column_model(n1, 3, seed=n1)
    for c in range(n1 // 4):
        first = c == 0
        kb = item_b(c, m)
        w = np.exp(-2j * np.pi * c / n1)
        w1 = 1.0 if first else w
        w2 = np.exp(-2j * np.pi * (m // 2) / n1) if first else np.conj(w)
        e1, o1 = work[c], work[m + c] * w1
        e2, o2 = work[kb], work[m + kb] * w2
        p, q, r, s = e1 + o1, e1 - o1, e2 + o2, e2 - o2
        a, am, b, bm = p, (q if first else r), (r if first else s), (s if first else q)
        np.testing.assert_allclose(a, V[c], atol=1e-9)
        np.testing.assert_allclose(am, V[mirror(c, n1)], atol=1e-9)
        np.testing.assert_allclose(b, V[kb], atol=1e-9)
        np.testing.assert_allclose(bm, V[mirror(kb, n1)], atol=1e-9)


@pytest.mark.parametrize("n1", [16, 32, 512])
def test_inverse_pairing_gives_the_half_length_inverses(n1):
    """E'[k] = V[k] + V[M+k], O'[k] = W^-k (V[k] - V[M+k]) written by the
    inverse pairing from the four rows of its group; IDFT_M of E' and O' are
    the even and odd positions of the length-N1 inverse column DFT."""
    v, _, V, m = _column_model(n1, 2, seed=n1 + 1)
    ep = np.zeros((m, V.shape[1]), complex)
    op = np.zeros_like(ep)
    for c in range(n1 // 4):
        first = c == 0
        kb = item_b(c, m)
        w = np.exp(-2j * np.pi * c / n1)
        za0, za1 = V[c], V[mirror(c, n1)]
        zb0, zb1 = V[kb], V[mirror(kb, n1)]
        x1 = za1 if first else zb1
        x2 = zb1 if first else za1
        d1, d2 = za0 - x1, zb0 - x2
        ep[c] = za0 + x1
        op[c] = d1 if first else np.conj(w) * d1
        ep[kb] = zb0 + x2
        op[kb] = 1j * d2 if first else -d2 * w
    full = np.fft.ifft(V, axis=0) * n1                 # = n1 * v
    np.testing.assert_allclose(np.fft.ifft(ep, axis=0) * m, full[0::2], atol=1e-8 * n1)
    np.testing.assert_allclose(np.fft.ifft(op, axis=0) * m, full[1::2], atol=1e-8 * n1)
    np.testing.assert_allclose(full, n1 * v, atol=1e-8 * n1)


def strip_ok(m, n2, np_):
    """Strip widths the column pass is built for (tp_strip_ok in dct2d_launch.cuh)."""
    threads = np_ * (m // 16)
    smem = np_ * (m + m // 16) * 16
    return 64 <= threads <= 512 and smem <= 227 * 1024 - 256 and (n2 // 4) % np_ == 0


@pytest.mark.parametrize("n1", SIZES)
@pytest.mark.parametrize("n2", [128, 256, 512, 1024, 2048, 4096, 8192])
def test_default_strip_width_is_valid(n1, n2):
    m = n1 // 2
    assert strip_ok(m, n2, max(2, 128 // fft_tps(m)))     # tp_default_np: 128 threads, >= 2 pairs


@pytest.mark.parametrize("n1", SIZES)
@pytest.mark.parametrize("n2", [128, 256, 512, 1024, 2048, 4096, 8192])
@pytest.mark.parametrize("np_", [1, 2, 4, 8, 16, 32])
def test_column_pass_geometry(n1, n2, np_):
    """Column pass: NP column pairs (float4) per CTA, TPS = M/16 threads per
    pair, grid (N2/4/NP, 2 parities); thread (g, pi) loads reordered rows
    2 (g + TPS j) + parity and float4 column strip * NP + pi."""
    m = n1 // 2
    tps = fft_tps(m)
    if not strip_ok(m, n2, np_):
        pytest.skip("strip width not built for this shape")
    assert (n2 // 4) % np_ == 0 and np_ * tps <= 512
    strips = n2 // 4 // np_
    # rows of one strip and parity: every reordered row of that parity once,
    # every input row once over both parities
    rows = []
    for par in range(2):
        rows += [reorder_src(2 * (g + tps * j) + par, n1) for g in range(tps) for j in range(16)]
    assert sorted(rows) == list(range(n1))
    cols = sorted(s * np_ + p for s in range(strips) for p in range(np_))
    assert cols == list(range(n2 // 4))
    # workspace row of output k of parity par, and the store's point order
    ks = sorted(g + tps * r for g in range(tps) for r in range(16))
    assert ks == list(range(m))
    assert max(par * m + k for par in range(2) for k in ks) == n1 - 1


@pytest.mark.parametrize("np_", [1, 2, 4, 8, 16])
def test_interleaved_shared_memory_is_conflict_free(np_):
    """Point i of pair pi at float4 slot NP * pidx4(i) + pi: the eight lanes of
    a quarter warp (4-aligned runs of consecutive points, NP pairs) hit eight
    distinct 16-byte bank groups."""
    def pidx4(i):
        return i + (i >> 4)
    lanes_per_q = 8
    g_per_q = max(1, lanes_per_q // np_)
    for base in range(0, 256, g_per_q):
        if (base % 4) + g_per_q > 4 and g_per_q <= 4:
            continue
        slots = {(np_ * pidx4(base + d) + p) % 8 for d in range(g_per_q) for p in range(min(np_, 8))}
        assert len(slots) == min(8, g_per_q * np_)
