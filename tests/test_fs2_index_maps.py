"""Index arithmetic of the fs2 kernels, checked on the CPU for every supported N1.

The formulas below restate the kernels' index maps (dct2d_fs2_kernels.cuh):
the four-step split N1 = A B, the slab rows each column step reads and writes,
the output rows of the register DFT (cs_out_row / the vector form's
o = q T/Q + i + T p), the physical workspace row (k1 % B) A + k1 / B, the
reorder, and the row-pass pairing.  Each step must touch every row exactly
once per column, and every index must stay inside its buffer, for every
size the family supports (N1 = 256 ... 8192).
"""

import pytest

SIZES = [256, 512, 1024, 2048, 4096, 8192]


def split(n1):
    """The default four-step split N1 = A B."""
    a = 16 if n1 == 2048 else (64 if n1 >= 4096 else (32 if n1 >= 512 else 16))
    return a, n1 // a


# every split the column steps are built for (A and B in {16, 32, 64, 128});
# the autotuner chooses among them
SPLITS = [(n1, a) for n1 in SIZES for a in (16, 32, 64, 128) if 16 <= n1 // a <= 128]


def reorder_src(n, length):
    return 2 * n if n <= (length - 1) // 2 else 2 * length - 2 * n - 1


def col_cfg(s):
    """(Q threads per column group, T points per thread) of the vector column steps."""
    q = 8 if s >= 64 else 4
    return q, s // q


def prow(k1, a, b):
    return (k1 % b) * a + k1 // b


@pytest.mark.parametrize("n1,a", SPLITS)
def test_column_steps_touch_every_row_once(n1, a):
    b = n1 // a
    assert a * b == n1
    for kind in range(4):
        s = b if kind in (0, 3) else a          # DFT length of the step
        nslab = a if kind in (0, 3) else b      # CTAs along the slab axis
        q_, t = col_cfg(s)
        assert q_ * t == s and t % q_ == 0      # the cross-thread DFT_Q has T/Q m-values per thread
        reads, writes, twiddles = [], [], []
        for r in range(nslab):
            for q in range(q_):
                for j in range(t):              # loads: slab row i = q + Q j
                    i = q + q_ * j
                    if kind == 0:
                        reads.append(reorder_src(r + a * i, n1))
                    elif kind == 3:
                        reads.append(i * a + r)
                    else:
                        reads.append(r * a + i)
                for i in range(t // q_):        # stores: output row o of the slab
                    for p in range(q_):
                        o = q * (t // q_) + i + t * p
                        assert 0 <= o < s
                        if kind == 0:
                            writes.append(o * a + r)
                            twiddles.append(r * b + o)
                        elif kind == 1:
                            writes.append(r * a + o)
                        elif kind == 2:
                            writes.append(r * a + o)
                            twiddles.append(o * b + r)
                        else:
                            writes.append(reorder_src(r + a * o, n1))
        assert sorted(reads) == list(range(n1)), kind
        assert sorted(writes) == list(range(n1)), kind
        if twiddles:
            assert sorted(twiddles) == list(range(n1))   # the W_N1 table has N1 entries, each used once


@pytest.mark.parametrize("n1,a", SPLITS)
def test_four_step_layout_is_the_column_spectrum_order(n1, a):
    """C1 writes DFT_B output k1b of slab n1a to row k1b A + n1a; C2 turns the
    A rows k1b A + i into k1 = k1b + B k1a at row k1b A + k1a = prow(k1)."""
    b = n1 // a
    rows = [prow(k1, a, b) for k1 in range(n1)]
    assert sorted(rows) == list(range(n1))
    for k1 in range(n1):
        k1b, k1a = k1 % b, k1 // b
        assert prow(k1, a, b) == k1b * a + k1a


@pytest.mark.parametrize("n1", SIZES)
def test_row_pass_items_pair_every_row_once(n1):
    """Item k1 < N1/2 owns rows k1 and N1 - k1; item 0 the packed rows 0 and N1/2."""
    owned = []
    for k1 in range(n1 // 2):
        owned += [k1, n1 - k1] if k1 else [0, n1 // 2]
    assert sorted(owned) == list(range(n1))


@pytest.mark.parametrize("n2", [256, 512, 1024, 2048, 4096, 8192, 16384])
def test_row_pass_thread_geometry(n2):
    """16 points per thread, TPS = N2/16 threads per item, NI items per CTA
    (at least 256 threads), the combine's 4-column groups and the pairing's
    2-column stores cover the row exactly."""
    tps = n2 // 16
    ni = max(1, 256 // tps)
    assert ni * tps >= 256 or tps >= 256
    pts = sorted(g + j * tps for g in range(tps) for j in range(16))
    assert pts == list(range(n2))
    cols = set()
    for g in range(tps):
        for i in range(g, n2 // 8, tps):        # forward combine: columns c..c+3 and L-c-4..L-c-1
            c = 4 * i
            cols.update(range(c, c + 4))
            cols.update(range(n2 - c - 4, n2 - c))
    assert cols == set(range(n2))
    pairs = set()
    for g in range(tps):
        for h in range(g, n2 // 4, tps):        # inverse pairing: p = 2h, 2h + 1 of L/2 complex
            pairs.update((2 * h, 2 * h + 1))
    assert pairs == set(range(n2 // 2))
