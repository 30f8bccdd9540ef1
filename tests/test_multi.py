"""GPU tests of the uneven-size batch executor, the autotuner and forced
kernel families (needs a GB300).

The workload follows the batched configuration of the benchmark suite: 2D
transforms whose sides are log-uniform powers of two between 64 and 1024,
squares and 1:2 rectangles (``inputs.batched_shapes``).  Every transform is
compared with the FP64 oracle on its own (full comparison up to 512, sampled
entries plus the round trip at the full 512-transform size), and the error of
each transform is reported.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2110_01172_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_ABS = 1e-4
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def errors(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return (np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300),
            np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _inputs(shapes, seed):
    return [inputs.uniform(sh, seed=seed + i) for i, sh in enumerate(shapes)]


@pytest.mark.parametrize("graph", [True, False])
def test_multi_small_full_oracle_per_transform(graph):
    from paper_2110_01172_gb300 import MultiPlan
    shapes = inputs.batched_shapes(48, seed=3, lo=64, hi=512)
    xs = _inputs(shapes, 100)
    m = MultiPlan(shapes, graph=graph)
    assert m.groups == len(set(shapes))
    xin = m.pack([torch.from_numpy(x) for x in xs])
    X = m.forward(xin)
    Y = m.inverse(X)
    X2 = m.forward(xin)  # a second exec (graph replay when graph=True)
    torch.cuda.synchronize()
    assert torch.equal(X, X2)
    worst = 0.0
    for x, Xi, Yi in zip(xs, m.unpack(X), m.unpack(Y)):
        rel, mx = errors(Xi.cpu().numpy(), oracle.dct2_2d(x))
        assert rel <= REL_L2 and mx <= MAX_ABS, (x.shape, rel, mx)
        rel2, mx2 = errors(Yi.cpu().numpy(), x)
        assert rel2 <= REL_L2 and mx2 <= MAX_ABS
        worst = max(worst, rel)
    print(f"worst per-transform rel-L2 {worst:.2e} over {len(xs)} transforms")


def test_multi_graph_and_streams_agree_bitwise():
    from paper_2110_01172_gb300 import MultiPlan
    shapes = inputs.batched_shapes(40, seed=4, lo=64, hi=1024)
    xs = _inputs(shapes, 200)
    a, b = MultiPlan(shapes, graph=True), MultiPlan(shapes, graph=False)
    assert a.offsets == b.offsets
    xin = a.pack([torch.from_numpy(x) for x in xs])
    ya, yb = a.forward(xin), b.forward(xin)
    za, zb = a.inverse(ya), b.inverse(yb)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb) and torch.equal(za, zb)
    # each transform equals the single-transform plan of its shape
    from paper_2110_01172_gb300 import Plan
    for x, Xi, sh in list(zip(xs, a.unpack(ya), shapes))[:8]:
        single = Plan(sh).forward(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        assert torch.equal(single, Xi)


def test_multi_full_size_batch_sampled_per_transform():
    """512 transforms, sides 64..1024: sampled entries of every transform and
    every round trip, per-transform errors reported."""
    from paper_2110_01172_gb300 import MultiPlan
    shapes = inputs.batched_shapes(512, seed=0, lo=64, hi=1024)
    m = MultiPlan(shapes, graph=True)
    rng = np.random.default_rng(9)
    xs = _inputs(shapes, 1000)
    xin = m.pack([torch.from_numpy(x) for x in xs])
    X = m.forward(xin)
    Y = m.inverse(X)
    torch.cuda.synchronize()
    rels = []
    for x, Xi, Yi, (n1, n2) in zip(xs, m.unpack(X), m.unpack(Y), shapes):
        Xh = Xi.cpu().numpy()
        k1 = np.concatenate([rng.integers(0, n1, 4), [0, n1 - 1, n1 // 2]])
        k2 = np.concatenate([rng.integers(0, n2, 4), [0, n2 // 2, n2 - 1]])
        ref = oracle.dct2_2d_entries(x, k1, k2)
        assert np.abs(Xh[k1, k2] - ref).max() <= MAX_ABS * np.abs(Xh).max()
        rel, mx = errors(Yi.cpu().numpy(), x)
        assert rel <= REL_L2 and mx <= MAX_ABS
        rels.append(rel)
    print(f"round-trip rel-L2 per transform: median {np.median(rels):.2e}, max {max(rels):.2e}")


def test_multi_variant_kinds():
    from paper_2110_01172_gb300 import MultiPlan, GbdctError
    shapes = [(64, 128), (128, 64), (64, 128), (256, 256)]
    xs = _inputs(shapes, 300)
    m = MultiPlan(shapes, kind="dst2")
    X = m.forward(m.pack([torch.from_numpy(x) for x in xs]))
    torch.cuda.synchronize()
    for x, Xi in zip(xs, m.unpack(X)):
        rel, mx = errors(Xi.cpu().numpy(), oracle.dst2_2d(x))
        assert rel <= REL_L2 and mx <= MAX_ABS
    mi = MultiPlan(shapes, kind="idct_idxst")
    buf = mi.pack([torch.from_numpy(x) for x in xs])
    with pytest.raises(GbdctError):
        mi.forward(buf)
    Z = mi.inverse(buf)
    torch.cuda.synchronize()
    for x, Zi in zip(xs, mi.unpack(Z)):
        rel, mx = errors(Zi.cpu().numpy(), oracle.idct_idxst(x))
        assert rel <= REL_L2 and mx <= MAX_ABS


def test_tuned_multi_and_forced_families():
    from paper_2110_01172_gb300 import MultiPlan, Plan, GbdctError
    shapes = [(256, 512), (1024, 1024), (64, 64), (256, 512)]
    xs = _inputs(shapes, 400)
    m = MultiPlan(shapes, tuned=True)
    fams = m.group_families()
    assert len(fams) == 3 and all(f in ("seq", "pair", "fs2", "tp") or f.startswith(("fs2/", "tp/")) for f in fams)
    X = m.forward(m.pack([torch.from_numpy(x) for x in xs]))
    torch.cuda.synchronize()
    for x, Xi in zip(xs, m.unpack(X)):
        rel, mx = errors(Xi.cpu().numpy(), oracle.dct2_2d(x))
        assert rel <= REL_L2 and mx <= MAX_ABS
    x = inputs.uniform((256, 512), seed=7)
    ref = oracle.dct2_2d(x)
    for fam in ("seq", "pair", "fs2"):
        p = Plan((256, 512), family=fam)
        assert p.family == fam
        out = p.forward(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        rel, mx = errors(out.cpu().numpy(), ref)
        assert rel <= REL_L2 and mx <= MAX_ABS
    with pytest.raises(GbdctError):
        Plan((128, 512), family="fs2")    # fs2 needs N1 >= 256
    with pytest.raises(GbdctError):
        Plan((64, 512), family="tp")      # tp needs N1 >= 128
    assert Plan((512, 256), family="tp").family == "tp"
    assert Plan((64, 64, 64), family="seq").family == "seq"


def test_tune_cache_file_is_written_and_reused(tmp_path):
    cache = tmp_path / "tune.txt"
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2110_01172_gb300 import Plan\n"
            "p = Plan((512, 512), batch=3, tuned=True)\n"
            "print(p.choice)\n") % ROOT
    env = dict(os.environ, GBDCT_TUNE_CACHE=str(cache))
    first = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert first.returncode == 0, first.stderr
    lines = cache.read_text().split("\n")
    assert lines[0].startswith("d2x512x512_b3_k0 ") and lines[0].split()[1] == first.stdout.strip()
    second = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert second.returncode == 0 and second.stdout.strip() == first.stdout.strip()
    assert cache.read_text().count("\n") == 1   # read back, not timed again
