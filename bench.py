#!/usr/bin/env python
"""Benchmark of the 2D DCT-II + inverse on GB300: prints ONE JSON line.

A step is one pass of the whole hot path over one synthetic batch: the
forward 2D DCT-II of a 4096 x 4096 float32 array (U[-1,1], seeded) followed
by the exact inverse of the resulting spectrum.  The metric is microseconds
per step (lower is better); the forward and inverse times, GB/s and the
fraction of the measured HBM copy bandwidth (minimum traffic: one read and one
write of the float32 array per transform) are reported beside it.

Timing: W >= 3 untimed warm-up steps, then exactly K steps bracketed by a
barrier and torch.cuda.synchronize() on both sides, timed with CUDA events on
the launching stream; the maximum over ranks is reported.  Four input/output
buffer sets (512 MiB in total) rotate between steps, so every step reads
inputs that are not in the 126 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 the script runs under torchrun; every rank runs the same workload on
its own GPU (replicas only: a single transform is not split across GPUs), so
scaling is weak.  `--impl reference` times the FP64 CPU oracle on the host
cores on the same workload (rank 0 only).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N1 = N2 = 4096
METRIC = "4096² FP32 2D DCT/IDCT µs & % HBM roofline; Poisson-serve p50/p99 ms"
UNIT = "us"
WORKLOAD = "2D DCT-II + inverse (DCT-III) 4096x4096 FP32, U[-1,1] seed 0"
NBUF = 4
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one whole
# forward and one whole inverse 4096^2 transform, summed over its launches,
# from an ncu capture of warm back-to-back transforms (no cache flush between
# launches, so the workspace stays in L2 as it does here).  Valid only for the
# kernel sources with this digest; otherwise reported as null.
TRAFFIC = {
    "sources_sha256": "c65eb368e1eeb8a80a7c5d1a9a03d361187dc9ab315b758b1b4701972b81dc6d",
    "family": "tp",
    "forward_bytes": 162805504,
    "inverse_bytes": 153853184,
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n1", type=int, default=N1)
    ap.add_argument("--n2", type=int, default=N2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the secondary configurations")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--family", default=None,
                    help="force a kernel family for the headline plan (default: the plan's own choice)")
    ap.add_argument("--precision", choices=["fp32", "split_bf16"], default="fp32",
                    help="precision mode of the plan (--profile runs only)")
    ap.add_argument("--profile", action="store_true",
                    help="only run W + K untimed steps of the plan (a fixed launch sequence for ncu captures)")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed helpers (host logic; also exercised by the gloo tests on CPU)
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(backend: str):
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity at world size 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# measurement helpers
# ---------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# Files that define the timed kernels of the default family (the ncu traffic in
# TRAFFIC is valid only while these are unchanged).
KERNEL_SOURCES = ("dct2d_tp_kernels.cuh", "dct2d_fs2_kernels.cuh", "dct2d_kernels.cuh", "dct2d_launch.cuh",
                  "fft_core.cuh", "fft_soa.cuh", "l2_hint.cuh", "tma_util.cuh", "launch_dep.cuh",
                  "pass_tp_cols.cu", "pass_tp_rows.cu")


def sources_digest() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2110_01172_gb300", "csrc", name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, enabled: bool = True):
        self.gpu = gpu_index
        self.enabled = enabled
        self.proc = None
        self.path = os.path.join("/tmp", f"gbdct_clocks_{os.getpid()}.csv")

    def start(self):
        if not self.enabled:
            return
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        loaded = [v for v in sm if smax and v >= 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(n1: int, n2: int, steps: int = 6):
    """Time the FP64 oracle (as it stands) on the host cores in a subprocess."""
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "import numpy as np, oracle\n"
        "from paper_2110_01172_gb300 import inputs\n"
        "x = inputs.uniform((%d, %d), seed=0)\n"
        "ts = []\n"
        "for _ in range(%d):\n"
        "    t = time.perf_counter(); X = oracle.dct2_2d(x); y = oracle.idct2_2d(X.astype(np.float32))\n"
        "    ts.append(time.perf_counter() - t)\n"
        "print(json.dumps({'step_s': min(ts), 'total_s': sum(ts)}))\n" % (ROOT, n1, n2, steps))
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=600)
        res = json.loads(r.stdout.strip().splitlines()[-1])
        step_s, total_s = res["step_s"], res["total_s"]
    except Exception as e:  # the baseline is reported, never required
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"failed: {e}"}
    return {"value": step_s * 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} full steps (FP64 separable direct-sum DCT-II + inverse, {n1}x{n2}; "
                      f"{total_s:.1f} s of host work), best"}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_2110_01172_gb300 import inputs
    n1, n2 = args.n1, args.n2
    cores = os.cpu_count() or 1
    x = inputs.uniform((n1, n2), seed=0)
    for _ in range(args.warmup):
        X = oracle.dct2_2d(x)
        oracle.idct2_2d(X.astype(np.float32))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        X = oracle.dct2_2d(x)
        oracle.idct2_2d(X.astype(np.float32))
    us = (time.perf_counter() - t0) / args.steps * 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": us, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": us / 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if (n1, n2) == (N1, N2) else
                   f"2D DCT-II + inverse (DCT-III) {n1}x{n2} FP32, U[-1,1] seed 0",
                   "shape": [n1, n2], "parallelism": "replicas1", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": us, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"full {n1}x{n2} step (FP64 separable direct sums), "
                                   f"BLAS threads = default ({cores} cores)"},
        "e2e": {"value": us, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


SERVE_RATES = (2000.0, 5000.0, 10000.0, 20000.0)


def run_serving(args, dev):
    """Poisson-arrival spectral Poisson solves: continuous batching vs one at a
    time.  Payloads arrive in pageable host memory; each path copies them into
    its own reused page-locked ingress buffers on the request's critical path."""
    import torch
    from paper_2110_01172_gb300.serving import PoissonServer, _Resources, latency_summary, make_requests, serve_plain
    n = args.serve_requests
    sets = {rate: make_requests(n, rate, seed=int(rate)) for rate in SERVE_RATES}
    shapes = sorted({tuple(r.rho.shape) for reqs in sets.values() for r in reqs})
    server = PoissonServer(slots=8, device=dev.index)
    server.warm(shapes, per_shape=8)   # one resident solver per slot and shape: no creation mid-run
    server.serve(make_requests(64, 1e6, seed=1))   # first use of every code path
    solvers = {sh: _Resources(sh, dev) for sh in shapes}
    out = {"requests_per_rate": n, "slots": 8, "sizes": "N1, N2 in {64, ..., 2048}, 100-2000 blobs",
           "ingress": "pageable payloads copied into reused page-locked buffers (both paths)", "rates": []}
    for rate, reqs in sets.items():
        served = latency_summary(server.serve(reqs))
        plain = latency_summary(serve_plain(reqs, device=dev.index, solvers=solvers))
        out["rates"].append({"rate_per_s": rate, "served": served, "plain": plain})
    torch.cuda.synchronize()
    return out


def load_baselines():
    """ctypes handle to the comparison baselines (B1: cuFFT three-stage, B2:
    row-column); builds them if needed.  Raises if they cannot be built."""
    import ctypes
    sys.path.insert(0, ROOT)
    from paper_2110_01172_gb300 import build as _b
    lib = ctypes.CDLL(_b.build_baselines())
    vp, i = ctypes.c_void_p, ctypes.c_int
    for name, args in (("gbdct_b1_create", [ctypes.POINTER(vp), i, i]), ("gbdct_b1_forward", [vp, vp, vp, vp]),
                       ("gbdct_b1_inverse", [vp, vp, vp, vp]), ("gbdct_b1_destroy", [vp]),
                       ("gbdct_b1_r2c_only", [vp, vp]), ("gbdct_b1_c2r_only", [vp, vp]),
                       ("gbdct_b2_create", [ctypes.POINTER(vp), i, i]), ("gbdct_b2_forward", [vp, vp, vp, vp]),
                       ("gbdct_b2_destroy", [vp])):
        fn = getattr(lib, name)
        fn.restype = i
        fn.argtypes = args
    return lib


def run_baselines(dev, n1, n2, ours_fwd_us, ours_inv_us, peak):
    """B1 and B2 timed like the product (CUDA events, two rotating buffer sets
    larger than L2 together) on the same GPU; checked against our forward."""
    import ctypes
    import torch
    try:
        lib = load_baselines()
    except Exception as e:
        return {"unavailable": str(e).splitlines()[0]}
    from paper_2110_01172_gb300 import Plan
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    xs = [torch.rand(n1, n2, device=dev) * 2 - 1 for _ in range(2)]
    ys = [torch.empty_like(xs[0]) for _ in range(2)]
    out = {}
    h1, h2 = ctypes.c_void_p(), ctypes.c_void_p()
    if lib.gbdct_b1_create(ctypes.byref(h1), n1, n2) != 0:
        return {"unavailable": "baseline B1 plan creation failed"}
    if lib.gbdct_b2_create(ctypes.byref(h2), n1, n2) != 0:
        lib.gbdct_b1_destroy(h1)
        return {"unavailable": "baseline B2 plan creation failed"}
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    b1f = _event_loop_us(lambda i: lib.gbdct_b1_forward(h1, ptr(xs[i % 2]), ptr(ys[i % 2]), sp), 20, stream)
    b1i = _event_loop_us(lambda i: lib.gbdct_b1_inverse(h1, ptr(ys[i % 2]), ptr(xs[i % 2]), sp), 20, stream)
    b2f = _event_loop_us(lambda i: lib.gbdct_b2_forward(h2, ptr(xs[i % 2]), ptr(ys[i % 2]), sp), 20, stream)
    # the library 2D real FFTs alone (Table V's RFFT2D / IRFFT2D columns)
    r2c = _event_loop_us(lambda i: lib.gbdct_b1_r2c_only(h1, sp), 20, stream)
    c2r = _event_loop_us(lambda i: lib.gbdct_b1_c2r_only(h1, sp), 20, stream)
    # agreement with the product's forward on the same input
    plan = Plan((n1, n2))
    ref = plan.forward(xs[0])
    lib.gbdct_b1_forward(h1, ptr(xs[0]), ptr(ys[0]), sp)
    d1 = ((ys[0] - ref).norm() / ref.norm()).item()
    lib.gbdct_b2_forward(h2, ptr(xs[0]), ptr(ys[1]), sp)
    d2 = ((ys[1] - ref).norm() / ref.norm()).item()
    torch.cuda.synchronize()
    lib.gbdct_b1_destroy(h1)
    lib.gbdct_b2_destroy(h2)
    algo = 8.0 * n1 * n2
    out["b1_cufft_three_stage"] = {"fwd_us": b1f, "inv_us": b1i, "fwd_frac": algo / (b1f * 1e-6) / 1e9 / peak,
                                   "rel_l2_vs_ours": d1, "ours_speedup_fwd": b1f / ours_fwd_us,
                                   "ours_speedup_inv": b1i / ours_inv_us}
    out["b2_row_column"] = {"fwd_us": b2f, "fwd_frac": algo / (b2f * 1e-6) / 1e9 / peak,
                            "rel_l2_vs_ours": d2, "ours_speedup_fwd": b2f / ours_fwd_us}
    out["cufft_r2c_us"] = r2c
    out["cufft_c2r_us"] = c2r
    out["ours_vs_cufft_r2c"] = r2c / ours_fwd_us
    out["ours_vs_cufft_c2r"] = c2r / ours_inv_us
    out["note"] = "comparison builds around cuFFT (own pre/post kernels), not the product"
    return out


def _event_loop_us(fn, iters, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for i in range(3):
        fn(i)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(iters):
        fn(i)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e3 / iters


def run_configs(dev, peak):
    """The other benchmark configurations (secondary lines; the headline is 4096^2):
    C2 shapes, C3 (3D and the DST/IDXST kinds), C4 (512 uneven transforms under
    a CUDA graph).  Two rotating buffer sets per shape; at >= 1024^2 the sets
    exceed L2."""
    import torch
    from paper_2110_01172_gb300 import MultiPlan, Plan, inputs
    stream = torch.cuda.current_stream(dev)
    out = {"2d": [], "3d": [], "kinds_2048": [], "batched": None}

    def one(shape, kind="dct2"):
        plan = Plan(shape, kind)
        n = 1
        for v in shape:
            n *= v
        xs = [torch.rand(shape, device=dev) * 2 - 1 for _ in range(2)]
        ys = [torch.empty_like(xs[0]) for _ in range(2)]
        rec = {"shape": list(shape), "kind": kind, "family": plan.family}
        if kind in ("dct2", "dst2"):
            rec["fwd_us"] = _event_loop_us(lambda i: plan.forward(xs[i % 2], ys[i % 2]), 20, stream)
            rec["fwd_frac"] = 8.0 * n / (rec["fwd_us"] * 1e-6) / 1e9 / peak
        rec["inv_us"] = _event_loop_us(lambda i: plan.inverse(xs[i % 2], ys[i % 2]), 20, stream)
        rec["inv_frac"] = 8.0 * n / (rec["inv_us"] * 1e-6) / 1e9 / peak
        plan.close()
        return rec

    for shape in [(1024, 1024), (2048, 2048), (8192, 8192), (2048, 4096), (1024, 8192)]:
        out["2d"].append(one(shape))
    for shape in [(128, 128, 128), (256, 256, 256)]:
        out["3d"].append(one(shape))
    # the autotuner's tile candidates: the four-step split N1 = A * (N1 / A)
    out["fs2_splits"] = []
    for shape in [(4096, 4096), (2048, 2048), (8192, 8192), (1024, 8192)]:
        for a in (16, 32, 64, 128):
            if not 16 <= shape[0] // a <= 128:
                continue
            plan = Plan(shape, family=f"fs2/{a}")
            xs = [torch.rand(shape, device=dev) * 2 - 1 for _ in range(2)]
            ys = [torch.empty_like(xs[0]) for _ in range(2)]
            out["fs2_splits"].append({
                "shape": list(shape), "A": a, "B": shape[0] // a,
                "fwd_us": _event_loop_us(lambda i: plan.forward(xs[i % 2], ys[i % 2]), 20, stream),
                "inv_us": _event_loop_us(lambda i: plan.inverse(xs[i % 2], ys[i % 2]), 20, stream)})
            plan.close()
    # the two-pass family's tile candidates: column strips of NP column pairs
    out["tp_strips"] = []
    for shape in [(4096, 4096), (2048, 2048), (8192, 8192), (1024, 8192), (2048, 4096), (1024, 1024)]:
        m = shape[0] // 2
        for np_ in (1, 2, 4, 8, 16, 32):
            thr, smem = np_ * (m // 16), np_ * (m + m // 16) * 16
            if not (128 <= thr <= 512 and smem <= 227 * 1024 and (shape[1] // 4) % np_ == 0):
                continue
            plan = Plan(shape, family=f"tp/{np_}")
            xs = [torch.rand(shape, device=dev) * 2 - 1 for _ in range(2)]
            ys = [torch.empty_like(xs[0]) for _ in range(2)]
            out["tp_strips"].append({
                "shape": list(shape), "NP": np_, "threads": thr,
                "fwd_us": _event_loop_us(lambda i: plan.forward(xs[i % 2], ys[i % 2]), 20, stream),
                "inv_us": _event_loop_us(lambda i: plan.inverse(xs[i % 2], ys[i % 2]), 20, stream)})
            plan.close()
    for kind in ("dst2", "idct_idxst", "idxst_idct"):
        out["kinds_2048"].append(one((2048, 2048), kind))

    # split-BF16 DFT-GEMM precision mode (hand-written tcgen05 kernels) beside the FP32 path
    out["split_bf16"] = []
    for shape, batch in (((1024, 1024), 1), ((256, 256), 64), ((2048, 2048), 1)):
        p32 = Plan(shape, batch=batch)
        pg = Plan(shape, batch=batch).set_precision("split_bf16")
        full = ((batch,) if batch > 1 else ()) + shape
        xs = [torch.rand(full, device=dev) * 2 - 1 for _ in range(2)]
        ys = [torch.empty_like(xs[0]) for _ in range(2)]
        rec = {"shape": list(shape), "batch": batch}
        rec["fp32_fwd_us"] = _event_loop_us(lambda i: p32.forward(xs[i % 2], ys[i % 2]), 20, stream)
        rec["split_bf16_fwd_us"] = _event_loop_us(lambda i: pg.forward(xs[i % 2], ys[i % 2]), 20, stream)
        a, b = p32.forward(xs[0]), pg.forward(xs[0])
        rec["rel_l2_vs_fp32_path"] = ((b - a).norm() / a.norm()).item()
        flops = 3 * 2.0 * batch * shape[0] * shape[1] * (shape[0] + shape[1])
        rec["split_bf16_tflops"] = flops / (rec["split_bf16_fwd_us"] * 1e-6) / 1e12
        out["split_bf16"].append(rec)
        p32.close()
        pg.close()

    shapes = inputs.batched_shapes(512, seed=0, lo=64, hi=1024)
    rec = {"transforms": len(shapes), "sides": "log-uniform powers of two 64..1024, squares and 1:2 rectangles"}
    for graph in (True, False):
        m = MultiPlan(shapes, graph=graph)
        xin = torch.rand(m.total, device=dev) * 2 - 1
        mid, back = torch.empty_like(xin), torch.empty_like(xin)
        key = "graph" if graph else "streams"
        rec[key + "_fwd_us"] = _event_loop_us(lambda i: m.forward(xin, mid), 10, stream)
        rec[key + "_inv_us"] = _event_loop_us(lambda i: m.inverse(mid, back), 10, stream)
        rec["groups"] = m.groups
        rec["elements"] = m.total
        m.close()
    rec["fwd_frac"] = 8.0 * rec["elements"] / (rec["graph_fwd_us"] * 1e-6) / 1e9 / peak
    out["batched"] = rec
    torch.cuda.synchronize()
    return out


def run_profile(args):
    """W + K forward/inverse steps of one plan with nothing else on the GPU,
    so an ncu capture can address launches by position (2 or 3 launches per
    transform, forward first)."""
    import torch
    from paper_2110_01172_gb300 import Plan, inputs
    n1, n2 = args.n1, args.n2
    plan = Plan((n1, n2), "dct2", family=args.family)
    if args.precision != "fp32":
        plan.set_precision(args.precision)
    xs = [torch.from_numpy(inputs.uniform((n1, n2), seed=s)).cuda() for s in range(2)]
    cs = [torch.empty_like(xs[0]) for _ in range(2)]
    ys = [torch.empty_like(xs[0]) for _ in range(2)]
    for i in range(args.warmup + args.steps):
        plan.forward(xs[i % 2], cs[i % 2])
        if args.precision == "fp32":
            plan.inverse(cs[i % 2], ys[i % 2])
    torch.cuda.synchronize()
    print(json.dumps({"profile": True, "shape": [n1, n2], "family": plan.family, "precision": args.precision,
                      "launches_per_transform": plan.launches_per_exec,
                      "steps": args.warmup + args.steps}), flush=True)
    plan.close()
    return 0


def run_ours(args):
    import torch
    if args.profile:
        return run_profile(args)
    rank, world, local = dist_init("nccl")
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2110_01172_gb300 import Plan, inputs

    n1, n2 = args.n1, args.n2
    plan = Plan((n1, n2), "dct2", family=args.family)
    stream = torch.cuda.current_stream(dev)
    x0 = torch.from_numpy(inputs.uniform((n1, n2), seed=0)).to(dev)
    xs = [x0] + [torch.from_numpy(inputs.uniform((n1, n2), seed=s)).to(dev) for s in range(1, NBUF)]
    cs = [torch.empty_like(x0) for _ in range(NBUF)]
    ys = [torch.empty_like(x0) for _ in range(NBUF)]

    def step(i):
        j = i % NBUF
        plan.forward(xs[j], cs[j])
        plan.inverse(cs[j], ys[j])

    for i in range(max(3, args.warmup)):
        step(i)
    torch.cuda.synchronize()

    # per-transform timing (CUDA events on the launching stream)
    def time_loop(fn, iters):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(iters):
            fn(i)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e3 / iters

    iters = max(args.steps, 20)
    fwd_us = time_loop(lambda i: plan.forward(xs[i % NBUF], cs[i % NBUF]), iters)
    inv_us = time_loop(lambda i: plan.inverse(cs[i % NBUF], ys[i % NBUF]), iters)

    # the timed region: exactly K steps, barrier + sync on both sides
    clocks = ClockSampler(local, enabled=not args.no_clocks)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    step_us = e0.elapsed_time(e1) * 1e3 / args.steps
    step_us_max = max_over_ranks(step_us, world, dev)

    # end to end through the public API with HOST buffers: the forward's first
    # kernel reads the page-locked input and the inverse's last kernel writes
    # the page-locked output directly over the host link (no staging copies)
    xh = torch.from_numpy(inputs.uniform((n1, n2), seed=0)).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    dc = torch.empty_like(x0)

    def e2e_step(_):
        plan.forward(xh, dc)
        plan.inverse(dc, yh)

    for i in range(3):
        e2e_step(i)
    e2e_seq_us = time_loop(e2e_step, max(5, args.steps))
    # the reconstruction is checked, so the e2e loop cannot silently skip work
    err = (yh - xh).abs().max().item()
    if not err < 1e-4:
        raise RuntimeError(f"end-to-end reconstruction error {err}")

    # the same steps alternating between two plans on two streams, so that one
    # step's host reads (forward, first launch) overlap the other's host writes
    # (inverse, last launch): the host link is full duplex.  Every step still
    # reads its input from and writes its result to page-locked host memory
    # inside the timed region.
    plan_b = Plan((n1, n2), "dct2", family=args.family)
    xh_b = torch.from_numpy(inputs.uniform((n1, n2), seed=1)).pin_memory()
    yh_b = torch.empty_like(xh_b).pin_memory()
    dc_b = torch.empty_like(x0)
    lanes = [(plan, xh, dc, yh, torch.cuda.Stream(dev)), (plan_b, xh_b, dc_b, yh_b, torch.cuda.Stream(dev))]

    def pipelined_us(iters):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for lane in lanes:
            lane[4].wait_event(e0)
        for i in range(iters):
            p, xi, di, yi, si = lanes[i % 2]
            p.forward(xi, di, stream=si)
            p.inverse(di, yi, stream=si)
        for lane in lanes:
            done = torch.cuda.Event()
            done.record(lane[4])
            stream.wait_event(done)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e3 / iters

    pipelined_us(4)
    e2e_us = pipelined_us(2 * max(4, args.steps // 2))
    e2e_us = max_over_ranks(e2e_us, world, dev)
    for xi, yi in ((xh, yh), (xh_b, yh_b)):
        err = (yi - xi).abs().max().item()
        if not err < 1e-4:
            raise RuntimeError(f"end-to-end (two streams) reconstruction error {err}")
    plan_b.close()
    # the same through explicit pinned-host <-> device copies, for comparison
    din, dout = torch.empty_like(x0), torch.empty_like(x0)
    yh2 = torch.empty_like(xh).pin_memory()

    def staged_step(_):
        din.copy_(xh, non_blocking=True)
        plan.forward(din, dc)
        plan.inverse(dc, dout)
        yh2.copy_(dout, non_blocking=True)

    for i in range(3):
        staged_step(i)
    e2e_staged_us = time_loop(staged_step, max(5, args.steps))

    # per-kernel durations: each launch of the two sequences timed alone on the
    # launching stream (same buffers as the full calls)
    kernels = []
    for inverse in (False, True):
        for k in range(plan.launches_per_exec):
            src = cs if inverse else xs
            dst = ys if inverse else cs
            us = time_loop(lambda i, k=k, inverse=inverse, src=src, dst=dst:
                           plan.step(inverse, k, src[i % NBUF], dst[i % NBUF]), iters)
            kernels.append({"name": ("inverse " if inverse else "forward ") + plan.step_name(inverse, k),
                            "us": us})
    # restore valid spectra/outputs after the single-step runs
    for i in range(NBUF):
        step(i)
    torch.cuda.synchronize()

    peak, peak_kind = measured_peaks()
    algo_bytes = 8.0 * n1 * n2          # one read + one write of an N1 x N2 float32 array
    # roofline of the whole transform: the slower direction, algorithmic bytes
    # over its CUDA-event time (all launches of one transform)
    slow_us = max(fwd_us, inv_us)
    slow_dir = "inverse" if inv_us >= fwd_us else "forward"
    achieved = algo_bytes / (slow_us * 1e-6) / 1e9
    traffic = None
    if (TRAFFIC["sources_sha256"] == sources_digest() and plan.family == TRAFFIC["family"]
            and (n1, n2) == (4096, 4096)):
        traffic = TRAFFIC[slow_dir + "_bytes"]
    # per-kernel diagnostic: the longest launch, with its own array-sized I/O
    dom = max(kernels, key=lambda k: k["us"])
    kernel_io_frac = algo_bytes / (dom["us"] * 1e-6) / 1e9 / peak
    launches = plan.launches_per_exec

    serve = None
    if not args.no_serve:
        serve = run_serving(args, dev)
    configs = None if args.no_configs else run_configs(dev, measured_peaks()[0])
    baselines = None if args.no_configs else run_baselines(dev, n1, n2, fwd_us, inv_us, measured_peaks()[0])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n1, n2)

    if rank == 0:
        line = {
            "metric": METRIC, "value": step_us_max, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": step_us_max / 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "shape": [n1, n2], "parallelism": f"replicas{world}",
                       "l2": f"inputs larger than L2: {NBUF} rotating buffer sets, "
                             f"{NBUF * 3 * 4 * n1 * n2 / 2**20:.0f} MiB"},
            "dct_us": fwd_us, "idct_us": inv_us,
            "dct_gbs": algo_bytes / (fwd_us * 1e-6) / 1e9,
            "idct_gbs": algo_bytes / (inv_us * 1e-6) / 1e9,
            "transforms_per_s": sum_over_ranks(2e6 / step_us, world, dev) if world > 1 else 2e6 / step_us,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": f"whole {slow_dir} transform ({launches} launches)",
                         "transform_us": slow_us,
                         "algorithmic_bytes_per_transform": algo_bytes,
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "kernel_io_frac": {"kernel": dom["name"], "us": dom["us"], "frac": kernel_io_frac,
                               "note": "one read + one write of an array-sized buffer over the "
                                       "longest launch's time (a per-kernel diagnostic)"},
            "transform_roofline": {"dct_frac": algo_bytes / (fwd_us * 1e-6) / 1e9 / peak,
                                   "idct_frac": algo_bytes / (inv_us * 1e-6) / 1e9 / peak},
            "kernels": kernels,
            "kernel_family": plan.family,
            "serve": serve,
            "configs": configs,
            "baselines": baselines,
            "e2e": {"value": e2e_us, "unit": UNIT, "h2d_bytes_per_step": 4 * n1 * n2,
                    "d2h_bytes_per_step": 4 * n1 * n2,
                    "mode": "host buffers read/written by the first/last kernels; steps alternate "
                            "between two plans on two streams (host reads and writes overlap)",
                    "sequential_us": e2e_seq_us,
                    "staged_copies_us": e2e_staged_us},
            "gpu_launches": args.steps * 2 * launches,
            "serve_p50_ms": serve["rates"][1]["served"]["p50_ms"] if serve else None,
            "serve_p99_ms": serve["rates"][1]["served"]["p99_ms"] if serve else None,
            "serve_solves_per_s": serve["rates"][1]["served"]["solves_per_s"] if serve else None,
            "plain_p50_ms": serve["rates"][1]["plain"]["p50_ms"] if serve else None,
            "plain_p99_ms": serve["rates"][1]["plain"]["p99_ms"] if serve else None,
            "plain_solves_per_s": serve["rates"][1]["plain"]["solves_per_s"] if serve else None,
            "serve_10k": ({"served": serve["rates"][2]["served"], "plain": serve["rates"][2]["plain"]}
                          if serve else None),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    barrier(world)
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
