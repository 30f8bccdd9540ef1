"""Continuous-batching server for spectral Poisson solves on one GPU.

Requests (density maps of mixed N1 x N2 sizes, Section V-B / Algorithm 4) arrive
over time; each is served by ``PoissonSolver`` (forward DCT-II, spectral divide,
three inverse transforms).  The server keeps solvers and device buffers resident
per shape, admits a request when a slot (CUDA stream) is free and the memory it
would need fits the budget, and runs admitted requests concurrently on their
own streams, so work of requests that arrive while others are on the GPU
overlaps on the device.  Between admissions the loop blocks on the oldest
in-flight request instead of spinning.  ``serve_plain`` is the reference path: one request at a
time, in arrival order, on one stream.

Ingress: a request's payload arrives in ordinary (pageable) host memory.  The
server owns one page-locked ingress buffer per slot, reused for every request
it admits into that slot: the payload is copied into it on the host, then to
the device on the slot's stream.  Reused pinned pages stay fast for the
device; a freshly pinned page is much slower on its first device read (on the
Grace host, 16 MB in 4.3 ms cold vs 0.09 ms warm), which is why the buffers are
allocated and touched once, ahead of the run.  The plain path has the same
ingress (one reused buffer).

Each request's result does not depend on what else is in flight: the kernels
are deterministic and the plan a request uses depends only on its shape.
"""

from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    rho: object            # host float32 tensor (N1, N2), pageable or pinned
    arrival: float         # seconds after the start of the run


@dataclass
class Result:
    rid: int
    shape: tuple
    arrival: float
    start: float
    done: float
    outputs: tuple = field(default=None, repr=False)   # host (psi, xi0, xi1) when kept

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class AdmissionController:
    """Host-side device-memory budget: admit a request only if its bytes fit."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.reserved = 0

    def try_reserve(self, nbytes: int) -> bool:
        if self.reserved + nbytes > self.budget:
            return False
        self.reserved += nbytes
        return True

    def release(self, nbytes: int):
        self.reserved -= nbytes
        assert self.reserved >= 0


class _Resources:
    """A resident solver, device buffers and pinned host outputs for one shape.

    Used by one request at a time; kept in the server's pool between requests.
    """

    def __init__(self, shape, device, graph: bool = False):
        import torch
        from .binding import PoissonSolver
        self.shape = shape
        self.solver = PoissonSolver(shape, device)
        self.rho = torch.empty(shape, dtype=torch.float32, device=device)
        self.out = torch.empty((3,) + tuple(shape), dtype=torch.float32, device=device)  # psi, xi0, xi1
        self.bufs = [self.rho, self.out[0], self.out[1], self.out[2]]
        self.host = torch.empty((3,) + tuple(shape), dtype=torch.float32, pin_memory=True)
        self.graph = None
        graph_pool = 0
        if graph:
            # The whole solve (forward DCT-II, spectral divide, three inverse
            # transforms: 13 kernel launches) as one CUDA graph, replayed per request.
            side = torch.cuda.Stream(device)
            side.wait_stream(torch.cuda.current_stream(device))
            with torch.cuda.stream(side):
                self.solver.solve(self.rho, self.out[0], self.out[1], self.out[2], stream=side)
            side.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            alloc0 = torch.cuda.memory_allocated(device)
            with torch.cuda.graph(self.graph, stream=side):
                self.solver.solve(self.rho, self.out[0], self.out[1], self.out[2], stream=side)
            graph_pool = max(0, torch.cuda.memory_allocated(device) - alloc0)
            # the first launch of an instantiated graph uploads it to the device;
            # do it here so that no request pays for it
            self.graph.replay()
            torch.cuda.synchronize(device)
        # device bytes this resource allocates: the solver's own allocations,
        # the four arrays, and what the graph capture allocated in its pool
        self.device_bytes = (self.solver.workspace_bytes + self.rho.nbytes + self.out.nbytes + graph_pool)
        # The first device access to a pinned host page costs far more than
        # later ones (measured ~50x on a coherent Grace host: 16 MB in 4.3 ms
        # cold vs 0.09 ms warm); touch the output buffer once here.
        self.host.copy_(self.out, non_blocking=True)
        torch.cuda.synchronize(device)

    def launch(self, rho_host, stream, ingress=None):
        """Host input -> (ingress buffer ->) device, solve, results -> pinned
        host; the device work is asynchronous on `stream`.  `ingress` is a
        page-locked buffer of at least N1*N2 floats that no earlier work on
        the device still reads."""
        import torch
        if ingress is not None:
            staged = ingress[: rho_host.numel()].view(rho_host.shape)
            staged.copy_(rho_host)
            rho_host = staged
        with torch.cuda.stream(stream):
            self.rho.copy_(rho_host, non_blocking=True)
            if self.graph is not None:
                self.graph.replay()
            else:
                self.solver.solve(self.rho, self.out[0], self.out[1], self.out[2], stream=stream)
            self.host.copy_(self.out, non_blocking=True)

    def close(self):
        self.solver.close()
        self.graph = self.bufs = self.host = self.rho = self.out = None


def request_bytes(shape) -> int:
    """Device bytes charged for one resident solve of this shape: an upper bound
    of what ``_Resources`` allocates (checked against its measured
    ``device_bytes`` in the GPU tests): three plan workspaces (4 N1 N2 bytes
    each), the two staging arrays of the families that use them, the
    denominator table, the four arrays, the small tables, and a 1 MiB margin
    for the CUDA graph and its pool."""
    n = shape[0] * shape[1]
    return 4 * n * 3 + 8 * n + 4 * n + 4 * 4 * n + 16 * (shape[0] + shape[1]) + (1 << 20)


class PoissonServer:
    def __init__(self, slots: int = 8, budget_bytes: int | None = None, device: int = 0,
                 keep_outputs: bool = False, graphs: bool = True, block_horizon: float = 2e-4):
        """block_horizon: seconds; with a free slot, the loop does not block on
        in-flight work when the next request arrives within this horizon."""
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.slots = slots
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(0.5 * free)
        self.admission = AdmissionController(budget_bytes)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.pool = collections.defaultdict(list)   # shape -> idle _Resources
        self.keep_outputs = keep_outputs
        self.graphs = graphs
        self.block_horizon = float(block_horizon)
        self.ingress_bufs = [None] * slots

    def _ingress(self, slot, numel):
        """The slot's page-locked ingress buffer, grown (and touched once) if too small."""
        torch = self.torch
        buf = self.ingress_bufs[slot]
        if buf is None or buf.numel() < numel:
            buf = torch.empty(numel, dtype=torch.float32, pin_memory=True)
            torch.empty(numel, dtype=torch.float32, device=self.device).copy_(buf, non_blocking=True)
            torch.cuda.synchronize(self.device)
            self.ingress_bufs[slot] = buf
        return buf

    def _acquire(self, shape):
        idle = self.pool[shape]
        if idle:
            return idle.pop()
        need = request_bytes(shape)
        while not self.admission.try_reserve(need):
            # evict an idle resident solver of another shape, if any
            victim = next((k for k, v in self.pool.items() if v and k != shape), None)
            if victim is None:
                return None
            self.pool[victim].pop().close()
            self.admission.release(request_bytes(victim))
        return self._make(shape)

    def _make(self, shape):
        """New resident resources for `shape` (the only place that creates them)."""
        return _Resources(shape, self.device, graph=self.graphs)

    def _release(self, res):
        self.pool[res.shape].append(res)

    def warm(self, shapes, per_shape: int = 1):
        """Create `per_shape` resident solvers per shape ahead of the run.

        Plan creation synchronises the device, so solvers created while requests
        are in flight stall them; a warmed pool keeps creation off the request path.
        """
        shapes = set(tuple(x) for x in shapes)
        for s in shapes:
            held = [self._acquire(s) for _ in range(per_shape)]
            for r in held:
                if r is not None:
                    self._release(r)
        biggest = max(a * b for a, b in shapes)
        for slot in range(self.slots):
            self._ingress(slot, biggest)
        self.torch.cuda.synchronize(self.device)

    def serve(self, requests):
        """Serve `requests` (arrival times relative to the call) and return their results.

        The loop admits ready requests into free slots, retires finished ones,
        and otherwise *blocks* on the oldest in-flight request's event rather
        than spinning on event queries: on a coherent Grace host, a host thread
        that polls CUDA events while host<->device copies are in flight was
        measured to slow those copies to ~10 GB/s (5k requests/s: 3.1k solves/s
        and p50 36 ms when polling, 5.2k solves/s and p50 0.16 ms when blocking).
        """
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        ready = collections.deque()
        free_slots = list(range(self.slots))
        inflight = collections.OrderedDict()   # slot -> (request, resources, done_event, start), launch order
        results = []
        t0 = time.perf_counter()
        while pending or ready or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                ready.append(pending.popleft())
            # retire finished work first: frees slots and memory
            for slot in list(inflight):
                req, res, ev, start = inflight[slot]
                if ev.query():
                    outs = tuple(h.clone() for h in res.host.unbind(0)) if self.keep_outputs else None
                    results.append(Result(req.rid, res.shape, req.arrival, start, time.perf_counter() - t0, outs))
                    self._release(res)
                    free_slots.append(slot)
                    del inflight[slot]
            # admit ready requests into free slots (FIFO; a request whose memory
            # does not fit waits until earlier requests release theirs)
            while ready and free_slots:
                req = ready[0]
                res = self._acquire(tuple(req.rho.shape))
                if res is None:
                    break
                ready.popleft()
                slot = free_slots.pop()
                stream = self.streams[slot]
                start = time.perf_counter() - t0
                res.launch(req.rho, stream, self._ingress(slot, req.rho.numel()))
                ev = torch.cuda.Event()
                ev.record(stream)
                inflight[slot] = (req, res, ev, start)
            if not inflight and ready and not free_slots:
                raise RuntimeError("no slot available")
            if not inflight and ready and free_slots:
                raise RuntimeError("request does not fit the memory budget")
            # nothing to admit now: block on the oldest in-flight request (unless
            # the next arrival is imminent and a slot is free)
            if inflight:
                soon = bool(pending) and pending[0].arrival <= time.perf_counter() - t0 + self.block_horizon
                if not free_slots or not (ready or soon):
                    next(iter(inflight.values()))[2].synchronize()
        return sorted(results, key=lambda r: r.rid)


def serve_plain(requests, device: int = 0, keep_outputs: bool = False, solvers=None):
    """Reference path: one request at a time in arrival order on one stream,
    through one reused page-locked ingress buffer."""
    import torch
    dev = torch.device("cuda", device)
    solvers = {} if solvers is None else solvers
    stream = torch.cuda.current_stream(dev)
    biggest = max(r.rho.numel() for r in requests)
    ingress = torch.empty(biggest, dtype=torch.float32, pin_memory=True)
    torch.empty(biggest, dtype=torch.float32, device=dev).copy_(ingress, non_blocking=True)
    torch.cuda.synchronize(dev)
    results = []
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        while time.perf_counter() - t0 < req.arrival:
            pass
        shape = tuple(req.rho.shape)
        if shape not in solvers:
            solvers[shape] = _Resources(shape, dev)
        res = solvers[shape]
        start = time.perf_counter() - t0
        res.launch(req.rho, stream, ingress)
        stream.synchronize()
        outs = tuple(h.clone() for h in res.host.unbind(0)) if keep_outputs else None
        results.append(Result(req.rid, shape, req.arrival, start, time.perf_counter() - t0, outs))
    return results


def make_requests(count: int, rate_per_s: float, seed: int = 0, lo: int = 64, hi: int = 2048):
    """Seeded Poisson-arrival requests of blob density maps with sides in {lo, ..., hi}."""
    import torch
    from .inputs import density_blobs, poisson_arrivals, serving_shapes
    shapes = serving_shapes(count, seed=seed, lo=lo, hi=hi)
    arrivals = poisson_arrivals(count, rate_per_s, seed=seed + 1)
    reqs = []
    cache = {}
    for i, (shape, t) in enumerate(zip(shapes, arrivals)):
        key = (shape, i % 4)   # a few distinct maps per shape keep generation cheap
        if key not in cache:
            cache[key] = torch.from_numpy(density_blobs(shape, seed=seed * 1000 + i % 4,
                                                        n_blobs=100 + (i * 37) % 1900))
        reqs.append(Request(i, cache[key], float(t)))
    return reqs


def latency_summary(results):
    lat = np.array([r.latency for r in results]) * 1e3
    span = max(r.done for r in results) - min(r.arrival for r in results)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "solves_per_s": len(results) / span, "requests": len(results)}
