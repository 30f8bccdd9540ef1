"""Host logic of the Poisson server loop, on the CPU with fake GPU work.

The real ``PoissonServer.serve`` loop runs against fake resources and events:
a request's work "finishes" after a fixed number of event queries, or at once
when the loop blocks on it.  Checks: every request is served once, admission
is FIFO, no more than ``slots`` requests are in flight, the memory budget is
never exceeded (idle resources of other shapes are evicted to make room), and
the loop blocks instead of spinning when every slot is busy.
"""

import collections

import pytest

from paper_2110_01172_gb300 import serving
from paper_2110_01172_gb300.serving import AdmissionController, PoissonServer, Request, request_bytes


class FakeEvent:
    log = None

    def __init__(self):
        self.queries = 0
        self.done = False

    def record(self, stream):
        FakeEvent.log.append(("record", stream))

    def query(self):
        self.queries += 1
        if self.queries >= 3:
            self.done = True
        return self.done

    def synchronize(self):
        FakeEvent.log.append(("block",))
        self.done = True


class FakeTorch:
    class cuda:
        Event = FakeEvent


class FakeRes:
    live = 0
    peak = 0
    order = []

    def __init__(self, shape):
        self.shape = shape
        self.closed = False

    def launch(self, rho, stream, ingress=None):
        FakeRes.order.append(rho)


def make_server(slots, budget):
    srv = object.__new__(PoissonServer)
    srv.torch = FakeTorch
    srv.device = None
    srv.slots = slots
    srv.admission = AdmissionController(budget)
    srv.streams = [f"s{i}" for i in range(slots)]
    srv.pool = collections.defaultdict(list)
    srv.keep_outputs = False
    srv.graphs = False
    srv.block_horizon = 0.0
    srv.made = []
    srv._ingress = lambda slot, numel: None

    def make(shape):
        r = FakeRes(shape)
        r.close = lambda r=r: setattr(r, "closed", True)
        srv.made.append(r)
        return r

    srv._make = make
    return srv


class Payload:
    def __init__(self, shape, tag):
        self.shape = shape
        self.tag = tag

    def numel(self):
        return self.shape[0] * self.shape[1]

    def __repr__(self):
        return f"P{self.tag}"


def reqs(shapes):
    return [Request(i, Payload(sh, i), 0.0) for i, sh in enumerate(shapes)]


def track_inflight(srv):
    """Wrap launch/retire bookkeeping to record the peak number in flight."""
    state = {"now": 0, "peak": 0}
    orig_acquire, orig_release = srv._acquire, srv._release

    def acquire(shape):
        r = orig_acquire(shape)
        if r is not None:
            state["now"] += 1
            state["peak"] = max(state["peak"], state["now"])
        return r

    def release(res):
        state["now"] -= 1
        orig_release(res)

    srv._acquire, srv._release = acquire, release
    return state


@pytest.fixture(autouse=True)
def fresh_logs():
    FakeEvent.log = []
    FakeRes.order = []


def test_every_request_served_once_in_fifo_order_within_the_slot_limit():
    shapes = [(64, 64), (128, 64), (64, 64), (256, 256), (64, 64), (128, 64)] * 3
    srv = make_server(slots=3, budget=10 ** 12)
    state = track_inflight(srv)
    rs = reqs(shapes)
    res = srv.serve(rs)
    assert [r.rid for r in res] == list(range(len(rs)))
    assert [p.tag for p in FakeRes.order] == list(range(len(rs)))       # FIFO admission
    assert state["peak"] <= 3
    assert all(r.done >= r.start >= r.arrival for r in res)
    # resources are reused per shape: at most `slots` per shape were created
    per_shape = collections.Counter(r.shape for r in srv.made)
    assert max(per_shape.values()) <= 3


def test_loop_blocks_when_every_slot_is_busy():
    srv = make_server(slots=1, budget=10 ** 12)
    srv.serve(reqs([(64, 64)] * 4))
    assert ("block",) in FakeEvent.log


def test_budget_is_never_exceeded_and_idle_shapes_are_evicted():
    big, small = (512, 512), (64, 64)
    budget = request_bytes(big) + request_bytes(small)       # room for one of each, not two big
    srv = make_server(slots=2, budget=budget)
    seen = []
    orig = srv.admission.try_reserve

    def try_reserve(n):
        ok = orig(n)
        seen.append(srv.admission.reserved)
        return ok

    srv.admission.try_reserve = try_reserve
    res = srv.serve(reqs([small, big, small, (256, 128), big]))
    assert len(res) == 5
    assert max(seen) <= budget
    assert any(r.closed for r in srv.made)                    # something was evicted to fit


def test_request_larger_than_the_budget_is_reported():
    srv = make_server(slots=2, budget=request_bytes((64, 64)))
    with pytest.raises(RuntimeError, match="budget"):
        srv.serve(reqs([(512, 512)]))
