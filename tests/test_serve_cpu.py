"""Host logic of the serving loop, on a simulated clock with a fake executor (no GPU).

The fake executor models one device that runs batches back to back (fixed launch cost plus
a cost per request), rejects inadmissible lattices the way the library does
(DGT_ERR_LENGTH when L is not a multiple of lam2 lcm(a, M)), and can be told to fail
chosen batches at launch or at completion: the failure is made on the host, as a raised
exception, never on a device.
"""
import math

import pytest

from paper_1307_4569_gb300._capi import DGTError
from paper_1307_4569_gb300.serve import Scheduler, request_key
from workloads import Request, serve_requests


class SimClock:
    def __init__(self):
        self.now = 0.0

    def __call__(self):
        return self.now

    def idle(self, dt):
        self.now += max(dt, 1e-6)


class FakeExecutor:
    def __init__(self, clock, t_launch=50e-6, t_req=20e-6, fail_launch=(), fail_finish=(), ws=1 << 20):
        self.clock = clock
        self.t_launch, self.t_req = t_launch, t_req
        self.fail_launch, self.fail_finish = set(fail_launch), set(fail_finish)
        self.ws = ws
        self.free_at = 0.0
        self.launched = []            # (key, kind, rids)
        self.prepared = set()

    def prepare(self, key):
        L, a, M, lam1, lam2, _ = key
        lcm = a * M // math.gcd(a, M)
        if L % (lam2 * lcm):
            raise DGTError(2, "L=%d is not a multiple of lam2 lcm(a, M) = %d" % (L, lam2 * lcm))
        self.prepared.add(key)

    def coefs(self, key):
        return (key[0] // key[1]) * key[2]

    def bytes_for(self, key, kind, n):
        L, a, M = key[0], key[1], key[2]
        return n * 8 * (L + (L // a) * M) + self.ws

    def launch(self, key, kind, reqs, rids):
        assert key in self.prepared
        idx = len(self.launched)
        self.launched.append((key, kind, list(rids)))
        if idx in self.fail_launch:
            raise RuntimeError("injected launch failure")
        start = max(self.clock.now, self.free_at)
        self.free_at = start + self.t_launch + self.t_req * len(rids)
        return (idx, self.free_at)

    def done(self, h):
        return self.clock.now >= h[1]

    def finish(self, h):
        if h[0] in self.fail_finish:
            raise RuntimeError("injected device error")


def _run(reqs, cap=40 << 30, max_batch=64, max_inflight=2, **kw):
    clk = SimClock()
    ex = FakeExecutor(clk, **kw)
    st = Scheduler(ex, cap, max_batch=max_batch, max_inflight=max_inflight).run(reqs, clock=clk, idle=clk.idle)
    return st, ex


def test_every_request_accounted_and_infeasible_rejected_at_plan_time():
    reqs = serve_requests(2000, 0.5, seed=4, infeasible_every=50)
    st, ex = _run(reqs)
    s = st.summary()
    bad = [i for i, r in enumerate(reqs) if not r.feasible]
    assert bad, "the stream must contain deliberately infeasible requests"
    assert s["requests"] == len(reqs)
    assert s["errors"] == len(bad) and s["ok"] == len(reqs) - len(bad)
    for i in bad:
        assert st.served[i].status == "error" and "DGT_ERR_LENGTH" in st.served[i].error
    for sv in st.served:
        assert sv.status in ("ok", "error")
        assert sv.t_done >= sv.t_arrival
    # no lambda2 = 3 lattice is admissible for the power-of-two lengths (only the forced ones)
    assert all(r.lam2 != 3 for r in reqs if r.feasible)


def test_batches_are_homogeneous_bounded_and_fifo():
    reqs = serve_requests(20000, 0.2, seed=5)
    st, ex = _run(reqs, max_batch=16, t_req=200e-6)
    for key, kind, rids in ex.launched:
        assert 1 <= len(rids) <= 16
        for r in rids:
            assert request_key(reqs[r]) == key and reqs[r].kind == kind
        arr = [reqs[r].t_arrival for r in rids]
        assert arr == sorted(arr)
    # FIFO within a group: batch indices never go back in arrival order
    last = {}
    for i in sorted(range(len(reqs)), key=lambda i: reqs[i].t_arrival):
        g = (request_key(reqs[i]), reqs[i].kind)
        b = st.served[i].batch
        assert b >= last.get(g, -1)
        last[g] = b
    # overload (20k req/s against >= 250 us per request) makes batches form
    assert st.summary()["mean_batch"] > 1.5


def test_admission_cap_bounds_inflight_bytes_and_rejects_oversized():
    reqs = serve_requests(4000, 0.25, seed=6)
    # 2^20-sample requests need > 72 MB each (input + 8L coefficients, complex64): a 64 MB cap
    # can never admit them, while the smaller lengths are served under the cap
    cap = 64 << 20
    st, ex = _run(reqs, cap=cap)
    s = st.summary()
    assert s["peak_inflight_bytes"] <= cap
    big = [i for i, r in enumerate(reqs) if r.L == 1 << 20 and r.feasible]
    assert big and all(st.served[i].status == "rejected" for i in big)
    small = [i for i, r in enumerate(reqs) if r.L < 1 << 20 and r.feasible]
    assert all(st.served[i].status == "ok" for i in small)
    assert s["rejected"] == len(big)


def test_injected_failures_fail_only_their_batch():
    reqs = serve_requests(3000, 0.3, seed=7)
    st, ex = _run(reqs, fail_launch={3}, fail_finish={5, 9})
    failed = set()
    for idx in (3, 5, 9):
        failed |= set(ex.launched[idx][2])
    for i, sv in enumerate(st.served):
        if i in failed:
            assert sv.status == "error" and "injected" in sv.error
        elif reqs[i].feasible:
            assert sv.status == "ok"
    assert st.summary()["ok"] == sum(r.feasible for r in reqs) - len(failed)


def test_latency_is_queueing_plus_service_on_an_idle_server():
    # widely spaced requests on an idle device: latency = launch cost + one request, plus at
    # most one polling interval (20 us) before the completion is seen
    reqs = [Request(0.01 * (i + 1), 16384, 16, 128, 1, 2, "gauss", "dgt", True, 0) for i in range(20)]
    st, ex = _run(reqs, t_launch=100e-6, t_req=50e-6)
    lat = [sv.latency for sv in st.served]
    assert all(150e-6 - 1e-9 <= x <= 170e-6 + 1e-9 for x in lat), lat
    assert st.summary()["mean_batch"] == 1.0


def test_inflight_limit_holds():
    reqs = serve_requests(50000, 0.05, seed=8)
    clk = SimClock()
    ex = FakeExecutor(clk, t_req=100e-6)
    seen = []
    orig_launch = ex.launch

    def launch(key, kind, r, rids):
        seen.append(sum(1 for h in ex_handles if not ex.done(h)))
        h = orig_launch(key, kind, r, rids)
        ex_handles.append(h)
        return h

    ex_handles = []
    ex.launch = launch
    Scheduler(ex, 40 << 30, max_batch=8, max_inflight=3).run(reqs, clock=clk, idle=clk.idle)
    assert max(seen) <= 2          # at most 3 in flight including the one being launched


@pytest.mark.parametrize("max_batch", [1, 4])
def test_batch_one_serves_everything(max_batch):
    reqs = serve_requests(1000, 0.2, seed=9)
    st, ex = _run(reqs, max_batch=max_batch)
    assert all(len(r) <= max_batch for _, _, r in ex.launched)
    assert st.summary()["ok"] == sum(r.feasible for r in reqs)


def test_per_batch_limit_of_fixed_buffers():
    # an executor with fixed per-stream buffers bounds each batch: batches shrink to fit, and
    # requests that cannot fit one buffer are rejected even though the global cap is large
    reqs = serve_requests(20000, 0.1, seed=10)
    clk = SimClock()
    ex = FakeExecutor(clk, t_req=200e-6)
    ex.max_batch_bytes = 40 << 20
    st = Scheduler(ex, 40 << 30, max_batch=64).run(reqs, clock=clk, idle=clk.idle)
    for key, kind, rids in ex.launched:
        assert ex.bytes_for(key, kind, len(rids)) <= ex.max_batch_bytes
    big = [i for i, r in enumerate(reqs) if r.feasible and ex.bytes_for(
        (r.L, r.a, r.M, r.lam1, r.lam2, r.window), r.kind, 1) > ex.max_batch_bytes]
    assert big and all(st.served[i].status == "rejected" for i in big)
