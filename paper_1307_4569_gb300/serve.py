"""Serving loop: a stream of independent DGT / iDGT requests of mixed lattices on one GPU.

Every request names a lattice (L, a, M, lambda = lam1/lam2), a window ("gauss" for the
periodised Gaussian of width sqrt(L), "hann<Lg>" for a zero-centred Hann FIR window of Lg
taps) and an operation: "dgt" (analysis of a length-L signal, Sec. 2, Eq. DGT) or "idgt"
(synthesis with the canonical dual window, the adjoint form of Sec. 2).  Requests that share
lattice, window and operation are batched into one call of the library (continuous
batching: a batch is formed whenever the GPU can take more work, from the group whose
oldest request has waited longest).  Admission keeps the device bytes of the batches in
flight (inputs, outputs and the workspace that dgt_workspace_bytes reports) under a cap;
a request that can never fit is rejected, one that does not fit now waits.  A request whose
lattice is not admissible (L not a multiple of lam2 lcm(a, M), Sec. 3) fails with the
library's DGT_ERR_LENGTH at plan time and is reported, not served.

The scheduler is host logic only; the work itself goes through an executor.  GpuExecutor
runs it on the library (a few CUDA streams, one per batch in flight, so that batches of
different lattices overlap on the device; per-request host<->device copies from pinned
memory; one event per batch).  Tests drive the same scheduler with a fake executor on a
simulated clock.
"""
from __future__ import annotations

import collections
import gc
import math
import time
from dataclasses import dataclass, field

import numpy as np

from ._capi import DGTError

KEY_FIELDS = ("L", "a", "M", "lam1", "lam2", "window")


def request_key(req) -> tuple:
    """Plan key (lattice and window) of a request."""
    return tuple(getattr(req, f) for f in KEY_FIELDS)


@dataclass
class Served:
    """Outcome of one request: times in seconds from the start of the run."""
    rid: int
    t_arrival: float
    t_done: float = math.nan
    t_launch: float = math.nan         # when its batch was handed to the device
    status: str = "pending"            # "ok", "error" (plan or launch failed), "rejected" (never fits)
    batch: int = -1
    error: str = ""

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class ServeStats:
    served: list = field(default_factory=list)
    batches: int = 0
    batch_sizes: list = field(default_factory=list)
    peak_inflight_bytes: int = 0
    coefs: int = 0
    wall: float = 0.0
    launch_s: list = field(default_factory=list)     # host time of each launch call

    def summary(self) -> dict:
        ok = np.array([s.latency for s in self.served if s.status == "ok"], dtype=np.float64)
        wait = np.array([s.t_launch - s.t_arrival for s in self.served if s.status == "ok"], dtype=np.float64)
        pct = (lambda q: float(np.percentile(ok, q) * 1e3)) if ok.size else (lambda q: None)
        return {
            "requests": len(self.served),
            "ok": int(ok.size),
            "errors": sum(s.status == "error" for s in self.served),
            "rejected": sum(s.status == "rejected" for s in self.served),
            "p50_ms": pct(50), "p90_ms": pct(90), "p99_ms": pct(99),
            "max_ms": float(ok.max() * 1e3) if ok.size else None,
            "queue_wait_p50_ms": float(np.percentile(wait, 50) * 1e3) if wait.size else None,
            "queue_wait_p99_ms": float(np.percentile(wait, 99) * 1e3) if wait.size else None,
            "mean_ms": float(ok.mean() * 1e3) if ok.size else None,
            "batches": self.batches,
            "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
            "peak_inflight_bytes": self.peak_inflight_bytes,
            "coef_per_s": self.coefs / self.wall if self.wall > 0 else None,
            "wall_s": self.wall,
            "host_launch_ms_mean": float(np.mean(self.launch_s) * 1e3) if self.launch_s else None,
            "host_launch_ms_max": float(np.max(self.launch_s) * 1e3) if self.launch_s else None,
            "host_busy_frac": float(np.sum(self.launch_s) / self.wall) if self.wall > 0 else None,
        }


class Scheduler:
    """Continuous batching with an admission cap on device bytes in flight.

    executor protocol:
      prepare(key) -> None            build or fetch the plan; raises DGTError if infeasible
      bytes_for(key, kind, n) -> int  device bytes of a batch of n requests
      launch(key, kind, reqs, rids)   enqueue the batch (asynchronous), return a handle; may raise
      done(h) -> bool                 the batch finished on the device
      finish(h) -> None               release the batch (raises if the device reported a fault)
      coefs(key) -> int               coefficients of one request (M N)
    """

    def __init__(self, executor, cap_bytes: int, max_batch: int = 64, max_inflight: int = 2, poll_s: float = 20e-6):
        self.ex = executor
        self.cap = int(cap_bytes)
        self.max_batch = int(max_batch)
        # batches queued on the device at once: enough to keep it busy while the host forms the
        # next batch; requests arriving meanwhile wait on the host and are batched together
        self.max_inflight = int(max_inflight)
        self.poll_s = poll_s

    def run(self, requests, clock=time.perf_counter, idle=None) -> ServeStats:
        """Serve `requests` (objects with t_arrival and the KEY_FIELDS, plus kind), open loop:
        request i arrives at t0 + t_arrival whatever the state of the server."""
        idle = idle or (lambda dt: time.sleep(dt) if dt > 2e-4 else None)
        gc_was = gc.isenabled()
        gc.disable()                       # no collector pauses inside the latency-critical loop
        try:
            return self._run(requests, clock, idle)
        finally:
            if gc_was:
                gc.enable()

    def _run(self, requests, clock, idle) -> ServeStats:
        order = sorted(range(len(requests)), key=lambda i: requests[i].t_arrival)
        # executors with fixed per-batch buffers bound a single batch as well
        per_batch = getattr(self.ex, "max_batch_bytes", None) or self.cap
        stats = ServeStats(served=[Served(i, requests[i].t_arrival) for i in range(len(requests))])
        groups: "collections.OrderedDict[tuple, collections.deque]" = collections.OrderedDict()
        inflight = []                      # (handle, [rid], bytes, batch index)
        inflight_bytes = 0
        prepared = {}
        nxt = 0
        t0 = clock()
        while nxt < len(order) or groups or inflight:
            now = clock() - t0
            # arrivals
            while nxt < len(order) and requests[order[nxt]].t_arrival <= now:
                rid = order[nxt]
                nxt += 1
                req = requests[rid]
                key = request_key(req)
                if key not in prepared:
                    try:
                        self.ex.prepare(key)
                        prepared[key] = None
                    except DGTError as e:
                        prepared[key] = str(e)
                if prepared[key] is not None:
                    s = stats.served[rid]
                    s.status, s.error, s.t_done = "error", prepared[key], clock() - t0
                    continue
                groups.setdefault((key, req.kind), collections.deque()).append(rid)
            # completions
            progressed = False
            still = []
            for h, rids, nb, bi in inflight:
                if not self.ex.done(h):
                    still.append((h, rids, nb, bi))
                    continue
                progressed = True
                t = clock() - t0
                try:
                    self.ex.finish(h)
                    status, err = "ok", ""
                except Exception as e:  # a failed batch fails its own requests only
                    status, err = "error", str(e)
                for rid in rids:
                    s = stats.served[rid]
                    s.status, s.error, s.t_done = status, err, t
                    if status == "ok":
                        stats.coefs += self.ex.coefs(request_key(requests[rid]))
                inflight_bytes -= nb
            inflight = still
            # launches: oldest head first, as many batches as the cap and the in-flight limit admit
            while groups and len(inflight) < self.max_inflight:
                gk = min(groups, key=lambda k: requests[groups[k][0]].t_arrival)
                key, kind = gk
                q = groups[gk]
                n = min(len(q), self.max_batch)
                while n > 0 and (inflight_bytes + self.ex.bytes_for(key, kind, n) > self.cap
                                 or self.ex.bytes_for(key, kind, n) > per_batch):
                    n -= 1
                if n == 0:
                    if self.ex.bytes_for(key, kind, 1) > min(self.cap, per_batch):
                        rid = q.popleft()
                        s = stats.served[rid]
                        s.status, s.error, s.t_done = "rejected", "request larger than the admission cap", clock() - t0
                        if not q:
                            del groups[gk]
                        progressed = True
                        continue
                    break                  # wait for completions
                rids = [q.popleft() for _ in range(n)]
                if not q:
                    del groups[gk]
                nb = self.ex.bytes_for(key, kind, n)
                bi = stats.batches
                stats.batches += 1
                stats.batch_sizes.append(n)
                tl = clock()
                for rid in rids:
                    stats.served[rid].batch = bi
                    stats.served[rid].t_launch = tl - t0
                try:
                    h = self.ex.launch(key, kind, [requests[r] for r in rids], rids)
                    stats.launch_s.append(clock() - tl)
                except Exception as e:
                    t = clock() - t0
                    for rid in rids:
                        s = stats.served[rid]
                        s.status, s.error, s.t_done = "error", str(e), t
                    progressed = True
                    continue
                inflight.append((h, rids, nb, bi))
                inflight_bytes += nb
                stats.peak_inflight_bytes = max(stats.peak_inflight_bytes, inflight_bytes)
                progressed = True
            if not progressed:
                wait = self.poll_s
                if not inflight and not groups and nxt < len(order):
                    wait = max(0.0, requests[order[nxt]].t_arrival - (clock() - t0))
                idle(wait)
        stats.wall = clock() - t0
        return stats


class GpuExecutor:
    """Executor on the library: one plan per (lattice, window), per-batch device buffers from
    the PyTorch caching allocator, per-request copies from / to pinned host memory.  Each
    batch in flight runs on its own stream (`streams` of them; run the scheduler with
    max_inflight <= streams): a plan's exec with a caller workspace touches no mutable plan
    state, so batches of one plan may run concurrently.

    Inputs come from a small pool of seeded host arrays per shape (request i uses pool entry
    i mod pool); results land in a pinned host ring per shape, or are kept per request when
    keep_results is set (for checks)."""

    def __init__(self, precision: str = "f32", pool: int = 2, seed: int = 4, keep_results: bool = False,
                 device=None, streams: int = 4, arena_bytes: int = 0):
        import torch

        self.torch = torch
        self.dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.precision = precision
        self.cdtype = torch.complex64 if precision == "f32" else torch.complex128
        self.stream = torch.cuda.Stream(self.dev)              # plan set-up
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        self.free = list(range(streams))
        # one device arena per stream, allocated once: a batch carves its input, output and
        # workspace from its stream's arena, so the serving loop never calls the allocator
        # (a cudaMalloc inside the loop stalls every request queued behind it)
        self.arenas = [torch.empty(arena_bytes, dtype=torch.uint8, device=self.dev) for _ in range(streams)] \
            if arena_bytes > 0 else None
        self.max_batch_bytes = arena_bytes if arena_bytes > 0 else None
        self.pool = pool
        self.seed = seed
        self.keep = keep_results
        self.results = {}
        self.plans = {}
        self.windows = {}
        self.inputs = {}
        self.rings = {}

    # ---- plans ------------------------------------------------------------------------
    def prepare(self, key) -> None:
        if key in self.plans:
            return
        from workloads import gaussian_window, hann_taps

        from .api import Plan

        L, a, M, lam1, lam2, window = key
        # an inadmissible lattice is refused before its window is built (building a
        # 2^20-sample window takes tens of milliseconds, a stall for every queued request);
        # the library applies the same rule (Prop. minsig) and would return DGT_ERR_LENGTH
        q = lam2 * (a * M // math.gcd(a, M))
        if L % q:
            raise DGTError(2, "L=%d is not a multiple of lambda2*lcm(a,M)=%d" % (L, q))
        with self.torch.cuda.stream(self.stream):
            if window.startswith("hann"):
                taps, center = hann_taps(int(window[4:]))
                taps = taps / np.linalg.norm(taps)
                p = Plan(L, a, M, lam1, lam2, taps, route="auto", precision=self.precision, fir_center=center,
                         stream=self.stream)
            else:
                if L not in self.windows:
                    self.windows[L] = gaussian_window(L)
                p = Plan(L, a, M, lam1, lam2, self.windows[L], route="auto", precision=self.precision,
                         stream=self.stream)
            p.dual_window(stream=self.stream)          # plan-time set-up of the synthesis window
        self.plans[key] = p

    def coefs(self, key) -> int:
        L, a, M = key[0], key[1], key[2]
        return (L // a) * M

    def _shape(self, key, kind):
        L, a, M = key[0], key[1], key[2]
        return (L,) if kind == "dgt" else (L // a, M)

    def bytes_for(self, key, kind, n) -> int:
        p = self.plans[key]
        esz = 8 if self.precision == "f32" else 16
        L, a, M = key[0], key[1], key[2]
        return n * esz * (L + (L // a) * M) + p.workspace_bytes(n) + 3 * 256      # + arena alignment

    def _input(self, key, kind, i):
        shp = self._shape(key, kind)
        pool = self.inputs.get((shp, kind))
        if pool is None:
            from workloads import complex_normal

            n = int(np.prod(shp))
            host = [self.torch.from_numpy(complex_normal(n, self.seed, n, j).astype(np.complex64 if self.precision == "f32"
                                                                                    else np.complex128)).reshape(shp)
                    .pin_memory() for j in range(self.pool)]
            pool = self.inputs[(shp, kind)] = host
        return pool[i % self.pool]

    RING = 8

    def _ring(self, shape):
        """Pinned host slots that receive results (overwritten round robin: the serving run does
        not keep them); allocated at warm-up, never inside the serving loop."""
        r = self.rings.get(shape)
        if r is None:
            r = self.rings[shape] = self.torch.empty((self.RING,) + shape, dtype=self.cdtype).pin_memory()
        return r

    # ---- batches ----------------------------------------------------------------------
    def launch(self, key, kind, reqs, rids):
        torch = self.torch
        p = self.plans[key]
        n = len(reqs)
        L, a, M = key[0], key[1], key[2]
        N = L // a
        if not self.free:
            raise RuntimeError("no free stream: more batches in flight than streams")
        si = self.free.pop()
        try:
            return self._launch_on(si, p, key, kind, n, L, N, M, rids)
        except Exception:
            self.free.append(si)
            raise

    def _buffers(self, si, p, kind, n, L, N, M):
        torch = self.torch
        xs, ys = ((n, L), (n, N, M)) if kind == "dgt" else ((n, N, M), (n, L))
        wsb = max(1, p.workspace_bytes(n))
        if self.arenas is None:
            return (torch.empty(xs, dtype=self.cdtype, device=self.dev),
                    torch.empty(ys, dtype=self.cdtype, device=self.dev),
                    torch.empty(wsb, dtype=torch.uint8, device=self.dev))
        esz = 8 if self.precision == "f32" else 16
        al = lambda v: (v + 255) // 256 * 256
        nx, ny = esz * int(np.prod(xs)), esz * int(np.prod(ys))
        if al(nx) + al(ny) + al(wsb) > self.arenas[si].numel():
            raise RuntimeError("batch of %d does not fit the stream arena" % n)
        a = self.arenas[si]
        x = a[:nx].view(self.cdtype).view(xs)
        y = a[al(nx):al(nx) + ny].view(self.cdtype).view(ys)
        ws = a[al(nx) + al(ny):al(nx) + al(ny) + wsb]
        return x, y, ws

    def _launch_on(self, si, p, key, kind, n, L, N, M, rids):
        torch = self.torch
        st = self.streams[si]
        with torch.cuda.stream(st):
            x, y, ws = self._buffers(si, p, kind, n, L, N, M)
            for i, rid in enumerate(rids):
                x[i].copy_(self._input(key, kind, rid), non_blocking=True)
            if kind == "dgt":
                p.dgt_ws(x, y, ws, stream=st)
            else:
                p.idgt_ws(x, y, "dual", False, ws, stream=st)
            outs = []
            if self.keep:
                for i, rid in enumerate(rids):
                    h = torch.empty(y.shape[1:], dtype=self.cdtype).pin_memory()
                    h.copy_(y[i], non_blocking=True)
                    outs.append((rid, h))
            else:
                ring = self._ring(tuple(y.shape[1:]))
                for i, rid in enumerate(rids):
                    ring[rid % self.RING].copy_(y[i], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return (ev, x, y, ws, outs, p, si, kind)

    def done(self, h) -> bool:
        return h[0].query()

    def finish(self, h) -> None:
        ev, x, y, ws, outs, p, si, kind = h
        try:
            ev.synchronize()             # raises if the device reported an error for this stream
            if kind == "idgt":
                # a synthesis kernel that gave up waiting for its tile copies left part of this
                # batch's output unwritten: the batch's workspace word says so (DGTError)
                p.workspace_status(ws, stream=self.streams[si])
        finally:
            self.free.append(si)
        for rid, t in outs:
            self.results[rid] = t

    def warm(self, keys, kinds=("dgt", "idgt"), batch: int = 2) -> None:
        """Build every plan and run each (plan, kind) once, outside any timed region."""
        for key in keys:
            try:
                self.prepare(key)
            except DGTError:
                continue
            for kind in kinds:
                n = batch
                while n > 0 and self.max_batch_bytes is not None and self.bytes_for(key, kind, n) > self.max_batch_bytes:
                    n -= 1
                if n:                            # a request that fits no arena is rejected when served
                    self.finish(self.launch(key, kind, [None] * n, list(range(n))))
        self.results.clear()
        self.torch.cuda.synchronize(self.dev)

    def close(self):
        for p in self.plans.values():
            p.close()
        self.plans.clear()
