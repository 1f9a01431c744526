#!/usr/bin/env python
"""DGT coefficient throughput on one GB300: the audio batch workload.

Workload: 64 real pink-noise signals, L = 2^20, a = 128, M = 1024 (N = 8192, b = 1024),
quincunx lattice lambda = 1/2; windows: Hann FIR of length 1024 and the full-length
Gaussian of width sqrt(L).  One step, in float32 on the whole batch:

    Hann (FIR route):          analysis  +  synthesis with the canonical dual
    Gaussian (shear route):    analysis  +  synthesis with the canonical dual
    Gaussian (coset route):    analysis  +  synthesis with the canonical dual

value = DGT coefficients produced or consumed per second over the batch
(6 * 64 * M * N per step), device-timed with CUDA events, inputs resident in HBM.
The same step in float64 is timed separately ("fp64").  Multi-GPU runs are independent
replicas (weak scaling), one process per GPU under torchrun.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DGT coeffs/sec FP32 vs FP64 on 1 GB300, % HBM roofline; serve p50/p99 ms"
UNIT = "coef/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# -------------------------------------------------------------------------------------
# clocks sampled during the timed region
# -------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.time(), parts))

    def mark(self):
        return time.time()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [p for (t, p) in self.rows if t0 - 0.15 <= t <= t1 + 0.15] or [p for (_, p) in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(p[1]) for p in rows if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for p in rows if p[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in rows for i in range(4) if p[5 + i].lower().startswith("active")})
        pw = [float(p[3]) for p in rows if p[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# -------------------------------------------------------------------------------------
# host memory placement of the end-to-end buffers
# -------------------------------------------------------------------------------------
def _cpulist(text):
    out = set()
    for part in text.strip().split(","):
        if not part:
            continue
        if "-" in part:
            lo, hi = part.split("-")
            out.update(range(int(lo), int(hi) + 1))
        else:
            out.add(int(part))
    return out


def gpu_host_locality(index):
    """(NUMA node, CPUs) that sysfs lists as local to the GPU's PCI function, or (None, None)."""
    try:
        bus = subprocess.check_output(["nvidia-smi", "-i", str(index), "--query-gpu=pci.bus_id",
                                       "--format=csv,noheader"], text=True, timeout=20).strip()
        dom, rest = bus.split(":", 1)
        path = "/sys/bus/pci/devices/%04x:%s" % (int(dom, 16), rest.lower())
        node = int(open(os.path.join(path, "numa_node")).read())
        cpus = _cpulist(open(os.path.join(path, "local_cpulist")).read())
        cpus &= os.sched_getaffinity(0)
        return (node if node >= 0 else None), (cpus or None)
    except Exception:
        return None, None


def page_nodes(tensors):
    """NUMA nodes of the first page of each host tensor (move_pages with no target: a query)."""
    import ctypes
    import platform

    nr = {"aarch64": 239, "x86_64": 279}.get(platform.machine())
    if nr is None:
        return None
    try:
        libc = ctypes.CDLL(None, use_errno=True)
        n = len(tensors)
        pages = (ctypes.c_void_p * n)(*[t.data_ptr() for t in tensors])
        status = (ctypes.c_int * n)()
        if libc.syscall(nr, 0, n, pages, None, status, 0) != 0:
            return None
        return sorted({int(v) for v in status})
    except Exception:
        return None


# -------------------------------------------------------------------------------------
# replicas: one process per GPU, each on its own signals; no data-path collective
# -------------------------------------------------------------------------------------
def replica_start(rank: int, batch: int) -> int:
    """Index of the first signal of rank `rank` (signals [start, start + batch) of the stream)."""
    return rank * batch


def max_over_ranks(value: float, world: int, device) -> float:
    """Max of a per-rank float over the process group (timing: the slowest replica)."""
    if world <= 1:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# -------------------------------------------------------------------------------------
# the step
# -------------------------------------------------------------------------------------
def make_plans(w, prec, torch):
    from paper_1307_4569_gb300 import Plan
    from workloads import gaussian_window, hann_taps

    taps, center = hann_taps(1024)
    taps = taps / math.sqrt(float((taps ** 2).sum()))
    g = gaussian_window(w.L)
    plans = [
        ("hann-fir", Plan(w.L, w.a, w.M, w.lam1, w.lam2, taps, route="fir", precision=prec, fir_center=center)),
        ("gauss-shear", Plan(w.L, w.a, w.M, w.lam1, w.lam2, g, route="shear", precision=prec)),
        ("gauss-coset", Plan(w.L, w.a, w.M, w.lam1, w.lam2, g, route="coset", precision=prec)),
    ]
    for _, p in plans:
        p.dual_window()                      # plan-time set-up, outside every timed region
    torch.cuda.synchronize()
    return plans


# full-batch passes of each hot-path kernel in one step (two Zak routes, one FIR route)
PASSES_PER_STEP = {"zak_fwd": 2, "prod_ifft": 2, "fft_post": 2, "pre_ifft": 2, "fft_prod_adj": 2, "zak_inv": 2,
                   "zak_prod_ifft": 2, "fir_analysis": 1, "fir_synthesis": 1}


def flop_model(w, Lg=1024):
    """Flops per coefficient of each route of the step on the workload's lattice, from the
    paper's counts: a separable lattice (a, M) costs 4 L log2 d (Zak transform) + 8 L q (block
    products, p = 1) + 4 M N log2 d + 4 M N log2 M (eq. rect-flops); the coset route runs
    lambda2 separable lattices (lambda2 a, M); the shear route one separable lattice of the same
    size; the FIR route 8 L Lg / a + 4 M N log2 M (eq. rect-flops-FIR)."""
    L, a, M, l2 = w.L, w.a, w.M, w.lam2
    MN = M * (L // a)

    def sep(at):
        c = math.gcd(at, M)
        Nt = L // at
        d = math.gcd(L // M, Nt)
        q = M // c
        MNt = M * Nt
        return 4 * L * math.log2(d) + 8 * L * q + 4 * MNt * math.log2(d) + 4 * MNt * math.log2(M)

    return {"shear": sep(a) / MN, "coset": l2 * sep(l2 * a) / MN, "fir": (8 * L * Lg / a + 4 * MN * math.log2(M)) / MN}


def algorithmic_bytes(name, w, B, csz, rsz, J):
    """Compulsory bytes of one launch of a hot-path kernel for B signals (inputs + outputs)."""
    L, MN = w.L, w.M * w.N
    table = {
        "fir_analysis": B * (L * rsz + MN * csz),
        "fir_synthesis": B * (MN * csz + L * rsz),
        "zak_fwd": B * (L * rsz + L * csz),
        "prod_ifft": B * (L * csz + MN * csz),
        "fft_post": B * 2 * MN * csz,
        "pre_ifft": B * 2 * MN * csz,
        "fft_prod_adj": B * (MN * csz + L * csz),
        "zak_inv": B * (L * csz + L * rsz),
        "zak_prod_ifft": B * (L * rsz + MN * csz),
    }
    return table.get(name)


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_audio_batch_f32.json")


def kernel_sources_sha256() -> str:
    """Hash of the CUDA sources and the C header, in the order the traffic file was hashed."""
    import glob
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1307_4569_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))
                   + glob.glob(os.path.join(csrc, "*.h"))) + [os.path.join(ROOT, "include", "dgt.h")]
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, B):
    """ncu DRAM bytes per launch of `kernel` for B signals, from the committed capture; None when
    the kernels changed since the capture (source hash differs) or the kernel was not captured."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
    except Exception:
        return None, "no capture"
    if d.get("sources_sha256") != kernel_sources_sha256():
        return None, "capture predates the current kernel sources"
    v = d.get("bytes_per_launch", {}).get(kernel)
    if v is None:
        return None, "kernel not captured"
    return v * B / (d["batch_captured"] * d["scale"]), "ncu capture at %d signals scaled to %d" % (
        d["batch_captured"], B)


def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_1307_4569_gb300 import _capi as K
    from workloads import AUDIO_BATCH, signal_batch

    w = AUDIO_BATCH
    B = args.batch or w.batch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    from paper_1307_4569_gb300 import build as bld

    bld.build()

    f_host = torch.from_numpy(signal_batch(w, count=B, cfg_id=1, start=replica_start(rank, B))
                              .astype(np.float32)).pin_memory()
    f = f_host.to(dev)
    coefs_per_step = 6 * B * w.M * w.N

    def step(plans, fin, cbuf, fr):
        for _, p in plans:
            p.dgt(fin, out=cbuf)
            p.idgt(cbuf, window="dual", real=True, out=fr)

    def timed(plans, fin, cbuf, fr, steps, warmup, profile=False):
        for _ in range(warmup):
            step(plans, fin, cbuf, fr)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if profile:
            K.check(K.lib().dgt_profile_start())
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.time()
        e0.record()
        for _ in range(steps):
            step(plans, fin, cbuf, fr)
        e1.record()
        torch.cuda.synchronize()
        t1 = time.time()
        prof = None
        if profile:
            buf = __import__("ctypes").create_string_buffer(1 << 16)
            K.check(K.lib().dgt_profile_stop(buf, len(buf)))
            prof = json.loads(buf.value.decode())
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)
        return ms, prof, t0, t1

    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    # ---------------- float32 (the headline) ----------------
    plans = make_plans(w, "f32", torch)
    cbuf = torch.empty((B, w.N, w.M), dtype=torch.complex64, device=dev)
    fr = torch.empty((B, w.L), dtype=torch.float32, device=dev)
    clocks.start()
    time.sleep(0.3)
    ms, prof, t0, t1 = timed(plans, f, cbuf, fr, args.steps, args.warmup, profile=True)
    value = world * coefs_per_step / (ms * 1e-3)

    # reconstruction check of the timed output (last variant)
    err = float(torch.linalg.vector_norm(fr - f) / torch.linalg.vector_norm(f))

    # ---------------- end to end through the public API, pinned host buffers ----------------
    # Every step copies the signals in from pinned host memory and every route's coefficients
    # and reconstruction back out.  The results leave on one copy stream, route after route, so
    # the device-to-host traffic of one route overlaps the transforms of the next (copies of
    # several routes in flight at once on separate streams shared the link badly: 3-4x slower).
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    nroutes = len(plans)
    # the pinned result buffers are allocated (and so placed) from the CPUs local to the GPU
    node, cpus = gpu_host_locality(dev.index if dev.index is not None else 0)
    old_aff = os.sched_getaffinity(0)
    if cpus:
        os.sched_setaffinity(0, cpus)
    try:
        c_hosts = [torch.empty((B, w.N, w.M), dtype=torch.complex64).pin_memory() for _ in range(nroutes)]
        fr_hosts = [torch.empty((B, w.L), dtype=torch.float32).pin_memory() for _ in range(nroutes)]
    finally:
        os.sched_setaffinity(0, old_aff)
    host_nodes = page_nodes(c_hosts + fr_hosts + [f_host])
    d2h_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nroutes)]
    fr_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nroutes)]
    h2d_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    cbufs = [cbuf] + [torch.empty_like(cbuf) for _ in range(nroutes - 1)]
    frs = [fr] + [torch.empty_like(fr) for _ in range(nroutes - 1)]
    cs = torch.cuda.Stream(dev)
    copied = [None] * nroutes                    # per route: its buffers' copies are done
    fin = torch.empty_like(f)

    def e2e_step():
        cur = torch.cuda.current_stream(dev)
        h2d_ev[0].record(cur)
        fin.copy_(f_host, non_blocking=True)
        h2d_ev[1].record(cur)
        for r, (_, p) in enumerate(plans):
            if copied[r] is not None:
                cur.wait_event(copied[r])        # the previous step's copies of this route's buffers
            p.dgt(fin, out=cbufs[r])
            e_c = torch.cuda.Event()
            e_c.record(cur)
            p.idgt(cbufs[r], window="dual", real=True, out=frs[r])
            e_f = torch.cuda.Event()
            e_f.record(cur)
            with torch.cuda.stream(cs):
                cs.wait_event(e_c)
                d2h_ev[r][0].record(cs)
                c_hosts[r].copy_(cbufs[r], non_blocking=True)
                d2h_ev[r][1].record(cs)
                cs.wait_event(e_f)
                fr_ev[r][0].record(cs)
                fr_hosts[r].copy_(frs[r], non_blocking=True)
                fr_ev[r][1].record(cs)
                copied[r] = torch.cuda.Event()
                copied[r].record(cs)
        cur.wait_stream(cs)                      # the step ends when its results are on the host

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps - 1)]
    a0.record()
    for i in range(e2e_steps):
        e2e_step()
        if i < e2e_steps - 1:
            marks[i].record()
    a1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(a0.elapsed_time(a1) / e2e_steps, world, dev)
    bounds = [a0] + marks + [a1]
    e2e_per_step = [bounds[i].elapsed_time(bounds[i + 1]) for i in range(e2e_steps)]
    d2h_ms = [e0.elapsed_time(e1) for e0, e1 in d2h_ev]          # last step, per route
    fr_ms = [e0.elapsed_time(e1) for e0, e1 in fr_ev]
    h2d_ms = h2d_ev[0].elapsed_time(h2d_ev[1])
    te = time.time()
    clocks.stop()
    clk = clocks.summary(t0, te)
    h2d = B * w.L * 4
    d2h = 3 * (B * w.N * w.M * 8 + B * w.L * 4)

    # ---------------- end to end through the C ABI's host-buffer entry points ----------------
    # Per route: dgt_exec_host (host signals -> host coefficients), then idgt_exec_host (host
    # coefficients -> host reconstruction), chunks of E2E_CHUNK signals, the library's own copy
    # streams overlapping the copies with the transforms; the coefficients cross the host link
    # out and back in.
    E2E_CHUNK = 8
    cur = torch.cuda.current_stream(dev)
    hev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nroutes)]

    def host_step():
        for r, (_, p) in enumerate(plans):
            hev[r][0].record(cur)
            p.dgt_host(f_host, out=c_hosts[r], chunk=E2E_CHUNK)
            hev[r][1].record(cur)
            p.idgt_host(c_hosts[r], window="dual", real=True, out=fr_hosts[r], chunk=E2E_CHUNK)
            hev[r][2].record(cur)

    host_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    hb = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps + 1)]
    hb[0].record()
    for i in range(e2e_steps):
        host_step()
        hb[i + 1].record()
    torch.cuda.synchronize()
    host_per_step = [hb[i].elapsed_time(hb[i + 1]) for i in range(e2e_steps)]
    host_ms = max_over_ranks(hb[0].elapsed_time(hb[-1]) / e2e_steps, world, dev)
    host_ana_ms = [e[0].elapsed_time(e[1]) for e in hev]          # last step, per route
    host_syn_ms = [e[1].elapsed_time(e[2]) for e in hev]
    cbytes = B * w.N * w.M * 8
    host_h2d = 3 * (B * w.L * 4 + cbytes)
    host_d2h = 3 * (cbytes + B * w.L * 4)

    # ---------------- float64 comparison (same step, fewer iterations) ----------------
    fp64 = None
    if args.fp64_steps > 0:
        del plans
        torch.cuda.empty_cache()
        plans64 = make_plans(w, "f64", torch)
        f64 = f.double()
        c64 = torch.empty((B, w.N, w.M), dtype=torch.complex128, device=dev)
        fr64 = torch.empty((B, w.L), dtype=torch.float64, device=dev)
        ms64, _, _, _ = timed(plans64, f64, c64, fr64, args.fp64_steps, 1)
        fp64 = {"value": world * coefs_per_step / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                "steps": args.fp64_steps, "fp32_speedup": ms64 / ms}
        del plans64, c64, fr64, f64
        torch.cuda.empty_cache()

    # ---------------- arithmetic: measured FMA rates and the paper's flop counts ----------------
    import ctypes

    rates = {}
    for kind, name in ((0, "fp32_fma"), (1, "fp32_packed_fma"), (2, "fp64_fma")):
        v = ctypes.c_double()
        K.check(K.lib().dgt_fma_rate(kind, ctypes.byref(v), torch.cuda.current_stream(dev).cuda_stream))
        rates[name + "_tflops"] = v.value / 1e12
    fp32_peak = max(rates["fp32_fma_tflops"], rates["fp32_packed_fma_tflops"])
    fpc = flop_model(w)
    step_flops = 2 * B * w.M * w.N * (fpc["fir"] + fpc["shear"] + fpc["coset"])
    flops = {"model": "the paper's counts (4 n log2 n per FFT of length n, 8 flops per complex product; eq. "
                      "rect-flops per separable lattice, the coset route as lambda2 separable lattices, eq. "
                      "rect-flops-FIR), per coefficient, analysis and synthesis alike",
             "flop_per_coef": fpc, "flop_per_step": step_flops, "tflops": step_flops / (ms * 1e-3) / 1e12,
             "measured_peaks": rates, "frac_of_fp32_peak": step_flops / (ms * 1e-3) / 1e12 / fp32_peak}
    if fp64:
        fp64["tflops"] = step_flops / (fp64["ms_per_step"] * 1e-3) / 1e12
        fp64["frac_of_dfma_peak"] = fp64["tflops"] / rates["fp64_fma_tflops"]

    # ---------------- roofline of the dominant kernel ----------------
    peak, peak_kind = _peaks()
    kernels = {}
    total_prof_ms = sum(v["ms"] for v in prof.values()) if prof else 0.0
    for name, v in (prof or {}).items():
        passes = PASSES_PER_STEP.get(name)
        ab_full = algorithmic_bytes(name, w, B, 8, 4, 2)
        avg = v["ms"] / v["launches"]
        ent = {"launches": v["launches"], "ms_per_launch": avg, "share": v["ms"] / total_prof_ms, "achieved_gbs": None}
        if ab_full and passes:
            # the Zak routes run the batch in passes of a few signals: a launch covers
            # B * passes * steps / launches signals
            sig = B * passes * args.steps / v["launches"]
            ab = ab_full * sig / B
            ent.update({"signals_per_launch": sig, "algorithmic_bytes_per_launch": ab,
                        "achieved_gbs": ab / (avg * 1e-3) / 1e9})
        kernels[name] = ent
    ranked = sorted((k for k in kernels if kernels[k]["achieved_gbs"] is not None), key=lambda k: -kernels[k]["share"])
    dom = ranked[0] if ranked else None
    roof = None
    if dom:
        kd = kernels[dom]
        ach = kd["achieved_gbs"]
        traffic, tnote = measured_traffic(dom, kd["signals_per_launch"])
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_kind": peak_kind, "traffic": traffic, "traffic_note": tnote,
                "algorithmic_bytes_per_launch": kd["algorithmic_bytes_per_launch"],
                "signals_per_launch": kd["signals_per_launch"]}
    launches = sum(v["launches"] for v in (prof or {}).values())
    step_bytes = 3 * 2 * B * (w.L * 4 + w.M * w.N * 8)
    path = {"algorithmic_bytes_per_step": step_bytes, "achieved_gbs": step_bytes / (ms * 1e-3) / 1e9,
            "frac_of_peak": step_bytes / (ms * 1e-3) / 1e9 / peak, "frac_of_8tbs": step_bytes / (ms * 1e-3) / 8e12}

    # ---------------- serving loop (mixed request stream) ----------------
    serve = None
    if args.serve_seconds > 0 and rank == 0:      # replicas: the serving run is a one-GPU measurement
        serve = run_serve(args.serve_seconds)
    others = run_other_configs(dev) if (args.other_configs and rank == 0) else None
    if others is not None:
        # the experiment of Fig. 2: coset and shear analysis times as lambda2 goes from 1 to 10
        others["lambda_sweep"] = run_lambda_sweep(dev, steps=3)

    # ---------------- CPU baseline (oracle), rank 0 only ----------------
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_procs)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "batch": B, "L": w.L, "a": w.a, "M": w.M, "lambda": "%d/%d" % (w.lam1, w.lam2),
                   "windows": ["hann1024-fir", "gauss-full"], "routes": [n for n, _ in make_plan_names()],
                   "step": "analysis + dual synthesis for each of hann-fir, gauss-shear, gauss-coset",
                   "coefs_per_step": coefs_per_step, "l2": "inputs larger than L2 (4.3 GB coefficient array)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "path_roofline": path,
        "kernels": kernels,
        "gpu_launches": launches * 1 if launches else 0,
        "e2e": {"value": world * coefs_per_step / (host_ms * 1e-3), "unit": UNIT, "ms_per_step": host_ms,
                "steps": e2e_steps, "h2d_bytes_per_step": host_h2d, "d2h_bytes_per_step": host_d2h,
                "api": "dgt_exec_host + idgt_exec_host per route (HOST buffers, pinned; chunks of %d signals)" % E2E_CHUNK,
                "per_step_ms": host_per_step, "median_ms_per_step": statistics.median(host_per_step),
                "analysis_ms_per_route": host_ana_ms, "synthesis_ms_per_route": host_syn_ms,
                "coef_out_gbs_per_route": [cbytes / (x * 1e-3) / 1e9 if x > 0 else None for x in host_ana_ms],
                "coef_in_gbs_per_route": [cbytes / (x * 1e-3) / 1e9 if x > 0 else None for x in host_syn_ms],
                "gpu_numa_node": node, "gpu_local_cpus": len(cpus) if cpus else None,
                "pinned_buffer_numa_nodes": host_nodes,
                "resident_coefficients": {
                "what": "the Python API with device-resident coefficients: the signals copied in once, every "
                        "route's coefficients and reconstruction copied out (synthesis from the device copy)",
                "value": world * coefs_per_step / (e2e_ms * 1e-3), "ms_per_step": e2e_ms,
                "steps": e2e_steps, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "coef_copy_ms_per_route": d2h_ms,
                "coef_copy_gbs_per_route": [B * w.N * w.M * 8 / (x * 1e-3) / 1e9 if x > 0 else None for x in d2h_ms],
                "signal_copy_ms_per_route": fr_ms, "input_copy_ms": h2d_ms,
                "per_step_ms": e2e_per_step, "median_ms_per_step": statistics.median(e2e_per_step),
                "link_floor_ms": d2h / (max(B * w.N * w.M * 8 / (x * 1e-3) for x in d2h_ms if x > 0)) * 1e3
                if any(x > 0 for x in d2h_ms) else None,
                "note": "the device-to-host bytes of a step cross the host link, measured at about 193 GB/s by the "
                        "copy engine and by SM stores alike; occasional copies 3-8 times slower than that, at "
                        "changing points of a run of identical steps, raise the mean above the median",
                }},
        "fp64": fp64,
        "flops": flops,
        "clocks": clk,
        "reconstruction_rel_err": err,
        "serve": serve,
        "other_configs": others,
        "cpu_baseline": cpu,
    }
    return line


def _time_cuda(fn, steps, warmup=2):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_other_configs(dev, steps=5):
    """The other workloads, briefly: the lambda = 1/3 batch (both routes, float32 and float64),
    the differentiable batch (analysis + hand-written backward with the window gradient) and
    the small float64 quincunx lattice (launch-bound latency).  Coefficients per second count
    the coefficients produced plus consumed, as in the headline."""
    import numpy as np
    import torch

    from paper_1307_4569_gb300 import Plan
    from paper_1307_4569_gb300 import dgt as dgt_fn
    from workloads import DENSE_THIRD, DIFFERENTIABLE, QUINCUNX_FP64, complex_normal, gaussian_window, \
        noisy_gaussian_window, real_normal, signal_batch

    out = {}
    # lambda = 1/3: 128 complex signals (64 noise, 64 chirps), analysis + dual synthesis per route
    w = DENSE_THIRD
    f64 = signal_batch(w, cfg_id=2)
    g = gaussian_window(w.L)
    res = {}
    keep = {}
    half = w.batch // 2
    for prec, cdt in (("f64", torch.complex128), ("f32", torch.complex64)):
        f = torch.from_numpy(f64.astype(np.complex64 if prec == "f32" else np.complex128)).to(dev)
        c = torch.empty((w.batch, w.N, w.M), dtype=cdt, device=dev)
        fr = torch.empty_like(f)
        for route in ("coset", "shear"):
            p = Plan(w.L, w.a, w.M, w.lam1, w.lam2, g, route=route, precision=prec)
            p.dual_window()

            def step():
                p.dgt(f, out=c)
                p.idgt(c, window="dual", out=fr)

            ms = _time_cuda(step, steps if prec == "f32" else 2)
            err = float(torch.linalg.vector_norm(fr - f) / torch.linalg.vector_norm(f))
            ent = {"ms_per_step": ms, "coef_per_s": 2 * w.batch * w.M * w.N / (ms * 1e-3),
                   "reconstruction_rel_err": err}
            if prec == "f64":
                keep[route] = c.clone()
            else:
                # float32 against the float64 path on the same signals (the float64 path matches
                # the oracle to <= 1e-12 in the tests), per signal, for the noise and chirp halves
                ref = keep[route]
                e = (torch.linalg.vector_norm((c.to(torch.complex128) - ref).reshape(w.batch, -1), dim=1)
                     / torch.linalg.vector_norm(ref.reshape(w.batch, -1), dim=1)).cpu().numpy()
                ent["rel_l2_vs_f64"] = {"noise_max": float(e[:half].max()), "noise_median": float(np.median(e[:half])),
                                        "chirp_max": float(e[half:].max()), "chirp_median": float(np.median(e[half:]))}
            res["%s_%s" % (route, prec)] = ent
            p.close()
        del f, c, fr
    del keep
    out["dense_third"] = {"workload": w.name, "batch": w.batch, "step": "analysis + dual synthesis",
                          "signals": "64 complex N(0,1), then 64 linear chirps 0 -> L/2 with -60 dB noise",
                          "precision_study": "float32 coefficients against the float64 path's, per signal "
                                             "(relative l2 over the signal's M x N block)", **res}
    torch.cuda.empty_cache()
    # differentiable: 32 real float32 signals, learnable window, sum log(|c|^2 + 1e-6)
    from paper_1307_4569_gb300 import log_magnitude_loss

    w = DIFFERENTIABLE
    f = torch.from_numpy(np.stack([real_normal(w.L, 5, i) for i in range(w.batch)]).astype(np.float32)).to(dev)
    gw = torch.from_numpy(noisy_gaussian_window(w.L, 5).astype(np.float32)).to(dev)
    diff = {"workload": w.name, "batch": w.batch,
            "step": "set the learnable window, analysis, loss sum log(|c|^2 + 1e-6) (fused kernel), backward "
                    "(signal and window gradients)"}
    # algorithmic bytes: analysis (real in, complex out), loss (read c, write dl/dc), signal
    # gradient (read dl/dc, write real), window gradient (read f and dl/dc, write L)
    nc = w.batch * w.M * w.N
    diff_bytes = w.batch * w.L * 4 + nc * 8 + 2 * nc * 8 + nc * 8 + w.batch * w.L * 4 + w.batch * w.L * 4 + nc * 8
    for route in ("coset", "shear"):
        p = Plan(w.L, w.a, w.M, w.lam1, w.lam2, gw.cpu().numpy(), route=route, precision="f32")

        def train_step():
            ft = f.requires_grad_(True)
            gt = gw.detach().clone().requires_grad_(True)
            loss = log_magnitude_loss(dgt_fn(ft, gt, p), p)
            loss.backward()

        def eager_step():
            ft = f.requires_grad_(True)
            gt = gw.detach().clone().requires_grad_(True)
            cc = dgt_fn(ft, gt, p)
            loss = torch.log(cc.real ** 2 + cc.imag ** 2 + 1e-6).sum()
            loss.backward()

        ms = _time_cuda(train_step, steps)
        ms_eager = _time_cuda(eager_step, 3)
        cbuf = torch.empty((w.batch, w.N, w.M), dtype=torch.complex64, device=dev)
        lv, G = p.logmag_loss(p.dgt(f, out=cbuf))
        parts = {"set_window_ms": _time_cuda(lambda: p.set_window(gw), steps),
                 "analysis_ms": _time_cuda(lambda: p.dgt(f, out=cbuf), steps),
                 "loss_ms": _time_cuda(lambda: p.logmag_loss(cbuf), steps),
                 "signal_gradient_ms": _time_cuda(lambda: p.idgt(G, window="adjoint", real=True), steps),
                 "window_gradient_ms": _time_cuda(lambda: p.grad_window(f, G), steps)}
        diff[route] = {"ms_per_step": ms, "coef_per_s": nc / (ms * 1e-3), "eager_loss_ms_per_step": ms_eager,
                       "parts": parts, "algorithmic_bytes_per_step": diff_bytes,
                       "achieved_gbs": diff_bytes / (ms * 1e-3) / 1e9}
        del cbuf, G, lv
        p.close()
    best = min(("coset", "shear"), key=lambda r: diff[r]["ms_per_step"])
    diff.update({"route": best, "ms_per_step": diff[best]["ms_per_step"], "coef_per_s": diff[best]["coef_per_s"]})
    out["differentiable"] = diff
    del f, gw
    torch.cuda.empty_cache()
    # blockwise (overlap-add) plans on the audio batch, Hann window of 1024 taps: blocks of
    # 2^14 and 2^16 samples through the coset and the shear route, against the FIR route
    from workloads import AUDIO_BATCH, hann_taps

    w = AUDIO_BATCH
    Bo = 16
    f = torch.from_numpy(signal_batch(w, count=Bo, cfg_id=1).astype(np.float32)).to(dev)
    taps, center = hann_taps(1024)
    taps = taps / np.linalg.norm(taps)
    c = torch.empty((Bo, w.N, w.M), dtype=torch.complex64, device=dev)
    fr = torch.empty_like(f)
    ola = {"workload": w.name, "batch": Bo, "window": "hann1024", "step": "analysis + dual synthesis"}
    for name, kw in (("fir_route", {"route": "fir"}),
                     ("ola_b16384_coset", {"route": "coset", "block_len": 1 << 14}),
                     ("ola_b16384_shear", {"route": "shear", "block_len": 1 << 14}),
                     ("ola_b65536_coset", {"route": "coset", "block_len": 1 << 16})):
        try:
            p = Plan(w.L, w.a, w.M, w.lam1, w.lam2, taps, precision="f32", fir_center=center, **kw)
        except Exception as e:                    # an unsupported block length: say so
            ola[name] = {"unsupported": str(e)[:120]}
            continue
        p.dual_window()

        def step():
            p.dgt(f, out=c)
            p.idgt(c, window="dual", real=True, out=fr)

        ms = _time_cuda(step, steps)
        ent = {"ms_per_step": ms, "coef_per_s": 2 * Bo * w.M * w.N / (ms * 1e-3),
               "reconstruction_rel_err": float(torch.linalg.vector_norm(fr - f) / torch.linalg.vector_norm(f))}
        if "block_len" in kw:
            ent["block_transform_len"] = p.info["ola_len"]
            ent["rho"] = p.info["ola_len"] / kw["block_len"]
        ola[name] = ent
        p.close()
    out["blockwise"] = ola
    del f, c, fr
    torch.cuda.empty_cache()
    # real-signal coefficients (channels 0..M/2) on the audio batch, FIR route, 64 signals:
    # device time and end to end with the coefficients copied to pinned host memory
    B = w.batch
    f = torch.from_numpy(signal_batch(w, count=B, cfg_id=1).astype(np.float32)).to(dev)
    p = Plan(w.L, w.a, w.M, w.lam1, w.lam2, taps, route="fir", precision="f32", fir_center=center)
    p.dual_window()
    c = torch.empty((B, w.N, w.M), dtype=torch.complex64, device=dev)
    ch = torch.empty((B, w.N, w.M // 2 + 1), dtype=torch.complex64, device=dev)
    fr = torch.empty_like(f)
    c_host = torch.empty(c.shape, dtype=c.dtype).pin_memory()
    ch_host = torch.empty(ch.shape, dtype=ch.dtype).pin_memory()
    real = {"workload": w.name, "batch": B, "route": "fir", "window": "hann1024",
            "step": "analysis + dual synthesis; e2e adds the coefficients' copy to pinned host memory"}
    full_ms = _time_cuda(lambda: (p.dgt(f, out=c), p.idgt(c, window="dual", real=True, out=fr)), steps)
    half_ms = _time_cuda(lambda: (p.dgtreal(f, out=ch), p.idgtreal(ch, window="dual", out=fr)), steps)
    full_e2e = _time_cuda(lambda: (p.dgt(f, out=c), c_host.copy_(c, non_blocking=True),
                                   p.idgt(c, window="dual", real=True, out=fr)), 3, 1)
    half_e2e = _time_cuda(lambda: (p.dgtreal(f, out=ch), ch_host.copy_(ch, non_blocking=True),
                                   p.idgtreal(ch, window="dual", out=fr)), 3, 1)
    real.update({"full_ms": full_ms, "real_ms": half_ms, "full_e2e_ms": full_e2e, "real_e2e_ms": half_e2e,
                 "coefficient_bytes_full": c.numel() * 8, "coefficient_bytes_real": ch.numel() * 8,
                 "reconstruction_rel_err": float(torch.linalg.vector_norm(fr - f) / torch.linalg.vector_norm(f))})
    out["real_signal"] = real
    p.close()
    del f, c, ch, fr, c_host, ch_host
    torch.cuda.empty_cache()
    # two-dimensional tensor-product lattice: 4 complex images of 1024 x 1024, lattice
    # (a, M, lambda) = (32, 256, 1/2) on both axes (redundancy 64), Gaussian windows
    from paper_1307_4569_gb300 import Plan2

    lat = (1024, 32, 256, 1, 2)
    g = gaussian_window(1024)
    B2 = 4
    img = torch.from_numpy(np.stack([complex_normal(1 << 20, 61, i).reshape(1024, 1024) for i in range(B2)])
                           .astype(np.complex64)).to(dev)
    p2 = Plan2(lat, g, lat, g, precision="f32")
    c2 = p2.dgt(img)
    ms2 = _time_cuda(lambda: p2.idgt(p2.dgt(img), window="dual"), 3, 1)
    rec = p2.idgt(c2, window="dual")
    out["two_dimensional"] = {"images": B2, "shape": [1024, 1024], "lattice_per_axis": "a=32, M=256, lambda=1/2",
                              "step": "analysis + dual synthesis", "ms_per_step": ms2,
                              "coef_per_s": 2 * c2.numel() / (ms2 * 1e-3),
                              "reconstruction_rel_err": float(torch.linalg.vector_norm(rec - img)
                                                              / torch.linalg.vector_norm(img))}
    p2.close()
    del img, c2, rec
    torch.cuda.empty_cache()
    # small float64 lattice: one signal, analysis + dual synthesis, both routes (latency)
    w = QUINCUNX_FP64
    f = torch.from_numpy(complex_normal(w.L, 1, 0)).to(dev)[None]
    g = gaussian_window(w.L)
    lat = {}
    for route in ("coset", "shear"):
        p = Plan(w.L, w.a, w.M, w.lam1, w.lam2, g, route=route, precision="f64")
        p.dual_window()
        lat[route + "_us"] = 1e3 * _time_cuda(lambda: p.idgt(p.dgt(f), window="dual"), 50, 5)
        p.close()
    out["quincunx_fp64"] = {"workload": w.name, "step": "analysis + dual synthesis of one signal", **lat}
    return out


def run_serve(seconds, rate=2000.0, cap_bytes=40 << 30, seed=4, infeasible_every=500, max_batch=64):
    """The serving workload: Poisson request stream over the four power-of-two lengths (mixed
    lattices, windows and operations, float32) through the continuous-batching scheduler on
    the library.  Plans are built and exercised before the clock starts.  Latency of a request =
    time its result is in pinned host memory - its scheduled arrival time."""
    import torch

    from paper_1307_4569_gb300.serve import GpuExecutor, Scheduler, request_key
    from workloads import serve_requests

    reqs = serve_requests(rate, seconds, seed=seed, infeasible_every=infeasible_every)
    ex = GpuExecutor("f32", streams=4, arena_bytes=cap_bytes // 4, pool=8)
    keys = sorted({request_key(r) for r in reqs if r.feasible})
    t0 = time.time()
    ex.warm(keys)
    warm_s = time.time() - t0
    st = Scheduler(ex, cap_bytes, max_batch=max_batch, max_inflight=len(ex.streams)).run(reqs)
    out = st.summary()
    import numpy as np

    by_len = {}
    for L in sorted({r.L for r in reqs}):
        lat = [s.latency for s, r in zip(st.served, reqs) if r.L == L and s.status == "ok"]
        if lat:
            by_len[str(L)] = {"n": len(lat), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                              "p99_ms": float(np.percentile(lat, 99) * 1e3)}
    out["by_length"] = by_len
    out.update({"rate_per_s": rate, "seconds": seconds, "cap_bytes": cap_bytes, "plans": len(keys),
                "plan_warmup_s": warm_s, "redraws": int(sum(r.redraws for r in reqs)),
                "latency": "result in pinned host memory - scheduled arrival (open loop)",
                "precision": "f32", "input_pool_per_shape": ex.pool,
                "accuracy": "float32 results; the serving tests hold every served result within 2e-6 relative "
                            "l2 of the float64 oracle and bit-identical alone and in the mix"})
    ex.close()
    torch.cuda.synchronize()
    return out


def run_lambda_sweep(dev, steps=5, batch=8):
    """The experiment of Fig. 2 on the GPU: time of the coset and the shear route of one
    analysis as lambda2 goes from 1 to 10 (lambda1 = 1), for (a, M) in {(32, 64), (40, 60),
    (60, 80)} and L = lcm(a, M) * 2520 (admissible for every lambda2 <= 10), float32,
    `batch` complex N(0,1) signals, periodised Gaussian window."""
    import math

    import numpy as np
    import torch

    from paper_1307_4569_gb300 import Plan
    from workloads import complex_normal, gaussian_window

    rows = []
    for a, M in ((32, 64), (40, 60), (60, 80)):
        L = a * M // math.gcd(a, M) * 2520
        f = torch.from_numpy(np.stack([complex_normal(L, 77, i) for i in range(batch)]).astype(np.complex64)).to(dev)
        g = gaussian_window(L)
        c = torch.empty((batch, L // a, M), dtype=torch.complex64, device=dev)
        for lam2 in range(1, 11):
            lam1 = 0 if lam2 == 1 else 1
            ent = {"a": a, "M": M, "L": L, "lambda2": lam2}
            for route in ("coset", "shear"):
                try:
                    p = Plan(L, a, M, lam1, lam2, g, route=route, precision="f32")
                except Exception as e:
                    ent[route] = {"unsupported": str(e)[:100]}
                    continue
                ms = _time_cuda(lambda: p.dgt(f, out=c), steps)
                ent[route] = {"ms": ms, "coef_per_s": batch * M * (L // a) / (ms * 1e-3), "s0": p.info["s0"]}
                p.close()
            if "ms" in ent.get("coset", {}) and "ms" in ent.get("shear", {}):
                ent["shear_over_coset"] = ent["shear"]["ms"] / ent["coset"]["ms"]
            rows.append(ent)
        del f, c
        torch.cuda.empty_cache()
    return rows


def make_plan_names():
    return [("hann-fir", None), ("gauss-shear", None), ("gauss-coset", None)]


# -------------------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline leg and the reference arm)
# -------------------------------------------------------------------------------------
def _oracle_signal_pass(idx):
    """One signal of the workload through the oracle: analysis + synthesis with the canonical
    dual for the Hann window (expanded to full length) and the Gaussian on both routes."""
    import numpy as np

    from oracle import dgt as OD
    from oracle import duals as OU
    from workloads import AUDIO_BATCH, gaussian_window, hann_window, signal_batch

    w = AUDIO_BATCH
    f = signal_batch(w, count=1, cfg_id=1, start=idx)[0]
    gh = hann_window(w.L, 1024)
    gg = gaussian_window(w.L)
    gdh = OU.fir_dual_diag(gh, w.a, w.M)
    gdg = OU.zak_gram_dual(gg, w.a, w.M, w.lam1, w.lam2)
    t0 = time.time()
    c = OD.dgt_coset(f, gh, w.a, w.M, w.lam1, w.lam2)
    OD.idgt_coset(c, gdh, w.a, w.M, w.lam1, w.lam2)
    c = OD.dgt_shear(f, gg, w.a, w.M, w.lam1, w.lam2)
    OD.idgt_shear(c, gdg, w.a, w.M, w.lam1, w.lam2)
    c = OD.dgt_coset(f, gg, w.a, w.M, w.lam1, w.lam2)
    OD.idgt_coset(c, gdg, w.a, w.M, w.lam1, w.lam2)
    return t0, time.time()


def cpu_baseline(max_procs=16):
    """The oracle as it stands on the host cores: one signal per spawned process (numpy's FFT
    is single-threaded), all processes at once; throughput = coefficients / (last end - first
    start) over the timed passes (window set-up excluded)."""
    import multiprocessing as mp

    from workloads import AUDIO_BATCH

    w = AUDIO_BATCH
    cores = len(os.sched_getaffinity(0))
    nproc = max(1, min(cores, max_procs))
    ctx = mp.get_context("spawn")
    with ctx.Pool(nproc) as pool:
        spans = pool.map(_oracle_signal_pass, range(nproc))
    wall = max(e for _, e in spans) - min(s for s, _ in spans)
    single = statistics.median(e - s for s, e in spans)
    coefs = nproc * 6 * w.M * w.N
    return {"value": coefs / wall, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": "%d signals of the 64-signal audio batch, one per process; each: analysis + dual synthesis "
                      "for hann (full-length, coset), gauss shear, gauss coset (median %.1f s per signal)"
                      % (nproc, single),
            "host_cores": cores, "single_signal_s": single}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from workloads import AUDIO_BATCH

    w = AUDIO_BATCH
    cores = 1
    times = []
    for i in range(args.steps):
        s0, s1 = _oracle_signal_pass(i)
        times.append(s1 - s0)
    ms = 1e3 * sum(times) / len(times)
    coefs = 6 * w.M * w.N
    v = coefs / (ms * 1e-3)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "batch_sample": 1, "L": w.L, "a": w.a, "M": w.M,
                       "step": "one signal of the batch through the CPU oracle (analysis + dual synthesis, "
                               "hann / gauss-shear / gauss-coset)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "1 signal per step of the 64-signal batch"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=16)
    ap.add_argument("--batch", type=int, default=0, help="signals per step (default: the workload's 64)")
    ap.add_argument("--other-configs", type=int, default=1, help="1: also time the other workloads briefly")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="run only the serving loop at rising request rates and under a 256 MB admission cap, "
                         "and print its rows as one JSON line")
    ap.add_argument("--lambda-sweep", action="store_true",
                    help="run only the coset / shear timing sweep over lambda2 = 1..10 (Fig. 2 setups) and "
                         "print its rows as one JSON line")
    ap.add_argument("--dense-third", choices=["coset", "shear"], default=None,
                    help="run only the lambda = 1/3 float32 step (128 signals, analysis + dual synthesis) on this "
                         "route, --steps times after 2 warm-up steps, and print one JSON line")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the serving run (Poisson 2000 requests/s); 0 skips it")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.serve_sweep:
        from paper_1307_4569_gb300 import build as bld

        bld.build()
        rows = []
        for rate in (2000, 4000, 8000, 16000, 32000):
            r = run_serve(5.0, rate=rate)
            rows.append({k: r[k] for k in ("rate_per_s", "requests", "ok", "p50_ms", "p99_ms", "max_ms",
                                            "queue_wait_p99_ms", "mean_batch", "coef_per_s", "host_busy_frac")})
        r = run_serve(5.0, rate=2000, cap_bytes=256 << 20)
        rows.append({"cap_bytes": 256 << 20, **{k: r[k] for k in ("rate_per_s", "requests", "ok", "rejected", "p50_ms",
                                                                   "p99_ms", "max_ms", "peak_inflight_bytes",
                                                                   "mean_batch")}})
        print(json.dumps({"serve_sweep": rows}), flush=True)
        return
    if args.dense_third:
        import numpy as np
        import torch

        from paper_1307_4569_gb300 import Plan
        from paper_1307_4569_gb300 import build as bld
        from workloads import DENSE_THIRD, gaussian_window, signal_batch

        bld.build()
        w, dev = DENSE_THIRD, torch.device("cuda", 0)
        f = torch.from_numpy(signal_batch(w, cfg_id=2).astype(np.complex64)).to(dev)
        c = torch.empty((w.batch, w.N, w.M), dtype=torch.complex64, device=dev)
        fr = torch.empty_like(f)
        p = Plan(w.L, w.a, w.M, w.lam1, w.lam2, gaussian_window(w.L), route=args.dense_third, precision="f32")
        p.dual_window()
        ms = _time_cuda(lambda: (p.dgt(f, out=c), p.idgt(c, window="dual", out=fr)), args.steps)
        err = float(torch.linalg.vector_norm(fr - f) / torch.linalg.vector_norm(f))
        print(json.dumps({"dense_third": {"workload": w.name, "route": args.dense_third, "ms_per_step": ms,
                                          "reconstruction_rel_err": err, "plan": p.info}}), flush=True)
        return
    if args.lambda_sweep:
        import torch

        from paper_1307_4569_gb300 import build as bld

        bld.build()
        print(json.dumps({"lambda_sweep": run_lambda_sweep(torch.device("cuda", 0))}), flush=True)
        return
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    if world > 1:
        import torch

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch

        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
