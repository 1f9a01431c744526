"""Run in a child process with DGT_DEBUG=1 (libdgt_debug.so, the guard-zone bounds-checking
build): analysis and synthesis of the coset, shear (both branches), FIR and mixed-radix paths,
the real-signal half coefficients, caller workspaces and the dual-window set-up, each compared
with the float64 oracle on seeded inputs, with no guard word of the library overwritten and
the caller's output buffers untouched outside their extent; then a guard word damaged on
purpose (inside the library's own allocation) must be reported by the next launch's check.
Prints one JSON line; exits non-zero on any failure."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import dgt as OD  # noqa: E402
from oracle import dgtreal as OR  # noqa: E402
from oracle import duals as OU  # noqa: E402
from workloads import complex_normal, gaussian_window, hann_taps, real_normal  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}
PAD = 4096                      # elements of 0xFF padding on each side of a caller buffer


def rnd(x, prec):
    if prec == "f64":
        return x
    return x.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(x) else x.astype(np.float32).astype(np.float64)


def dev(x, prec):
    if np.iscomplexobj(x):
        return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex128 if prec == "f64" else np.complex64))).cuda()
    return torch.from_numpy(np.ascontiguousarray(x.astype(np.float64 if prec == "f64" else np.float32))).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class Guarded:
    """A caller buffer of `shape` inside PAD elements of 0xFF bytes on each side."""

    def __init__(self, shape, dtype):
        self.n = int(np.prod(shape))
        self.buf = torch.empty(self.n + 2 * PAD, dtype=dtype, device="cuda")
        self.buf.view(torch.uint8).fill_(0xFF)
        self.t = self.buf[PAD:PAD + self.n].view(shape)

    def intact(self):
        u = self.buf.view(torch.uint8)
        es = self.buf.element_size()
        return bool((u[:PAD * es] == 255).all()) and bool((u[(PAD + self.n) * es:] == 255).all())


def main():
    from paper_1307_4569_gb300 import Plan, _capi as K, debug_status

    assert K.LIB_PATH.endswith("libdgt_debug.so"), K.LIB_PATH
    assert K.lib().dgt_debug_build() == 1
    debug_status()                                  # start from a clean record
    report = []

    def finish(case, errs, bufs):
        v, kern, off = debug_status()
        ok = v == 0 and all(b.intact() for b in bufs) and all(e <= TOL[case["prec"]] for e in errs)
        finite = all(bool(torch.isfinite(torch.view_as_real(b.t) if b.t.is_complex() else b.t).all()) for b in bufs)
        case.update(errs=errs, violations=v, kernel=kern, finite=finite, ok=ok and finite)
        report.append(case)
        assert case["ok"], case

    # ---- Zak routes: power-of-two (fused Zak kernels), generic small lattices, mixed radix
    zak_cases = [(16384, 32, 512, 1, 2), (36, 6, 6, 1, 2), (72, 2, 4, 1, 6), (2880, 60, 240, 1, 2)]
    for (L, a, M, l1, l2) in zak_cases:
        N = L // a
        for prec in ("f32", "f64"):
            g = rnd(gaussian_window(L), prec)
            for route in ("coset", "shear"):
                p = Plan(L, a, M, l1, l2, g, route=route, precision=prec)
                B = 2
                f = np.stack([rnd(complex_normal(L, 61, L, i), prec) for i in range(B)])
                cols = sorted(set([0, 1, N // 2, N - 1]))
                co = Guarded((B, N, M), p.cdtype)
                p.dgt(dev(f, prec), out=co.t)
                c = co.t.cpu().numpy()
                errs = [rel(c[b][cols].T, OD.dgt_fold(f[b], g, a, M, l1, l2, cols=cols)) for b in range(B)]
                cc = rnd(complex_normal(N * M, 62, L, 1).reshape(N, M), prec)
                fo = Guarded((1, L), p.cdtype)
                p.idgt(dev(cc[None], prec), window="adjoint", out=fo.t)
                errs.append(rel(fo.t.cpu().numpy()[0], OD.idgt_fold(cc.T, g, a, M, l1, l2)))
                finish(dict(path="zak", L=L, a=a, M=M, lam=(l1, l2), prec=prec, route=p.route,
                            branch="freq" if p.info["s0"] else "time"), errs, [co, fo])
                p.close()

    # ---- FIR route (real-input pairing in float32), analysis + real synthesis + half spectrum
    L, a, M, l1, l2, Lg = 16384, 128, 1024, 1, 2, 1024
    taps, center = hann_taps(Lg)
    taps = taps / np.linalg.norm(taps)
    gfull = np.zeros(L)
    gfull[(np.arange(Lg) - center) % L] = taps
    N = L // a
    for prec in ("f32", "f64"):
        p = Plan(L, a, M, l1, l2, rnd(taps, prec), route="fir", precision=prec, fir_center=center)
        B = 2
        f = np.stack([rnd(real_normal(L, 63, i), prec) for i in range(B)])
        co = Guarded((B, N, M), p.cdtype)
        p.dgt(dev(f, prec), out=co.t)
        c = co.t.cpu().numpy()
        gr = rnd(gfull, prec)
        errs = [rel(c[b].T, OD.dgt_fold(f[b], gr, a, M, l1, l2)) for b in range(B)]
        cc = rnd(OD.dgt_fold(f[0], gr, a, M, l1, l2), prec)          # the oracle's [m, n]
        fo = Guarded((1, L), p.rdtype)
        p.idgt(dev(np.ascontiguousarray(cc.T)[None], prec), window="adjoint", real=True, out=fo.t)
        errs.append(rel(fo.t.cpu().numpy()[0], OD.idgt_fold(cc, gr, a, M, l1, l2).real))
        ho = Guarded((B, N, M // 2 + 1), p.cdtype)
        p.dgtreal(dev(f, prec), out=ho.t)
        h = ho.t.cpu().numpy()
        errs += [rel(h[b], OR.dgtreal(f[b], gr, a, M, l1, l2).T) for b in range(B)]
        finish(dict(path="fir", L=L, a=a, M=M, lam=(l1, l2), prec=prec), errs, [co, fo, ho])
        p.close()

    # ---- caller workspaces (guard zones between the workspace's regions) and the dual window
    L, a, M, l1, l2 = 16384, 32, 512, 1, 2
    N = L // a
    g = rnd(gaussian_window(L), "f32")
    for route in ("coset", "shear"):
        p = Plan(L, a, M, l1, l2, g, route=route, precision="f32")
        B = 2
        f = np.stack([rnd(complex_normal(L, 64, i), "f32") for i in range(B)])
        ws = torch.empty(p.workspace_bytes(B), dtype=torch.uint8, device="cuda")
        co = Guarded((B, N, M), p.cdtype)
        p.dgt_ws(dev(f, "f32"), co.t, ws)
        c = co.t.cpu().numpy()
        cols = [0, 7, N - 1]
        errs = [rel(c[b][cols].T, OD.dgt_fold(f[b], g, a, M, l1, l2, cols=cols)) for b in range(B)]
        cc = rnd(complex_normal(N * M, 65, 0).reshape(N, M), "f32")
        fo = Guarded((1, L), p.cdtype)
        p.idgt_ws(dev(cc[None], "f32"), fo.t, "adjoint", False, ws)
        p.workspace_status(ws)
        errs.append(rel(fo.t.cpu().numpy()[0], OD.idgt_fold(cc.T, g, a, M, l1, l2)))
        finish(dict(path="workspace", L=L, a=a, M=M, prec="f32", route=p.route), errs, [co, fo])
        p.close()
    L, a, M, l1, l2 = 240, 4, 12, 1, 4
    g = gaussian_window(L)
    for route in ("coset", "shear"):
        p = Plan(L, a, M, l1, l2, g, route=route, precision="f64")
        d = p.dual_window().cpu().numpy()
        finish(dict(path="dual", L=L, a=a, M=M, prec="f64", route=p.route), [rel(d, OU.dense_dual(g, a, M, l1, l2))], [])
        p.close()

    # ---- the checker itself: one guard word damaged inside the library's own allocation
    L, a, M, l1, l2 = 16384, 32, 512, 1, 2
    p = Plan(L, a, M, l1, l2, gaussian_window(L), route="coset", precision="f32")
    f = dev(rnd(complex_normal(L, 66, 0), "f32")[None], "f32")
    p.dgt(f)
    assert debug_status()[0] == 0
    K.check(K.lib().dgt_debug_touch_guard(p._h))
    p.dgt(f)
    v, kern, off = debug_status()
    assert v == 1 and kern and off == 0, (v, kern, off)
    p.dgt(f)                                         # the word was restored: nothing new
    v2 = debug_status()[0]
    assert v2 == 0, v2
    report.append(dict(path="detector", violations=v, kernel=kern, zone_offset=off, after=v2, ok=True))
    p.close()
    print(json.dumps({"cases": len(report), "ok": all(r["ok"] for r in report), "report": report}))


if __name__ == "__main__":
    main()
