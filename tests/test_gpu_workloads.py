"""GPU parity at workload scale.

Medium power-of-two lattices are checked in full against the oracle; the full-size
workloads (in the launch configuration the benchmark times) are checked on sampled
time positions, which the oracle's fold form computes one by one in O(L), plus properties
that hold at any size (coset and shear routes agree; perfect reconstruction).
Tolerances: float64 1e-12, float32 2e-6 relative l2 (per block / per sampled column group,
float32 against the oracle on the float32-rounded inputs).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from oracle import duals as OU  # noqa: E402
from oracle import grads as OG  # noqa: E402
from workloads import (AUDIO_BATCH, DENSE_THIRD, DIFFERENTIABLE, complex_normal, gaussian_window,  # noqa: E402
                       hann_taps, hann_window, noisy_gaussian_window, real_normal, signal_batch)

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _plan(*a, **k):
    from paper_1307_4569_gb300 import Plan

    return Plan(*a, **k)


def _round(x, prec):
    if prec == "f64":
        return x
    return x.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(x) else x.astype(np.float32).astype(np.float64)


def _dev(x, prec):
    if np.iscomplexobj(x):
        return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex128 if prec == "f64" else np.complex64))).cuda()
    return torch.from_numpy(np.ascontiguousarray(x.astype(np.float64 if prec == "f64" else np.float32))).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# -------------------------------------------------------------------------------------
# medium power-of-two lattices: every coefficient, every route
# -------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("lam", [(1, 2), (1, 4), (0, 1)])
def test_medium_pow2_full(prec, lam):
    L, a, M = 65536, 64, 512
    l1, l2 = lam
    g = gaussian_window(L)
    rng = np.random.default_rng(8)
    B = 2
    f = rng.standard_normal((B, L)) + 1j * rng.standard_normal((B, L))
    refs = [OD.dgt_coset(_round(f[b], prec), _round(g, prec), a, M, l1, l2).T for b in range(B)]
    for route in ("coset", "shear"):
        p = _plan(L, a, M, l1, l2, _round(g, prec), route=route, precision=prec)
        c = p.dgt(_dev(_round(f, prec), prec))
        cn = c.cpu().numpy()
        for b in range(B):
            assert _rel(cn[b], refs[b]) <= TOL[prec], (route, b, p.info)
        fr = p.idgt(c, window="dual").cpu().numpy()
        for b in range(B):
            assert _rel(fr[b], _round(f[b], prec)) <= (1e-12 if prec == "f64" else 1e-5)
        p.status()                      # no bounded device wait expired
        p.close()
    # FIR route with a Hann window of length M
    taps, center = hann_taps(M)
    taps = taps / np.linalg.norm(taps)
    gh = hann_window(L, M)
    p = _plan(L, a, M, l1, l2, _round(taps, prec), route="fir", precision=prec, fir_center=center)
    c = p.dgt(_dev(_round(f, prec), prec)).cpu().numpy()
    for b in range(B):
        ref = OD.dgt_coset(_round(f[b], prec), _round(gh, prec), a, M, l1, l2).T
        assert _rel(c[b], ref) <= TOL[prec]
    p.close()


# -------------------------------------------------------------------------------------
# audio batch at full size (64 real pink-noise signals, L = 2^20), bench launch configuration
# -------------------------------------------------------------------------------------
def _sampled_check(c_dev, f, g, w, prec, signals, cols):
    for b in signals:
        ref = OD.dgt_fold(_round(f[b], prec), _round(g, prec), w.a, w.M, w.lam1, w.lam2, cols=cols)   # (M, len(cols))
        got = c_dev[b, cols, :].cpu().numpy().T
        assert _rel(got, ref) <= TOL[prec], (b, _rel(got, ref))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_audio_batch_full_size(prec):
    w = AUDIO_BATCH
    B = w.batch if prec == "f32" else 8
    f = signal_batch(w, count=B, cfg_id=1)
    fd = _dev(_round(f, prec), prec)
    g = gaussian_window(w.L)
    cols = [0, 1, 2, 4095, 4096, 8190, 8191, 1234]
    sig = [0, B // 2, B - 1]
    ps = _plan(w.L, w.a, w.M, w.lam1, w.lam2, _round(g, prec), route="shear", precision=prec)
    cs = ps.dgt(fd)
    _sampled_check(cs, f, g, w, prec, sig, cols)
    pc = _plan(w.L, w.a, w.M, w.lam1, w.lam2, _round(g, prec), route="coset", precision=prec)
    cc = pc.dgt(fd)
    # coset and shear agree everywhere
    for b in sig:
        assert float(torch.linalg.vector_norm(cc[b] - cs[b]) / torch.linalg.vector_norm(cs[b])) <= 2 * TOL[prec]
    fr = pc.idgt(cc, window="dual", real=True)
    err = float(torch.linalg.vector_norm(fr - fd) / torch.linalg.vector_norm(fd))
    assert err <= (1e-12 if prec == "f64" else 1e-5)
    ps.status()
    pc.status()
    del cc, cs, fr
    ps.close()
    pc.close()
    taps, center = hann_taps(1024)
    taps = taps / np.linalg.norm(taps)
    gh = hann_window(w.L, 1024)
    ph = _plan(w.L, w.a, w.M, w.lam1, w.lam2, _round(taps, prec), route="fir", precision=prec, fir_center=center)
    ch = ph.dgt(fd)
    _sampled_check(ch, f, gh, w, prec, sig, cols)
    fr = ph.idgt(ch, window="dual", real=True)
    assert float(torch.linalg.vector_norm(fr - fd) / torch.linalg.vector_norm(fd)) <= (1e-12 if prec == "f64" else 1e-5)
    ph.close()


# -------------------------------------------------------------------------------------
# the lambda = 1/3 lattice (L = 172800): frequency-shear branch, complex signals and chirps
# -------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_dense_third_full_size(prec):
    w = DENSE_THIRD
    B = w.batch if prec == "f32" else 16
    idx = list(range(B // 2)) + list(range(w.batch // 2, w.batch // 2 + B // 2))
    f = np.stack([signal_batch(w, count=1, cfg_id=2, start=i)[0] for i in idx])
    g = gaussian_window(w.L)
    fd = _dev(_round(f, prec), prec)
    cols = [0, 1, 2, 3, 1439, 1440, 2879, 777]
    sig = [0, B // 2 - 1, B // 2, B - 1]
    outs = {}
    for route in ("coset", "shear"):
        p = _plan(w.L, w.a, w.M, w.lam1, w.lam2, _round(g, prec), route=route, precision=prec)
        if route == "shear":
            assert p.info["s0"] != 0
        c = p.dgt(fd)
        _sampled_check(c, f, g, w, prec, sig, cols)
        outs[route] = c
        p.close()
    for b in sig:
        assert float(torch.linalg.vector_norm(outs["coset"][b] - outs["shear"][b])
                     / torch.linalg.vector_norm(outs["shear"][b])) <= 2 * TOL[prec]
    # tight window: Parseval on the GPU for the sampled signals
    p = _plan(w.L, w.a, w.M, w.lam1, w.lam2, _round(g, prec), route="coset", precision=prec)
    gt = p.tight_window()
    ref_gt = OU.zak_gram_tight(_round(g, prec), w.a, w.M, w.lam1, w.lam2)
    assert _rel(gt.cpu().numpy(), ref_gt) <= TOL[prec] * 5
    pt = _plan(w.L, w.a, w.M, w.lam1, w.lam2, gt.cpu().numpy(), route="shear", precision=prec)
    ct = pt.dgt(fd)
    for b in sig:
        ratio = float(torch.linalg.vector_norm(ct[b]) ** 2 / torch.linalg.vector_norm(fd[b]) ** 2)
        assert abs(ratio - 1) <= (1e-12 if prec == "f64" else 1e-5)


# -------------------------------------------------------------------------------------
# differentiable workload at full size: gradients of one signal against the oracle
# -------------------------------------------------------------------------------------
def test_differentiable_full_size_gradients():
    from paper_1307_4569_gb300 import dgt as dgt_fn

    w = DIFFERENTIABLE
    prec = "f64"
    f = real_normal(w.L, 5, 0)[None, :]
    g = noisy_gaussian_window(w.L, 5)
    p = _plan(w.L, w.a, w.M, w.lam1, w.lam2, g, precision=prec)
    ft = _dev(f, prec).requires_grad_(True)
    gt = _dev(g, prec).requires_grad_(True)
    c = dgt_fn(ft, gt, p)
    loss = torch.log(c.real ** 2 + c.imag ** 2 + 1e-6).sum()
    loss.backward()
    lv, gf, gg = OG.grads(f[0], g, w.a, w.M, w.lam1, w.lam2)
    assert abs(loss.item() - lv) <= 1e-10 * abs(lv)
    assert _rel(ft.grad.cpu().numpy()[0], gf) <= 1e-10
    assert _rel(gt.grad.cpu().numpy(), gg) <= 1e-10


# -------------------------------------------------------------------------------------
# M = 16384 (the largest serving lattice, L = 2^20, a = 2048): the 16384-point float row path
# -------------------------------------------------------------------------------------
@pytest.mark.parametrize("lam", [(1, 2), (0, 1)])
def test_rows_16384_f32(lam):
    L, a, M = 1 << 18, 1024, 16384
    l1, l2 = lam
    prec = "f32"
    g = gaussian_window(L)
    f = complex_normal(L, 21, l2)[None, :]
    ref = OD.dgt_coset(_round(f[0], prec), _round(g, prec), a, M, l1, l2).T
    for route in ("coset", "shear"):
        p = _plan(L, a, M, l1, l2, _round(g, prec), route=route, precision=prec)
        c = p.dgt(_dev(_round(f, prec), prec))
        assert _rel(c.cpu().numpy()[0], ref) <= TOL[prec], (route, p.info)
        fr = p.idgt(c, window="dual").cpu().numpy()
        assert _rel(fr[0], _round(f[0], prec)) <= 1e-5
        p.status()
        p.close()
    # float64 rows of this length do not fit one CTA: the coset route (rows of length M) says so
    from paper_1307_4569_gb300 import DGTError

    with pytest.raises(DGTError, match="DGT_ERR_UNSUPPORTED"):
        _plan(L, a, M, l1, l2, g, route="coset", precision="f64")
