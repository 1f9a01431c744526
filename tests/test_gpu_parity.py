"""GPU parity: the CUDA path through the C ABI against the float64 CPU oracle.

Tolerances (relative l2 error per signal's coefficient block):
  float64: 1e-12;  float32: 2e-6 against the oracle applied to the float32-rounded inputs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from oracle import duals as OU  # noqa: E402
from oracle import grads as OG  # noqa: E402
from oracle import lattice as OL  # noqa: E402
from workloads import complex_normal, gaussian_window, hann_taps, hann_window, real_normal  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _P():
    from paper_1307_4569_gb300 import Plan

    return Plan


def _round(x, prec):
    if prec == "f64":
        return x
    return x.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(x) else x.astype(np.float32).astype(np.float64)


def _to_dev(x, prec):
    if np.iscomplexobj(x):
        t = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex128 if prec == "f64" else np.complex64)))
    else:
        t = torch.from_numpy(np.ascontiguousarray(x.astype(np.float64 if prec == "f64" else np.float32)))
    return t.cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _ref_dgt(f, g, a, M, l1, l2):
    return OD.dgt_direct(f, g, a, M, l1, l2) if f.shape[0] <= 96 else OD.dgt_fold(f, g, a, M, l1, l2)


# -------------------------------------------------------------------------------------
# FFT building block
# -------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fft_building_block(prec):
    from paper_1307_4569_gb300 import fft_selftest

    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 4, 5, 7, 8, 15, 16, 32, 45, 48, 96, 128, 180, 240, 360, 480, 512, 720, 960, 1024, 1440,
              2048, 4096, 6144):
        if prec == "f64" and n > 4096:
            continue
        x = rng.standard_normal((5, n)) + 1j * rng.standard_normal((5, n))
        xd = _to_dev(_round(x, prec), prec)
        for direction in (-1, 1):
            y = fft_selftest(xd, direction).cpu().numpy()
            ref = np.fft.fft(_round(x, prec), axis=1) if direction < 0 else np.fft.ifft(_round(x, prec), axis=1) * n
            assert _rel(y, ref) <= (1e-14 * (1 + np.log2(n)) if prec == "f64" else 1e-6), (n, direction)


# -------------------------------------------------------------------------------------
# small lattices: every route and branch
# -------------------------------------------------------------------------------------
SMALL = [
    (36, 6, 6, 0, 1),       # separable (Fig. 1 a)
    (36, 6, 6, 1, 2),       # quincunx (Fig. 1 b), frequency shear
    (36, 6, 6, 1, 3),       # Fig. 1 c
    (36, 6, 6, 2, 3),       # Fig. 1 d
    (8, 1, 2, 1, 2),        # time shear with s1 != 0
    (8, 1, 2, 1, 4),        # time shear, coset p = 2
    (12, 2, 6, 1, 2),       # frequency shear, coset p = 2
    (72, 2, 4, 1, 6),       # both shears (s0 = 14, s1 = 1)
    (96, 4, 8, 1, 3),       # time shear s1 = 95, coset p = 3
    (120, 4, 10, 1, 2),     # frequency shear, coset p = 4
    (144, 4, 12, 3, 4),
    (240, 4, 12, 1, 4),
    (288, 6, 18, 1, 2),
]


@pytest.mark.parametrize("params", SMALL)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_small_lattices_every_route(params, prec):
    Plan = _P()
    L, a, M, l1, l2 = params
    rng = np.random.default_rng(L * 7 + M)
    B = 3
    g = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    fc = rng.standard_normal((B, L)) + 1j * rng.standard_normal((B, L))
    fr = rng.standard_normal((B, L))
    for route in ("coset", "shear"):
        p = Plan(L, a, M, l1, l2, _round(g, prec), route=route, precision=prec)
        for f in (fc, fr):
            c = p.dgt(_to_dev(_round(f, prec), prec)).cpu().numpy()
            for b in range(B):
                ref = _ref_dgt(_round(f[b], prec), _round(g, prec), a, M, l1, l2).T
                assert _rel(c[b], ref) <= TOL[prec], (route, b, _rel(c[b], ref), p.info)
        # synthesis with the analysis window (adjoint) against the oracle's adjoint
        cc = rng.standard_normal((B, L // a, M)) + 1j * rng.standard_normal((B, L // a, M))
        fs = p.idgt(_to_dev(_round(cc, prec), prec), window="adjoint").cpu().numpy()
        for b in range(B):
            ref = OD.idgt_fold(_round(cc[b], prec).T, _round(g, prec), a, M, l1, l2)
            assert _rel(fs[b], ref) <= TOL[prec], (route, "synthesis", b)
        p.close()


# -------------------------------------------------------------------------------------
# quincunx FP64 workload (L = 1440): coefficients, canonical dual, reconstruction
# -------------------------------------------------------------------------------------
@pytest.mark.parametrize("route", ["coset", "shear", "auto"])
def test_quincunx_fp64_full(route):
    Plan = _P()
    L, a, M, l1, l2 = 1440, 16, 48, 1, 2
    g = gaussian_window(L)
    f = complex_normal(L, 0, 0)
    p = Plan(L, a, M, l1, l2, g, route=route, precision="f64")
    c = p.dgt(_to_dev(f, "f64"))
    ref = OD.dgt_direct(f, g, a, M, l1, l2).T
    assert _rel(c.cpu().numpy(), ref) <= 1e-12
    gd = OU.zak_gram_dual(g, a, M, l1, l2)
    assert _rel(p.dual_window().cpu().numpy(), gd) <= 1e-12
    gt = OU.zak_gram_tight(g, a, M, l1, l2)
    assert _rel(p.tight_window().cpu().numpy(), gt) <= 1e-12
    fr = p.idgt(c, window="dual").cpu().numpy()
    assert _rel(fr, f) <= 1e-12


# -------------------------------------------------------------------------------------
# dual / tight windows on small frames, Parseval for the tight window
# -------------------------------------------------------------------------------------
@pytest.mark.parametrize("params", [(36, 3, 6, 1, 2), (96, 4, 8, 1, 3), (120, 4, 10, 1, 2), (144, 4, 12, 3, 4),
                                    (240, 4, 12, 1, 4), (288, 6, 18, 1, 2)])
@pytest.mark.parametrize("route", ["coset", "shear"])
def test_dual_tight_small(params, route):
    Plan = _P()
    L, a, M, l1, l2 = params
    g = gaussian_window(L)
    p = Plan(L, a, M, l1, l2, g, route=route, precision="f64")
    gd = OU.dense_dual(g, a, M, l1, l2)
    gt = OU.dense_tight(g, a, M, l1, l2)
    assert _rel(p.dual_window().cpu().numpy(), gd) <= 1e-12
    assert _rel(p.tight_window().cpu().numpy(), gt) <= 1e-12
    f = complex_normal(L, 5, L)
    pt = Plan(L, a, M, l1, l2, gt, route=route, precision="f64")
    ct = pt.dgt(_to_dev(f, "f64"))
    assert abs(np.linalg.norm(ct.cpu().numpy()) ** 2 / np.linalg.norm(f) ** 2 - 1) <= 1e-12
    assert _rel(p.idgt(p.dgt(_to_dev(f, "f64")), window="dual").cpu().numpy(), f) <= 1e-12
    assert _rel(p.idgt(p.dgt(_to_dev(f, "f64")), window="tight").cpu().numpy(),
                OD.idgt_fold(OD.dgt_fold(f, g, a, M, l1, l2), gt, a, M, l1, l2)) <= 1e-12


# -------------------------------------------------------------------------------------
# FIR route (weighted overlap-add) with a Hann window
# -------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("params", [(16384, 128, 1024, 1, 2, 1024), (4096, 16, 128, 1, 2, 128),
                                    (4096, 32, 256, 1, 4, 256), (8192, 32, 256, 1, 4, 128),
                                    (4096, 16, 256, 1, 2, 96), (1728, 12, 144, 1, 3, 96)])
def test_fir_route(params, prec):
    Plan = _P()
    L, a, M, l1, l2, Lg = params
    taps, center = hann_taps(Lg)
    taps = taps / np.linalg.norm(taps)
    gfull = np.zeros(L)
    gfull[(np.arange(Lg) - center) % L] = taps
    p = Plan(L, a, M, l1, l2, _round(taps, prec), route="fir", precision=prec, fir_center=center)
    assert p.route == "fir"
    B = 2
    f = np.stack([real_normal(L, 9, i) for i in range(B)])
    c = p.dgt(_to_dev(_round(f, prec), prec)).cpu().numpy()
    for b in range(B):
        ref = OD.dgt_fold(_round(f[b], prec), _round(gfull, prec), a, M, l1, l2).T
        assert _rel(c[b], ref) <= TOL[prec]
    # synthesis: adjoint and perfect reconstruction with the (FIR) canonical dual
    gd = OU.fir_dual_diag(_round(gfull, prec), a, M)
    assert _rel(p.dual_window().cpu().numpy(), gd) <= TOL[prec]
    fr = p.idgt(_to_dev(c, prec), window="dual", real=True).cpu().numpy()
    for b in range(B):
        assert _rel(fr[b], _round(f[b], prec)) <= 5 * TOL[prec]
    cc = _round(OD.dgt_fold(_round(f[0], prec), _round(gfull, prec), a, M, l1, l2), prec)   # the oracle's [m, n]
    fa = p.idgt(_to_dev(np.ascontiguousarray(cc.T), prec), window="adjoint").cpu().numpy()
    assert _rel(fa, OD.idgt_fold(cc, _round(gfull, prec), a, M, l1, l2)) <= TOL[prec]


# -------------------------------------------------------------------------------------
# gradients (learnable-window workload, 2048-long sub-case)
# -------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gradients_subcase(prec):
    from paper_1307_4569_gb300 import dgt as dgt_fn

    Plan = _P()
    L, a, M, l1, l2 = 2048, 16, 128, 1, 2
    B = 3
    rng = np.random.default_rng(21)
    f = rng.standard_normal((B, L))
    from workloads import noisy_gaussian_window

    g = noisy_gaussian_window(L, 3)
    p = Plan(L, a, M, l1, l2, _round(g, prec), route="auto", precision=prec)
    ft = _to_dev(_round(f, prec), prec).requires_grad_(True)
    gt = _to_dev(_round(g, prec), prec).requires_grad_(True)
    c = dgt_fn(ft, gt, p)
    loss = torch.log(c.real ** 2 + c.imag ** 2 + 1e-6).sum()
    loss.backward()
    ref_l, ref_gf, ref_gg = 0.0, np.zeros((B, L)), np.zeros(L)
    for b in range(B):
        lv, gf, gg = OG.grads(_round(f[b], prec), _round(g, prec), a, M, l1, l2)
        ref_l += lv
        ref_gf[b] = gf
        ref_gg += gg
    # float32: log(|c|^2 + eps) is stiff where |c|^2 ~ eps, so an error of the forward
    # transform's size (2e-6 relative) is amplified in u = c / (|c|^2 + eps).  The tolerance is
    # the oracle's own response to such an error (seeded random perturbations of c of relative
    # size 2e-6), times 3; the backward kernels alone are held to the transform's bound in
    # test_backward_kernels_on_oracle_gradient.
    tol = 1e-10 if prec == "f64" else 3 * _gradient_response(_round(f, prec), _round(g, prec), a, M, l1, l2, 2e-6)
    assert abs(loss.item() - ref_l) <= (1e-10 if prec == "f64" else 1e-4) * abs(ref_l)
    assert _rel(ft.grad.cpu().numpy(), ref_gf) <= tol
    assert _rel(gt.grad.cpu().numpy(), ref_gg) <= tol
    # library loss helper agrees
    lv, G = p.logmag_loss(c.detach())
    assert abs(lv.sum().item() - ref_l) <= (1e-10 if prec == "f64" else 1e-4) * abs(ref_l)
    # the fused loss as an autograd function: same value and gradients
    from paper_1307_4569_gb300 import log_magnitude_loss

    ft2 = _to_dev(_round(f, prec), prec).requires_grad_(True)
    gt2 = _to_dev(_round(g, prec), prec).requires_grad_(True)
    loss2 = log_magnitude_loss(dgt_fn(ft2, gt2, p), p)
    loss2.backward()
    assert abs(loss2.item() - ref_l) <= (1e-10 if prec == "f64" else 1e-4) * abs(ref_l)
    assert _rel(ft2.grad.cpu().numpy(), ref_gf) <= tol
    assert _rel(gt2.grad.cpu().numpy(), ref_gg) <= tol


def _gradient_response(f, g, a, M, l1, l2, rel, trials=2):
    """Largest relative change of the oracle's signal and window gradients when c = C_g f
    is replaced by c + e, ||e|| = rel ||c|| (seeded complex normal e), over the signals."""
    worst = 0.0
    for b in range(f.shape[0]):
        _, gf, gg = OG.grads(f[b], g, a, M, l1, l2)
        c = OD.dgt_fold(f[b], g, a, M, l1, l2)
        for t in range(trials):
            r = np.random.default_rng((61, b, t))
            e = r.standard_normal(c.shape) + 1j * r.standard_normal(c.shape)
            e *= rel * np.linalg.norm(c) / np.linalg.norm(e)
            _, gf2, gg2 = OG.grads(f[b], g, a, M, l1, l2, coefs=c + e)
            worst = max(worst, _rel(gf2, gf), _rel(gg2, gg))
    return worst


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_backward_kernels_on_oracle_gradient(prec):
    """The backward entry points fed the oracle's coefficient gradient G = 2c/(|c|^2+eps):
    the signal gradient (synthesis with the analysis window, real part) within the transform's
    bound, the window gradient within that bound times the cancellation of its sum over n and
    the batch (sum of the terms' magnitudes over the magnitude of the sum, from the oracle)."""
    Plan = _P()
    L, a, M, l1, l2 = 2048, 16, 128, 1, 2
    B = 3
    f = _round(np.random.default_rng(21).standard_normal((B, L)), prec)
    from workloads import noisy_gaussian_window

    g = _round(noisy_gaussian_window(L, 3), prec)
    lat = OL.Lattice(L, a, M, l1, l2)
    G = np.empty((B, L // a, M), dtype=np.complex128)
    ref_gf, ref_gg = np.zeros((B, L)), np.zeros(L)
    terms = np.zeros(L)
    l = np.arange(L)
    for b in range(B):
        _, gf, gg = OG.grads(f[b], g, a, M, l1, l2)
        c = OD.dgt_fold(f[b], g, a, M, l1, l2)
        u = c / (np.abs(c) ** 2 + 1e-6)
        G[b] = _round(2 * u, prec).T
        ref_gf[b] = gf
        ref_gg += gg
        for n in range(lat.N):
            Un = np.tile(np.fft.ifft(u[:, n]) * M, L // M) * np.exp(
                2j * np.pi * ((l * lat.freq_offset_num(n)) % (l2 * M)) / (l2 * M))
            terms += np.abs(2 * np.roll(f[b] * np.conj(Un), -a * n).real)
    cancel = float(np.linalg.norm(terms) / np.linalg.norm(ref_gg))
    p = Plan(L, a, M, l1, l2, g, route="auto", precision=prec)
    Gd = _to_dev(G, prec)
    gf_dev = p.idgt(Gd, window="adjoint", real=True).cpu().numpy()
    gg_dev = p.grad_window(_to_dev(f, prec), Gd, real=True).cpu().numpy()
    p.status()
    assert _rel(gf_dev, ref_gf) <= TOL[prec]
    assert _rel(gg_dev, ref_gg) <= TOL[prec] * max(1.0, cancel), cancel
    p.close()


# -------------------------------------------------------------------------------------
# errors and edge cases
# -------------------------------------------------------------------------------------
def test_errors_and_edges():
    from paper_1307_4569_gb300 import DGTError

    Plan = _P()
    g = gaussian_window(1440)
    assert not OL.feasible(1440, 16, 48, 1, 7)
    with pytest.raises(DGTError) as e:
        Plan(1440, 16, 48, 1, 7, g)                      # 7 * lcm(16, 48) = 336 does not divide 1440
    assert e.value.status == 2
    with pytest.raises(DGTError) as e:
        Plan(16384, 16, 128, 1, 3, gaussian_window(16384))   # lambda2 = 3 never fits a power of two
    assert e.value.status == 2
    with pytest.raises(DGTError) as e:
        Plan(1440, 16, 48, 2, 2, g)
    assert e.value.status == 1
    p = Plan(1440, 16, 48, 1, 2, g, precision="f64")
    empty = torch.empty((0, 1440), dtype=torch.complex128, device="cuda")
    out = p.dgt(empty)
    assert out.shape == (0, 90, 48)
    # workspace variant equals the allocating one
    f = _to_dev(complex_normal(1440, 1, 1)[None, :].repeat(2, 0), "f64")
    ws = torch.empty(p.workspace_bytes(2) // 8 + 64, dtype=torch.float64, device="cuda")
    c1 = p.dgt(f)
    c2 = torch.empty_like(c1)
    p.dgt_ws(f, c2, ws)
    assert torch.equal(c1, c2)


# -------------------------------------------------------------------------------------
# degenerate lattices: one channel, one sample per time step, critical sampling, a = M,
# a single column per coset, and the empty batch on every entry point
# -------------------------------------------------------------------------------------
DEGENERATE = [
    (16, 2, 1, 0, 1),       # M = 1: one frequency channel
    (64, 1, 4, 1, 2),       # a = 1: every time shift
    (96, 8, 8, 1, 2),       # a = M: critical sampling (redundancy 1)
    (64, 4, 64, 0, 1),      # M = L: one time-frequency tile per time step, b = 1
    (72, 6, 12, 1, 3),      # N = 12 columns, lambda2 = 3: four columns per coset
]


@pytest.mark.parametrize("params", DEGENERATE)
def test_degenerate_lattices(params):
    Plan = _P()
    L, a, M, l1, l2 = params
    assert OL.feasible(L, a, M, l1, l2)
    rng = np.random.default_rng(L + 13 * M + a)
    g = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    f = rng.standard_normal((2, L)) + 1j * rng.standard_normal((2, L))
    for route in ("coset", "shear"):
        p = Plan(L, a, M, l1, l2, g, route=route, precision="f64")
        c = p.dgt(_to_dev(f, "f64")).cpu().numpy()
        for b in range(2):
            ref = OD.dgt_direct(f[b], g, a, M, l1, l2).T
            assert _rel(c[b], ref) <= 1e-12, (route, b, p.info)
        cc = rng.standard_normal((2, L // a, M)) + 1j * rng.standard_normal((2, L // a, M))
        fs = p.idgt(_to_dev(cc, "f64"), window="adjoint").cpu().numpy()
        for b in range(2):
            assert _rel(fs[b], OD.idgt_direct(cc[b].T, g, a, M, l1, l2)) <= 1e-12, (route, "synthesis")
        # empty batches on every entry point
        e = torch.empty((0, L), dtype=torch.complex128, device="cuda")
        assert p.dgt(e).shape == (0, L // a, M)
        ec = torch.empty((0, L // a, M), dtype=torch.complex128, device="cuda")
        assert p.idgt(ec, window="adjoint").shape == (0, L)
        p.close()
