"""Synthesis with a window of the caller's choosing (idgt_exec_window, through the C ABI):
f(l) = sum c(m, n) gamma(l - a n) exp(+2 pi i l (m + w(n)) / M) (Section 2.1) for a seeded
random gamma, against the oracle's fold-form synthesis with the same gamma, on seeded
coefficients.  Coset and shear routes (both shear branches) on power-of-two and mixed-radix
lattices, and the FIR route with random taps; float32 (2e-6) and float64 (1e-12)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from workloads import gaussian_window, hann_taps  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


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


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("lat", [(4096, 32, 256, 1, 2), (2160, 30, 60, 1, 3), (4096, 64, 128, 1, 4)])
@pytest.mark.parametrize("route", ["coset", "shear"])
def test_user_window_full_length(prec, lat, route):
    from paper_1307_4569_gb300 import Plan

    L, a, M, l1, l2 = lat
    N = L // a
    r = np.random.default_rng((77, L, l2))
    B = 2
    c = _round(r.standard_normal((B, N, M)) + 1j * r.standard_normal((B, N, M)), prec)
    gam = _round(r.standard_normal(L) + 1j * r.standard_normal(L), prec)
    p = Plan(L, a, M, l1, l2, gaussian_window(L), route=route, precision=prec)
    cd = _dev(c, prec)
    for real_out in (False, True):
        out = p.idgt_window(cd, _dev(gam, prec), real=real_out).cpu().numpy()
        for b in range(B):
            ref = OD.idgt_fold(c[b].T, gam, a, M, l1, l2)
            assert _rel(out[b], ref.real if real_out else ref) <= TOL[prec], (route, lat, real_out, b)
    # a real window, and the plan's own windows afterwards are untouched
    gr = _round(r.standard_normal(L), prec)
    out = p.idgt_window(cd, _dev(gr, prec)).cpu().numpy()
    assert _rel(out[0], OD.idgt_fold(c[0].T, gr, a, M, l1, l2)) <= TOL[prec]
    adj = p.idgt(cd, window="adjoint").cpu().numpy()
    assert _rel(adj[0], OD.idgt_fold(c[0].T, _round(gaussian_window(L), prec), a, M, l1, l2)) <= TOL[prec]
    p.status()
    p.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("lat", [(16384, 64, 512, 1, 2), (14400, 20, 120, 1, 3)])
def test_user_window_fir_taps(prec, lat):
    from paper_1307_4569_gb300 import Plan

    L, a, M, l1, l2 = lat
    N = L // a
    Lg = M
    taps, center = hann_taps(Lg)
    r = np.random.default_rng((78, L))
    B = 2
    c = _round(r.standard_normal((B, N, M)) + 1j * r.standard_normal((B, N, M)), prec)
    ut = _round(r.standard_normal(Lg) + 1j * r.standard_normal(Lg), prec)
    full = np.zeros(L, dtype=np.complex128)
    for t in range(Lg):
        full[(t - center) % L] = ut[t]
    p = Plan(L, a, M, l1, l2, taps / np.linalg.norm(taps), route="fir", precision=prec, fir_center=center)
    out = p.idgt_window(_dev(c, prec), _dev(ut, prec)).cpu().numpy()
    for b in range(B):
        assert _rel(out[b], OD.idgt_fold(c[b].T, full, a, M, l1, l2)) <= TOL[prec], (lat, b)
    p.status()
    p.close()
