"""Real-signal coefficients on the GPU against the oracle: the channels 0..M/2 of real
signals with a real window (every route, both precisions), reconstruction from them with the
dual, and the refusal outside lambda2 <= 2 / real windows."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgtreal as OR  # noqa: E402
from oracle import duals as OU  # noqa: E402
from workloads import gaussian_window, hann_taps, real_normal  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _r(x, prec):
    return x if prec == "f64" else x.astype(np.float32).astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("route", ["coset", "shear", "fir"])
@pytest.mark.parametrize("lat", [(16384, 32, 256, 1, 2), (16384, 32, 256, 0, 1), (1440, 16, 48, 1, 2)])
def test_dgtreal(lat, route, prec):
    from paper_1307_4569_gb300 import Plan

    L, a, M, l1, l2 = lat
    B = 2
    f = np.stack([real_normal(L, 41, i) for i in range(B)])
    fr = _r(f, prec)
    if route == "fir":
        taps, center = hann_taps(M)
        taps = taps / np.linalg.norm(taps)
        g = np.zeros(L)
        g[(np.arange(M) - center) % L] = taps
        p = Plan(L, a, M, l1, l2, _r(taps, prec), route="fir", precision=prec, fir_center=center)
    else:
        g = gaussian_window(L)
        p = Plan(L, a, M, l1, l2, _r(g, prec), route=route, precision=prec)
    dt = torch.float64 if prec == "f64" else torch.float32
    fd = torch.from_numpy(fr.astype(np.float64 if prec == "f64" else np.float32)).cuda()
    ch = p.dgtreal(fd)
    assert ch.shape == (B, L // a, M // 2 + 1)
    chn = ch.cpu().numpy()
    for b in range(B):
        ref = OR.dgtreal(fr[b], _r(g, prec), a, M, l1, l2).T
        assert _rel(chn[b], ref) <= TOL[prec], (b, _rel(chn[b], ref))
    rec = p.idgtreal(ch, window="dual")
    assert rec.dtype == dt
    for b in range(B):
        assert _rel(rec[b].cpu().numpy(), fr[b]) <= 5 * TOL[prec]
    # the adjoint from the oracle's half channels equals the oracle's real synthesis with g
    hc = OR.dgtreal(fr[0], _r(g, prec), a, M, l1, l2)                     # [m <= M/2, n]
    if prec == "f32":
        hc = hc.astype(np.complex64).astype(np.complex128)
    cd = torch.complex128 if prec == "f64" else torch.complex64
    hd = torch.from_numpy(np.ascontiguousarray(hc.T)[None]).to(cd).cuda()
    fa = p.idgtreal(hd, window="adjoint").cpu().numpy()
    assert _rel(fa[0], OR.idgtreal(hc, _r(g, prec), a, M, l1, l2)) <= TOL[prec]
    p.close()


def test_dgtreal_refusals():
    from paper_1307_4569_gb300 import DGTError, Plan

    L = 1728
    p = Plan(L, 12, 144, 1, 3, gaussian_window(L), precision="f64")
    f = torch.zeros((1, L), dtype=torch.float64, device="cuda")
    with pytest.raises(DGTError, match="DGT_ERR_UNSUPPORTED"):
        p.dgtreal(f)                                  # lambda2 = 3: no symmetry
    rng = np.random.default_rng(2)
    g = gaussian_window(1440) * np.exp(1j * rng.standard_normal(1440) * 0.1)
    q = Plan(1440, 16, 48, 1, 2, g, precision="f64")
    with pytest.raises(DGTError, match="DGT_ERR_UNSUPPORTED"):
        q.dgtreal(torch.zeros((1, 1440), dtype=torch.float64, device="cuda"))   # complex window
