"""Blockwise (overlap-add) plans on the GPU against the oracle.

The blockwise analysis must give the coefficients of the full-length DGT with the same FIR
window (oracle coset route, and the oracle's own blockwise form); its synthesis is the
adjoint (checked against the oracle's blockwise synthesis) and reconstructs with the dual.
Float64 at 1e-12, float32 at 2e-6 relative l2 (float32 against the oracle on the
float32-rounded inputs).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from oracle import duals as OU  # noqa: E402
from oracle import ola as OO  # noqa: E402
from workloads import complex_normal, hann_taps  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _r(x, prec):
    return x if prec == "f64" else x.astype(np.complex64).astype(np.complex128)


def _dev(x, prec):
    return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex128 if prec == "f64" else np.complex64))).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    # L, a, M, lam1, lam2, taps ("hann" or "rand"), Lg, Lb
    (16384, 32, 256, 1, 2, "hann", 256, 2048),
    (32768, 64, 512, 1, 4, "hann", 512, 4096),
    (2304, 16, 48, 1, 3, "rand", 40, 288),
    (8192, 16, 128, 0, 1, "hann", 128, 1024),
]


def _taps(kind, Lg):
    if kind == "hann":
        t, center = hann_taps(Lg)
        return (t / np.linalg.norm(t)).astype(np.complex128), center
    rng = np.random.default_rng(Lg)
    t = rng.standard_normal(Lg) + 1j * rng.standard_normal(Lg)
    return t / np.linalg.norm(t), 5


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("route", ["coset", "shear"])
@pytest.mark.parametrize("case", CASES)
def test_ola_plan(case, route, prec):
    from paper_1307_4569_gb300 import Plan

    L, a, M, l1, l2, kind, Lg, Lb = case
    taps, center = _taps(kind, Lg)
    tr = _r(taps, prec)
    p = Plan(L, a, M, l1, l2, tr, route=route, precision=prec, fir_center=center, block_len=Lb)
    info = p.info
    assert info["ola_block"] == Lb and info["ola_len"] >= Lb + Lg and info["ola_len"] % (l2 * np.lcm(a, M)) == 0
    assert info["route_name"] == route
    Lx = info["ola_len"]
    B = 2
    f = np.stack([complex_normal(L, 31, i) for i in range(B)])
    fr = _r(f, prec)
    c = p.dgt(_dev(fr, prec)).cpu().numpy()
    gfull = OO.local_window(tr, center, L)
    for b in range(B):
        ref = OD.dgt_coset(fr[b], gfull, a, M, l1, l2).T
        assert _rel(c[b], ref) <= TOL[prec], (b, _rel(c[b], ref))
    # the adjoint of the oracle's coefficients against the oracle's blockwise synthesis (same Lx)
    u = _r(OD.dgt_coset(fr[0], gfull, a, M, l1, l2), prec)               # [m, n]
    fa = p.idgt(_dev(np.ascontiguousarray(u.T), prec), window="adjoint").cpu().numpy()
    assert _rel(fa, OO.idgt_ola(u, tr, center, a, M, l1, l2, Lb, Lx)) <= TOL[prec]
    # reconstruction with the dual (windows no longer than M), and the dual itself
    if Lg <= M:
        gd = OU.fir_dual_diag(gfull, a, M)
        assert _rel(p.dual_window().cpu().numpy(), gd) <= TOL[prec]
        rec = p.idgt(_dev(c, prec), window="dual").cpu().numpy()
        for b in range(B):
            assert _rel(rec[b], fr[b]) <= 5 * TOL[prec]
    p.status()
    p.close()


def test_ola_plan_errors():
    from paper_1307_4569_gb300 import DGTError, Plan

    taps, center = hann_taps(256)
    with pytest.raises(DGTError, match="DGT_ERR_LENGTH"):
        Plan(16384, 32, 256, 1, 2, taps, fir_center=center, block_len=3000)          # not admissible
    with pytest.raises(DGTError, match="DGT_ERR_ARG"):
        Plan(16384, 32, 256, 1, 2, taps, fir_center=center, block_len=512, route="fir")
    with pytest.raises(DGTError, match="DGT_ERR_ARG"):
        Plan(16384, 32, 256, 1, 2, np.ones(1024) / 32, fir_center=512, block_len=512)  # block < window
    with pytest.raises(ValueError):
        Plan(16384, 32, 256, 1, 2, np.ones(16384), block_len=2048)                    # not an FIR window
