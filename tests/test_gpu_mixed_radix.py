"""The compiled mixed-radix channel transforms (lengths 60 ... 2160 with factors 3 and 5):
analysis by the coset and shear routes and synthesis with the window on lattices whose channel
count M is each such length, against the oracle's coset route (eq. mw_frop, eq. mw_phases) and
its adjoint on the oracle's coefficients; float32 2e-6, float64 1e-12."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from workloads import complex_normal, gaussian_window  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}
LENGTHS = [60, 120, 180, 240, 360, 480, 720, 960, 2160]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _round(x, prec):
    return x if prec == "f64" else x.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("M", LENGTHS)
def test_mixed_radix_channel_lengths(prec, M):
    from paper_1307_4569_gb300 import Plan

    a = M // 4
    l1, l2 = 1, 2
    L = 2 * M * 6                                     # a multiple of lambda2 lcm(a, M)
    g = _round(gaussian_window(L).astype(np.complex128), prec).real
    B = 2
    f = np.stack([_round(complex_normal(L, 41, M, i), prec) for i in range(B)])
    dt = torch.complex128 if prec == "f64" else torch.complex64
    fd = torch.from_numpy(np.ascontiguousarray(f)).to(dt).cuda()
    for route in ("coset", "shear"):
        p = Plan(L, a, M, l1, l2, g, route=route, precision=prec)
        c = p.dgt(fd).cpu().numpy()
        refs = [OD.dgt_coset(f[b], g, a, M, l1, l2) for b in range(B)]
        for b in range(B):
            err = np.linalg.norm(c[b] - refs[b].T) / np.linalg.norm(refs[b])
            assert err <= TOL[prec], (route, M, b, err, p.info)
        # synthesis with the window (the adjoint) of the oracle's coefficients
        cin = np.ascontiguousarray(np.stack([_round(r.T, prec) for r in refs]))
        fr = p.idgt(torch.from_numpy(cin).to(dt).cuda(), window="adjoint").cpu().numpy()
        for b in range(B):
            want = OD.idgt_coset(cin[b].T, g, a, M, l1, l2)
            err = np.linalg.norm(fr[b] - want) / np.linalg.norm(want)
            assert err <= TOL[prec], (route, M, b, err)
        p.status()
        p.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("d", LENGTHS)
def test_mixed_radix_zak_lengths(prec, d):
    """Zak length d = each compiled mixed length (L = 64 d, a = 32, M = 64, lambda = 1/2: the
    separable lattices of both routes have d = gcd(L/M, L/a') = d): the column transforms of
    the Zak transform, the block products and their adjoints."""
    from paper_1307_4569_gb300 import Plan

    L, a, M, l1, l2 = 64 * d, 32, 64, 1, 2
    g = gaussian_window(L)
    B = 2
    f = np.stack([_round(complex_normal(L, 43, d, i), prec) for i in range(B)])
    dt = torch.complex128 if prec == "f64" else torch.complex64
    fd = torch.from_numpy(np.ascontiguousarray(f)).to(dt).cuda()
    gr = _round(g.astype(np.complex128), prec).real
    refs = [OD.dgt_coset(f[b], gr, a, M, l1, l2) for b in range(B)]
    cin = np.ascontiguousarray(np.stack([_round(r.T, prec) for r in refs]))
    for route in ("coset", "shear"):
        p = Plan(L, a, M, l1, l2, gr, route=route, precision=prec)
        assert p.info["d"] == d or route == "shear", p.info
        c = p.dgt(fd).cpu().numpy()
        for b in range(B):
            err = np.linalg.norm(c[b] - refs[b].T) / np.linalg.norm(refs[b])
            assert err <= TOL[prec], (route, d, b, err, p.info)
        fr = p.idgt(torch.from_numpy(cin).to(dt).cuda(), window="adjoint").cpu().numpy()
        for b in range(B):
            want = OD.idgt_coset(cin[b].T, gr, a, M, l1, l2)
            err = np.linalg.norm(fr[b] - want) / np.linalg.norm(want)
            assert err <= TOL[prec], (route, d, b, err)
        p.status()
        p.close()
