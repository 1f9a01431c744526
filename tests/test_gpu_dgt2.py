"""Two-dimensional tensor-product DGT on the GPU against the oracle (per-dimension algorithm,
itself pinned to the two-dimensional definition): coefficients, the adjoint, and
reconstruction with the tensor product of the axes' canonical duals."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt2 as O2  # noqa: E402
from oracle import duals as OU  # noqa: E402
from workloads import gaussian_window  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _r(x, prec):
    return x if prec == "f64" else x.astype(np.complex64).astype(np.complex128)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    ((64, 4, 8, 1, 2), (108, 6, 12, 1, 3)),
    ((144, 6, 12, 0, 1), (128, 8, 16, 1, 2)),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("route", ["coset", "shear"])
@pytest.mark.parametrize("case", CASES)
def test_dgt2(case, route, prec):
    from paper_1307_4569_gb300 import Plan2

    lat1, lat2 = case
    L1, L2 = lat1[0], lat2[0]
    g1, g2 = gaussian_window(L1), gaussian_window(L2)
    rng = np.random.default_rng(L1 * 3 + L2)
    B = 2
    f = rng.standard_normal((B, L1, L2)) + 1j * rng.standard_normal((B, L1, L2))
    fr = _r(f, prec)
    p = Plan2(lat1, _r(g1, prec).real, lat2, _r(g2, prec).real, route=route, precision=prec)
    dt = torch.complex128 if prec == "f64" else torch.complex64
    c = p.dgt(torch.from_numpy(fr.astype(np.complex128 if prec == "f64" else np.complex64)).cuda())
    assert c.shape == (B, L1 // lat1[1], lat1[2], L2 // lat2[1], lat2[2])
    cn = c.cpu().numpy()
    for b in range(B):
        ref = O2.dgt2(fr[b], _r(g1, prec).real, _r(g2, prec).real, lat1[1:], lat2[1:])   # [m1, n1, m2, n2]
        assert _rel(cn[b].transpose(1, 0, 3, 2), ref) <= TOL[prec], (b, _rel(cn[b].transpose(1, 0, 3, 2), ref))
    # adjoint of the oracle's own coefficients against the oracle's adjoint
    u = _r(O2.dgt2(fr[0], _r(g1, prec).real, _r(g2, prec).real, lat1[1:], lat2[1:]), prec)   # [m1, n1, m2, n2]
    ud = torch.from_numpy(np.ascontiguousarray(u.transpose(1, 0, 3, 2))[None]).to(dt).cuda()
    fa = p.idgt(ud, window="adjoint").cpu().numpy()[0]
    assert _rel(fa, O2.idgt2(u, _r(g1, prec).real, _r(g2, prec).real, lat1[1:], lat2[1:])) <= TOL[prec]
    # reconstruction with the tensor product of the duals
    rec = p.idgt(c, window="dual").cpu().numpy()
    for b in range(B):
        assert _rel(rec[b], fr[b]) <= 5 * TOL[prec]
    p.status()
    p.close()
