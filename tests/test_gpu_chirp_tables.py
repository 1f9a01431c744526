"""Chirp tables of the shear route (Algorithm 1's pchirp(L, s1) and, in the frequency-shear
branch, pchirp(L, -s0), kept by the plan as L exact values each): a plan built with them and one
built without (dgt_chirp_table_cap(0), factors computed per sample) give bit-identical analysis
and synthesis, both equal to the oracle, and differ in plan bytes by exactly the tables."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from workloads import complex_normal, gaussian_window  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}
CASES = [
    (8, 1, 2, 1, 2),          # time shear, s1 != 0
    (96, 4, 8, 1, 3),         # time shear, s1 = 95, coset p = 3
    (36, 6, 6, 1, 2),         # frequency shear
    (72, 2, 4, 1, 6),         # both shears (s0 and s1 non-zero)
    (16384, 32, 512, 1, 2),   # power-of-two Zak kernels (chirp in the fused analysis load and zak_inv)
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _rnd(x, prec):
    return x if prec == "f64" else x.astype(np.complex64).astype(np.complex128)


def _tables(info, L):
    s = set()
    if info["s1"] % (2 * L):
        s.add(info["s1"] % (2 * L))
    if info["s0"] and (-info["s0"]) % (2 * L):
        s.add((-info["s0"]) % (2 * L))
    return len(s)


@pytest.mark.parametrize("params", CASES)
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_chirp_tables_bit_identical(params, prec):
    from paper_1307_4569_gb300 import Plan, _capi as K

    L, a, M, l1, l2 = params
    N = L // a
    g = _rnd(gaussian_window(L).astype(np.complex128), prec)
    with_tab = Plan(L, a, M, l1, l2, g, route="shear", precision=prec)
    old = K.lib().dgt_chirp_table_cap(0)
    try:
        without = Plan(L, a, M, l1, l2, g, route="shear", precision=prec)
    finally:
        K.lib().dgt_chirp_table_cap(old)
    assert with_tab.info["s0"] or with_tab.info["s1"], with_tab.info
    ntab = _tables(with_tab.info, L)
    assert ntab >= 1
    csize = 16 if prec == "f64" else 8
    assert with_tab.plan_bytes() - without.plan_bytes() == ntab * L * csize

    B = 2
    f = np.stack([_rnd(complex_normal(L, 71, L, i), prec) for i in range(B)])
    dt = torch.complex128 if prec == "f64" else torch.complex64
    fd = torch.from_numpy(np.ascontiguousarray(f)).to(dt).cuda()
    c1, c0 = with_tab.dgt(fd), without.dgt(fd)
    assert torch.equal(c1, c0)
    cols = sorted(set([0, 1, N // 2, N - 1]))
    c = c1.cpu().numpy()
    for b in range(B):
        ref = OD.dgt_fold(f[b], g, a, M, l1, l2, cols=cols)
        assert np.linalg.norm(c[b][cols].T - ref) <= TOL[prec] * np.linalg.norm(ref)
    cc = _rnd(complex_normal(N * M, 72, L).reshape(1, N, M), prec)
    cd = torch.from_numpy(np.ascontiguousarray(cc)).to(dt).cuda()
    s1, s0 = with_tab.idgt(cd, window="adjoint"), without.idgt(cd, window="adjoint")
    assert torch.equal(s1, s0)
    ref = OD.idgt_fold(cc[0].T, g, a, M, l1, l2)
    assert np.linalg.norm(s1.cpu().numpy()[0] - ref) <= TOL[prec] * np.linalg.norm(ref)
    with_tab.close()
    without.close()
