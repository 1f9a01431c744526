"""Frequency-shear rows in tiles (fft_post_mr_tile / pre_ifft_mr_tile): lattices where Algorithm
1's output channel depends on the separable row alone (s1 = 0, b a multiple of C6; q rows per
channel, q = 2, 3, 4), analysis against the oracle's direct sum or fold and synthesis against
the oracle's adjoint, float32 2e-6 and float64 1e-12 (profiles/launches_dense_third_shear_f32.md
shows the tile kernels running on the full lambda = 1/3 workload)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from workloads import complex_normal, gaussian_window  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}
CASES = [
    (2160, 12, 36, 1, 3),      # q = 3, Nr = 60
    (10800, 60, 720, 1, 3),    # q = 3, Nr = 60, the lambda = 1/3 lattice at a smaller length
    (1920, 16, 48, 1, 2),      # q = 2, Nr = 60
    (7680, 32, 64, 1, 2),      # q = 2, Nr = 120
    (3840, 16, 48, 1, 4),      # q = 4, Nr = 60
    (7200, 60, 720, 1, 2),     # q = 2, Nr = 60; L = 60 * 120, both length-L factors compiled
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _rnd(x, prec):
    return x if prec == "f64" else x.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("params", CASES)
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_shear_tiles_against_oracle(params, prec):
    from paper_1307_4569_gb300 import Plan

    L, a, M, l1, l2 = params
    N = L // a
    g = _rnd(gaussian_window(L).astype(np.complex128), prec)
    p = Plan(L, a, M, l1, l2, g, route="shear", precision=prec)
    assert p.info["s0"] != 0 and p.info["s1"] == 0, p.info
    B = 2
    f = np.stack([_rnd(complex_normal(L, 91, L, i), prec) for i in range(B)])
    dt = torch.complex128 if prec == "f64" else torch.complex64
    c = p.dgt(torch.from_numpy(np.ascontiguousarray(f)).to(dt).cuda()).cpu().numpy()
    cols = list(range(N)) if L <= 4000 else sorted(set([0, 1, 2, N // 3, N // 2, N - 2, N - 1]))
    for b in range(B):
        ref = OD.dgt_fold(f[b], g, a, M, l1, l2, cols=cols)
        assert np.linalg.norm(c[b][cols].T - ref) <= TOL[prec] * np.linalg.norm(ref), (params, prec, b)
    cc = _rnd(complex_normal(N * M, 92, L).reshape(1, N, M), prec)
    fs = p.idgt(torch.from_numpy(np.ascontiguousarray(cc)).to(dt).cuda(), window="adjoint").cpu().numpy()[0]
    ref = OD.idgt_fold(cc[0].T, g, a, M, l1, l2)
    assert np.linalg.norm(fs - ref) <= TOL[prec] * np.linalg.norm(ref), (params, prec)
    p.status()
    p.close()

