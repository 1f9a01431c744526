"""Tile geometry of the tensor-copy-staged float adjoint (Zak routes, d = 1024, p = 1): a
channel count M = 90 leaves a ragged last tile of columns (tiles of 4: the copies read zeros
past M), and separable steps 2a = 6, 10 that are not multiples of the tile width, so the
window-factor tiles are loaded directly while the Y tiles are staged.  (With p = 1 the step
divides M, so a step that is a multiple of 4 implies whole tiles.)  Analysis and adjoint
against the oracle, float32 at 2e-6 relative l2 on the float32-rounded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from workloads import complex_normal, gaussian_window  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _r32(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


@pytest.mark.parametrize("a", [3, 5])
def test_ragged_tiles_and_unaligned_lattice_steps(a):
    from paper_1307_4569_gb300 import Plan

    L, M, l1, l2 = 92160, 90, 1, 2                 # d = L / M = 1024, separable step 2a
    g = gaussian_window(L)
    g32 = _r32(g).real
    p = Plan(L, a, M, l1, l2, g, route="coset", precision="f32")
    assert p.info["d"] == 1024 and p.info["sep_a"] == 2 * a and p.info["p"] == 1
    B = 2
    f = np.stack([_r32(complex_normal(L, 17, i)) for i in range(B)])
    c = p.dgt(torch.from_numpy(f.astype(np.complex64)).cuda())
    u = c.cpu().numpy().astype(np.complex128)
    refs = [OD.dgt_coset(f[b], g32, a, M, l1, l2) for b in range(B)]
    cin = np.ascontiguousarray(np.stack([_r32(r.T) for r in refs]))       # the oracle's coefficients
    back = p.idgt(torch.from_numpy(cin.astype(np.complex64)).cuda(), window="adjoint").cpu().numpy().astype(np.complex128)
    for b in range(B):
        assert _rel(u[b].T, refs[b]) <= 2e-6
        assert _rel(back[b], OD.idgt_coset(cin[b].T, g32, a, M, l1, l2)) <= 2e-6
    p.status()
    p.close()
