"""Bounded device waits: the float synthesis kernel that stages its column tiles with the
tensor memory accelerator waits for its own copies with a cycle limit.  With the limit set
to zero through the C ABI's test hook every wait expires at once: the kernel must let its
copies land and return, dgt_plan_status must report DGT_ERR_TIMEOUT (once), and the context
must stay usable: the next synthesis, with the limit restored, is bit-identical to one taken
before.  No fault, trap or hang is involved."""
import ctypes

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


def _seeded_coefs(L, a, M, B):
    N = L // a
    r = np.random.default_rng(515)
    return (r.standard_normal((B, N, M)) + 1j * r.standard_normal((B, N, M))).astype(np.complex64)


@pytest.mark.parametrize("route", ["coset", "shear"])
def test_expired_waits_report_timeout_and_leave_the_context_usable(route):
    from paper_1307_4569_gb300 import DGTError, Plan
    from paper_1307_4569_gb300 import _capi as K

    # d = L / M = 1024: the adjoint's column transforms take the tile-staged kernel
    L, a, M, l1, l2 = 1 << 18, 64, 256, 1, 2
    g = gaussian_window(L)
    p = Plan(L, a, M, l1, l2, g, route=route, precision="f32")
    assert p.info["d"] == 1024
    uh = _seeded_coefs(L, a, M, 2)
    c = torch.from_numpy(uh).cuda()
    ref = p.idgt(c, window="adjoint")
    torch.cuda.synchronize()
    p.status()
    # the adjoint against the oracle (the staged kernel is the one that ran)
    g32 = g.astype(np.float32).astype(np.float64)
    want = OD.idgt_coset(uh[0].astype(np.complex128).T, g32, a, M, l1, l2)
    got = ref[0].cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 2e-6
    stream = torch.cuda.current_stream().cuda_stream
    old = K.lib().dgt_wait_limit(0)
    try:
        p.idgt(c, window="adjoint")
        st = K.lib().dgt_plan_status(p._h, ctypes.c_void_p(stream))
    finally:
        assert K.lib().dgt_wait_limit(old) == 0
    assert st == K.DGT_ERR_TIMEOUT
    assert K.lib().dgt_plan_status(p._h, ctypes.c_void_p(stream)) == K.DGT_OK   # reported once
    again = p.idgt(c, window="adjoint")
    torch.cuda.synchronize()
    p.status()
    assert torch.equal(again, ref)

    # without a status call, the plan's next call reports the expiry (and enqueues nothing)
    old = K.lib().dgt_wait_limit(0)
    try:
        p.idgt(c, window="adjoint")
        torch.cuda.synchronize()
    finally:
        K.lib().dgt_wait_limit(old)
    with pytest.raises(DGTError, match="DGT_ERR_TIMEOUT"):
        p.idgt(c, window="adjoint")
    assert torch.equal(p.idgt(c, window="adjoint"), ref)

    # caller workspaces: the expiry lands in the word of the workspace its call used, not in
    # the plan's word or another workspace's
    nb = p.workspace_bytes(2)
    ws1 = torch.empty(nb, dtype=torch.uint8, device="cuda")
    ws2 = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out1, out2 = torch.empty_like(ref), torch.empty_like(ref)
    p.idgt_ws(c, out2, "adjoint", False, ws2)
    old = K.lib().dgt_wait_limit(0)
    try:
        p.idgt_ws(c, out1, "adjoint", False, ws1)
        torch.cuda.synchronize()
    finally:
        K.lib().dgt_wait_limit(old)
    with pytest.raises(DGTError, match="DGT_ERR_TIMEOUT"):
        p.workspace_status(ws1)
    p.workspace_status(ws1)                       # reported once
    p.workspace_status(ws2)
    p.status()
    assert torch.equal(out2, ref)
    p.idgt_ws(c, out1, "adjoint", False, ws1)
    p.workspace_status(ws1)
    assert torch.equal(out1, ref)
    p.close()
