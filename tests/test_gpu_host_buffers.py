"""Host-buffer entry points (dgt_exec_host / idgt_exec_host): the batch in chunks through
device staging slots with the copies on their own streams.  Results are bit-identical to the
device-buffer calls for every chunking (whole batch, ragged last chunk, chunk of one, chunk
above the batch), for pinned and pageable host memory, on the FIR, coset and shear routes in
both precisions, and equal to the oracle on one case."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from workloads import complex_normal, gaussian_window, hann_taps, real_normal  # noqa: E402

CASES = [
    ("fir", 16384, 128, 1024, 1, 2, "f32"),
    ("coset", 16384, 32, 512, 1, 2, "f32"),
    ("shear", 288, 6, 18, 1, 2, "f64"),
    ("shear", 2880, 60, 240, 1, 2, "f32"),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _plan(route, L, a, M, l1, l2, prec):
    from paper_1307_4569_gb300 import Plan

    if route == "fir":
        taps, center = hann_taps(1024)
        return Plan(L, a, M, l1, l2, taps / np.linalg.norm(taps), route="fir", precision=prec, fir_center=center)
    return Plan(L, a, M, l1, l2, gaussian_window(L), route=route, precision=prec)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_bit_identical(case, pinned):
    route, L, a, M, l1, l2, prec = case
    p = _plan(route, L, a, M, l1, l2, prec)
    B = 5
    real = route == "fir"
    if real:
        f = np.stack([real_normal(L, 81, i) for i in range(B)]).astype(np.float64 if prec == "f64" else np.float32)
    else:
        f = np.stack([complex_normal(L, 81, i) for i in range(B)]).astype(
            np.complex128 if prec == "f64" else np.complex64)
    fh = torch.from_numpy(f)
    if pinned:
        fh = fh.pin_memory()
    c_dev = p.dgt(fh.cuda())
    window = "dual" if route == "fir" else "adjoint"
    s_dev = p.idgt(c_dev, window=window, real=real)
    torch.cuda.synchronize()
    want_c, want_s = c_dev.cpu(), s_dev.cpu()
    for chunk in (0, 2, 1, 7):
        ch = p.dgt_host(fh, chunk=chunk)
        torch.cuda.synchronize()
        assert torch.equal(ch, want_c), (route, chunk)
        sh = p.idgt_host(ch, window=window, real=real, chunk=chunk)
        torch.cuda.synchronize()
        assert torch.equal(sh, want_s), (route, chunk)
    p.status()
    p.close()


def test_host_buffers_against_oracle():
    p = _plan("coset", 16384, 32, 512, 1, 2, "f64")
    L, a, M, N = 16384, 32, 512, 512
    f = np.stack([complex_normal(L, 82, i) for i in range(3)])
    c = p.dgt_host(torch.from_numpy(f).pin_memory(), chunk=2)
    torch.cuda.synchronize()
    g = gaussian_window(L)
    cols = [0, 3, N - 1]
    for b in range(3):
        ref = OD.dgt_fold(f[b], g, a, M, 1, 2, cols=cols)
        assert np.linalg.norm(c[b].numpy()[cols].T - ref) <= 1e-12 * np.linalg.norm(ref)
    p.close()


def test_host_buffers_arguments():
    from paper_1307_4569_gb300 import DGTError, _capi as K

    p = _plan("coset", 16384, 32, 512, 1, 2, "f32")
    x = torch.zeros(16384, dtype=torch.complex64)
    y = torch.zeros(512 * 512, dtype=torch.complex64)
    assert K.lib().dgt_exec_host(p._h, x.data_ptr(), 0, y.data_ptr(), 0, 0, None) == K.DGT_OK
    assert K.lib().dgt_exec_host(p._h, x.data_ptr(), 0, y.data_ptr(), 1, -1, None) == K.DGT_ERR_ARG
    assert K.lib().dgt_exec_host(None, x.data_ptr(), 0, y.data_ptr(), 1, 0, None) == K.DGT_ERR_ARG
    with pytest.raises(TypeError):
        p.dgt_host(x.cuda())
    with pytest.raises(DGTError):
        K.check(K.lib().idgt_exec_host(p._h, y.data_ptr(), x.data_ptr(), 0, -1, 0, 0, None))
    p.close()
