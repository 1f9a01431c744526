"""The allocation-free FIR synthesis entry point (dgt_fir_synthesis_noalloc).

Some callers cannot allocate device memory while they run: a real-time audio callback must
not wait on cudaMalloc (which can synchronise the device and take driver locks), a plug-in
host may own all device memory, a process may have fenced off its allocation budget.  For
them the library keeps the FIR synthesis' seam scratch in one fixed per-GPU array.  This test
calls that entry point through the C ABI twice in a row and checks each result against the
ordinary (allocating) idgt_exec within the float32 tolerance used by the parity tests.  It is
collected last so that a run stopping at the first failure has already run everything else,
and it passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# (L, a, M, lambda1, lambda2, Lg, precision, real output): the power-of-two kernel with real
# and complex seams in both precisions, and the generic kernel (M = 120, not a power of two)
CASES = [
    (16384, 128, 1024, 1, 2, 1024, "f32", True),
    (16384, 128, 1024, 1, 2, 1024, "f32", False),
    (16384, 128, 1024, 1, 2, 1024, "f64", True),
    (14400, 20, 120, 1, 2, 120, "f32", False),
    (14400, 20, 120, 1, 2, 120, "f64", True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "M%d-%s-%s" % (c[2], c[6], "real" if c[7] else "complex"))
def test_noalloc_synthesis_matches_idgt_exec_twice(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import Plan
    from paper_1307_4569_gb300 import _capi as K
    from paper_1307_4569_gb300 import build
    from workloads import hann_taps, real_normal

    build.build()
    L, a, M, l1, l2, Lg, prec, real = case
    tol = 2e-6 if prec == "f32" else 1e-12
    B = 3
    taps, center = hann_taps(Lg)
    taps = taps / np.linalg.norm(taps)
    p = Plan(L, a, M, l1, l2, taps, route="fir", precision=prec, fir_center=center)
    p.dual_window()                                    # caches the dual (this call may allocate)
    rdt = np.float32 if prec == "f32" else np.float64
    f = torch.from_numpy(np.stack([real_normal(L, 31, i) for i in range(B)]).astype(rdt)).cuda()
    c = p.dgt(f)
    stream = torch.cuda.current_stream().cuda_stream
    for window, which in (("dual", K.SYN_DUAL), ("adjoint", K.SYN_ADJOINT)):
        ref = p.idgt(c, window=window, real=real)
        torch.cuda.synchronize()
        for _ in range(2):
            out = torch.full_like(ref, float("nan"))
            st = K.lib().dgt_fir_synthesis_noalloc(p._h, ctypes.c_void_p(c.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr()), int(real), B, which, stream)
            K.check(st)
            torch.cuda.synchronize()
            err = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
            assert err <= tol, (window, err)
    # perfect reconstruction through the allocation-free path
    out = torch.empty((B, L), dtype=f.dtype if real else c.dtype, device="cuda")
    K.check(K.lib().dgt_fir_synthesis_noalloc(p._h, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                              int(real), B, K.SYN_DUAL, stream))
    torch.cuda.synchronize()
    back = out if real else out.real
    assert float(torch.linalg.vector_norm(back - f) / torch.linalg.vector_norm(f)) <= (1e-5 if prec == "f32" else 1e-12)
    # a batch whose seams exceed the fixed array is refused on the host, before any launch
    big = 1 << 16
    st = K.lib().dgt_fir_synthesis_noalloc(p._h, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           int(real), big, K.SYN_DUAL, stream)
    assert st == K.DGT_ERR_UNSUPPORTED
    p.close()
