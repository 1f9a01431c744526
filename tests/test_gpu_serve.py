"""Serving loop on the GPU: a mixed request stream through the scheduler and the library.

Checks that (1) every admissible request is served and every inadmissible one fails with
DGT_ERR_LENGTH, (2) a request served inside a batch, while other batches run concurrently on
other streams, gets exactly the coefficients (signal) it gets alone, bit for bit, and (3)
served results agree with the oracle
(float32 against the float64 oracle on the float32-rounded inputs, 2e-6 relative l2).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from oracle import duals as OU  # noqa: E402
from workloads import Request, gaussian_window, hann_window  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _stream():
    """Bursts of requests over two lengths, both a, lambda2 in {1, 2, 4}, both windows and
    both operations, plus inadmissible lambda2 = 3 requests."""
    rng = np.random.default_rng(11)
    reqs = []
    t = 0.0
    for burst in range(6):
        t += 0.02
        # four request kinds per burst, so that equal kinds arriving together form batches
        kinds = []
        for _ in range(4):
            L = int(rng.choice((16384, 65536)))
            a = L // int(rng.choice((1024, 512)))
            M = 8 * a
            lam2 = int(rng.choice((1, 2, 4)))
            lam1 = 0 if lam2 == 1 else 1
            win = "gauss" if rng.random() < 0.5 else "hann%d" % M
            kind = "dgt" if rng.random() < 0.6 else "idgt"
            kinds.append((L, a, M, lam1, lam2, win, kind))
        for _ in range(12):
            L, a, M, lam1, lam2, win, kind = kinds[int(rng.integers(4))]
            reqs.append(Request(t, L, a, M, lam1, lam2, win, kind, True, 0))
        if burst % 3 == 2:
            reqs.append(Request(t, 16384, 16, 128, 1, 3, "gauss", "dgt", False, 0))
    return reqs


def test_serve_mixed_equals_alone_and_oracle():
    from paper_1307_4569_gb300.serve import GpuExecutor, Scheduler, request_key

    reqs = _stream()
    ex = GpuExecutor("f32", keep_results=True, streams=3, arena_bytes=1 << 30)
    st = Scheduler(ex, cap_bytes=8 << 30, max_batch=8, max_inflight=3).run(reqs)
    s = st.summary()
    assert s["errors"] == sum(not r.feasible for r in reqs)
    for i, r in enumerate(reqs):
        sv = st.served[i]
        if not r.feasible:
            assert sv.status == "error" and "DGT_ERR_LENGTH" in sv.error
        else:
            assert sv.status == "ok", sv.error
    assert max(st.batch_sizes) > 1, "the bursts must form batches"

    # alone: the same request as a batch of one through the same plan
    checked_oracle = 0
    for i, r in enumerate(reqs):
        if not r.feasible:
            continue
        key = request_key(r)
        p = ex.plans[key]
        x = ex._input(key, r.kind, i).cuda()
        if r.kind == "dgt":
            alone = p.dgt(x[None])[0].cpu()
        else:
            alone = p.idgt(x[None].contiguous(), window="dual")[0].cpu()
        got = ex.results[i]
        assert torch.equal(got, alone), (i, r)
        # oracle on a few requests of the short length
        if r.L == 16384 and checked_oracle < 4:
            g = gaussian_window(r.L) if r.window == "gauss" else hann_window(r.L, r.M)
            g32 = g.astype(np.float32).astype(np.float64)
            xn = x.cpu().numpy().astype(np.complex128)
            if r.kind == "dgt":
                ref = OD.dgt_coset(xn, g32, r.a, r.M, r.lam1, r.lam2).T
            else:
                gam = OU.zak_gram_dual(g32, r.a, r.M, r.lam1, r.lam2)
                ref = OD.idgt_coset(xn.T, gam, r.a, r.M, r.lam1, r.lam2)
            gn = got.numpy().astype(np.complex128)
            err = np.linalg.norm(gn - ref) / np.linalg.norm(ref)
            assert err <= 2e-6, (i, r, err)
            checked_oracle += 1
    assert checked_oracle >= 2
    ex.close()


def test_expired_wait_marks_only_its_batch():
    """A synthesis batch whose tile-copy waits expire (the wait limit set to zero through the
    test hook; no fault involved) is reported by its own workspace word when the executor
    finishes it: finish() raises DGT_ERR_TIMEOUT for that batch, and the next batch of the same
    plan on the same stream arena finishes cleanly with the correct result."""
    from paper_1307_4569_gb300 import DGTError
    from paper_1307_4569_gb300 import _capi as K
    from paper_1307_4569_gb300.serve import GpuExecutor

    # d = L / M = 1024 for a = 64, M = 256: the float synthesis stages its tiles with the TMA
    key = (1 << 18, 64, 256, 1, 2, "gauss")
    ex = GpuExecutor("f32", streams=2, arena_bytes=1 << 30, keep_results=True)
    ex.prepare(key)
    assert ex.plans[key].info["d"] == 1024
    old = K.lib().dgt_wait_limit(0)
    try:
        h = ex.launch(key, "idgt", [None] * 2, [0, 1])
        with pytest.raises(DGTError, match="DGT_ERR_TIMEOUT"):
            ex.finish(h)
    finally:
        K.lib().dgt_wait_limit(old)
    h = ex.launch(key, "idgt", [None] * 2, [2, 3])
    ex.finish(h)
    # the clean batch against the oracle's synthesis of the same inputs
    L, a, M, l1, l2, _ = key
    gd = OU.zak_gram_dual(gaussian_window(L), a, M, l1, l2)       # the plan's dual comes from the float64 window
    for rid in (2, 3):
        cin = ex._input(key, "idgt", rid).numpy().astype(np.complex128)
        want = OD.idgt_fold(cin.T, gd, a, M, l1, l2)
        got = ex.results[rid].numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 2e-6
    ex.close()
