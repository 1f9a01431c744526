"""Element-wise synthesis parity at the audio batch's full size, in the launch configuration
the benchmark times: 64 signals, L = 2^20, a = 128, M = 1024, lambda = 1/2, the Hann FIR plan
and the Gaussian shear and coset plans, float32 and float64, real and complex output.

The coefficient arrays are zero except on a few sampled columns n (first, second, the middle
pair, last), so the oracle's synthesis (Section 2.1, inversion formula, in the fold form
restricted to those columns) costs O(L) per column at full length.  Every output sample of
the sampled signals is compared with it.  The kernels reached are the ones the benchmark
times: pre_ifft_p2<float, 1024> (real and complex output), fft_prod_adj_tma_p2<1024> (TMA
tiles, M = 1024 column tiles), zak_inv_p2 with the time-shear chirp, and
fir_synthesis_p2<float, 1024> with its seams, at 64 signals; and their float64 forms.
Tolerances: float32 2e-6, float64 1e-12 relative l2 per signal (float32 against the oracle on
the float32-rounded window)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from oracle import duals as OU  # noqa: E402
from workloads import AUDIO_BATCH, gaussian_window, hann_taps, hann_window  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}
COLS = [0, 1, 4095, 4096, 8191]
SIGNALS = [0, 31, 63]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_4569_gb300 import build

    build.build()


def _round(x, prec):
    if prec == "f64":
        return x
    return x.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(x) else x.astype(np.float32).astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _sparse_coefs(w, B, prec):
    """[B][N][M] on the device, zero outside COLS; values seeded per signal.  Returns the
    host values of the sampled columns too, shape (B, M, len(COLS))."""
    rng = np.random.default_rng(20240)
    vals = (rng.standard_normal((B, w.M, len(COLS))) + 1j * rng.standard_normal((B, w.M, len(COLS))))
    vals = _round(vals, prec)
    cd = torch.complex128 if prec == "f64" else torch.complex64
    c = torch.zeros((B, w.N, w.M), dtype=cd, device="cuda")
    vt = torch.from_numpy(np.ascontiguousarray(vals.transpose(0, 2, 1))).to(cd).cuda()   # (B, cols, M)
    c[:, COLS, :] = vt
    return c, vals


def _windows(w, prec):
    g = _round(gaussian_window(w.L), prec)
    taps, center = hann_taps(1024)
    taps = _round(taps / np.linalg.norm(taps), prec)
    gh = np.zeros(w.L)
    for t in range(len(taps)):
        gh[(t - center) % w.L] = taps[t]
    return g, taps, center, gh


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_audio_batch_synthesis_sampled_columns(prec):
    from paper_1307_4569_gb300 import Plan

    w = AUDIO_BATCH
    B = w.batch
    c, vals = _sparse_coefs(w, B, prec)
    g, taps, center, gh = _windows(w, prec)
    assert np.array_equal(gh, _round(hann_window(w.L, 1024), prec))      # the FIR plan's window at full length
    duals = {"gauss": OU.zak_gram_dual(g, w.a, w.M, w.lam1, w.lam2), "hann": OU.fir_dual_diag(gh, w.a, w.M)}
    plans = [
        ("hann-fir", "hann", lambda: Plan(w.L, w.a, w.M, w.lam1, w.lam2, taps, route="fir", precision=prec,
                                          fir_center=center)),
        ("gauss-shear", "gauss", lambda: Plan(w.L, w.a, w.M, w.lam1, w.lam2, g, route="shear", precision=prec)),
        ("gauss-coset", "gauss", lambda: Plan(w.L, w.a, w.M, w.lam1, w.lam2, g, route="coset", precision=prec)),
    ]
    for name, wkey, make in plans:
        p = make()
        for window, real in (("dual", True), ("dual", False), ("adjoint", False)):
            out = p.idgt(c, window=window, real=real)
            p.status()
            gam = duals[wkey] if window == "dual" else (gh if wkey == "hann" else g)
            for b in SIGNALS:
                ref = OD.idgt_fold(vals[b], gam, w.a, w.M, w.lam1, w.lam2, cols=COLS)
                got = out[b].cpu().numpy()
                if real:
                    ref = ref.real
                err = _rel(got, ref)
                assert err <= TOL[prec], (name, window, real, b, err)
            del out
        p.close()
