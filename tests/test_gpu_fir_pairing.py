"""FIR analysis of real signals with a real window (two columns of one w(n) share a complex
FFT, separated by the conjugate symmetry of a real sequence's transform, eq. DGT with the
modulation split as in eq. rect-flops-FIR), against the oracle's fold form on every
coefficient: lambda2 = 1 and 2, columns whose taps wrap around the end of the signal (the
first and last CTAs), an odd number of columns per w class (which takes the unpaired kernel),
real-signal half rows, and a complex window and a complex signal on the same lattice (no
pairing).  The real-output synthesis pairs the same way (two columns of one w share an
inverse FFT of their Hermitian parts): real output against the real part of the oracle's
synthesis, with the window and with its dual, and the real-signal half rows through
reconstruction.  float32 2e-6, float64 1e-12 relative l2 per signal."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dgt as OD  # noqa: E402
from oracle import dgtreal as OR  # noqa: E402
from workloads import hann_taps, real_normal  # noqa: E402

TOL = {"f64": 1e-12, "f32": 2e-6}


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


def _dev(x, prec):
    if np.iscomplexobj(x):
        return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex128 if prec == "f64" else np.complex64))).cuda()
    return torch.from_numpy(np.ascontiguousarray(x.astype(np.float64 if prec == "f64" else np.float32))).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _full(taps, center, L):
    g = np.zeros(L, dtype=taps.dtype)
    for t in range(len(taps)):
        g[(t - center) % L] = taps[t]
    return g


# (L, a, M, lambda1, lambda2, Lg)
LATTICES = [
    (4096, 64, 256, 1, 2, 256),        # pairs (n, n + 2); first / last CTA segments wrap
    (4096, 64, 256, 0, 1, 256),        # lambda2 = 1: pairs (n, n + 1)
    (65536, 128, 1024, 1, 2, 1024),    # the audio lattice at a smaller L
    (8448, 128, 128, 1, 2, 128),       # 33 columns per w class: the unpaired kernel
    (16384, 32, 512, 1, 2, 384),       # taps shorter than M, centre off the middle
]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("lat", LATTICES, ids=lambda v: "L%d-a%d-M%d-l%d_%d-g%d" % v)
def test_fir_real_pairing(prec, lat):
    from paper_1307_4569_gb300 import Plan

    L, a, M, l1, l2, Lg = lat
    taps, center = hann_taps(Lg)
    if Lg == 384:
        center = 100
    taps = _round(taps / np.linalg.norm(taps), prec)
    g = _full(taps, center, L)
    B = 3
    f = _round(np.stack([real_normal(L, 90, i) for i in range(B)]), prec)
    p = Plan(L, a, M, l1, l2, taps, route="fir", precision=prec, fir_center=center)
    fd = _dev(f, prec)
    c = p.dgt(fd).cpu().numpy()
    refs = [OD.dgt_fold(f[b], g, a, M, l1, l2).T for b in range(B)]
    for b in range(B):
        assert _rel(c[b], refs[b]) <= TOL[prec], (lat, b)
    # real-signal half rows (lambda2 <= 2, M even)
    ch = p.dgtreal(fd).cpu().numpy()
    for b in range(B):
        assert _rel(ch[b], refs[b][:, :M // 2 + 1]) <= TOL[prec], (lat, b)
        assert _rel(ch[b], OR.dgtreal(f[b], g, a, M, l1, l2).T) <= TOL[prec]
    # the same signals as complex input, and a complex window: no pairing, same coefficients
    cc = p.dgt(_dev(f.astype(np.complex128), prec)).cpu().numpy()
    for b in range(B):
        assert _rel(cc[b], refs[b]) <= TOL[prec]
    p.close()
    tz = _round(taps * np.exp(0.3j * np.arange(Lg)), prec)
    pz = Plan(L, a, M, l1, l2, tz, route="fir", precision=prec, fir_center=center)
    cz = pz.dgt(fd).cpu().numpy()
    gz = _full(tz, center, L)
    for b in range(B):
        assert _rel(cz[b], OD.dgt_fold(f[b], gz, a, M, l1, l2).T) <= TOL[prec]
    pz.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("lat", LATTICES, ids=lambda v: "L%d-a%d-M%d-l%d_%d-g%d" % v)
def test_fir_real_output_synthesis_pairing(prec, lat):
    from oracle import duals as OU
    from paper_1307_4569_gb300 import Plan

    L, a, M, l1, l2, Lg = lat
    N = L // a
    taps, center = hann_taps(Lg)
    if Lg == 384:
        center = 100
    taps = _round(taps / np.linalg.norm(taps), prec)
    g = _full(taps, center, L)
    B = 3
    r = np.random.default_rng((91, L))
    c = _round(r.standard_normal((B, N, M)) + 1j * r.standard_normal((B, N, M)), prec)
    p = Plan(L, a, M, l1, l2, taps, route="fir", precision=prec, fir_center=center)
    cd = _dev(c, prec)
    out = p.idgt(cd, window="adjoint", real=True).cpu().numpy()
    for b in range(B):
        assert _rel(out[b], OD.idgt_fold(c[b].T, g, a, M, l1, l2).real) <= TOL[prec], (lat, b)
    if N * M >= 2 * L:                                   # redundancy >= 2: a frame with the diagonal dual
        gd = OU.fir_dual_diag(g, a, M)
        out = p.idgt(cd, window="dual", real=True).cpu().numpy()
        for b in range(B):
            assert _rel(out[b], OD.idgt_fold(c[b].T, gd, a, M, l1, l2).real) <= TOL[prec], (lat, b)
        # half rows of a real signal's coefficients: perfect reconstruction
        f = _round(np.stack([real_normal(L, 92, i) for i in range(B)]), prec)
        back = p.idgtreal(p.dgtreal(_dev(f, prec)), window="dual").cpu().numpy()
        for b in range(B):
            assert _rel(back[b], f[b]) <= (1e-5 if prec == "f32" else 1e-12)
    p.close()
