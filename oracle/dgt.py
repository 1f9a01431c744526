"""The discrete Gabor transform on a nonseparable lattice, float64, CPU (test infrastructure only).

Result (eq. DGT, Section 2.1, read 0-based as g(l - a n)):

    c(m, n) = sum_{l<L} f(l) conj(g(l - a n)) exp(-2 pi i l (m + w(n)) / M),
    w(n) = ((n lam1) mod lam2) / lam2,   m < M, n < N = L/a,

i.e. c(m, n) = V_g f(a n, m b + (n s mod b)) with the frequency-invariant
phase convention of the STFT in Section 2.1.  Synthesis with a window gamma
is the adjoint  f(l) = sum_{m,n} c(m,n) gamma(l - a n) exp(+2 pi i l (m + w(n))/M).

Coefficient arrays are indexed c[m, n] (shape (M, N)).  Every phase is
reduced exactly in integers before ``exp`` is taken.

Routes, all computing the same c:
  dgt_direct       O1: the definition, as a sum over l for every (m, n).
  dgt_fold         O2: fold the windowed, modulated signal modulo M, then an
                   M-point FFT per time position (weighted overlap-add form).
  dgt_sep_zak      O3: separable lattice (lam = 0) through the Zak/polyphase
                   factorisation whose cost is eq. (rect-flops).
  dgt_coset        coset route: Prop. mwindec + eq. (mw_phases).
  dgt_shear        shear route: Algorithm 1 as printed (both branches).
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice, alg1_constants, sep_constants, shearfind

TWO_PI = 2.0 * np.pi


def _cexp(num, den, sign=-1.0):
    """exp(sign * 2 pi i num/den) for an exactly reduced integer numerator."""
    num = np.asarray(num, dtype=np.int64) % den
    return np.exp(sign * 1j * TWO_PI * num.astype(np.float64) / den)


def pchirp(L: int, s: int) -> np.ndarray:
    """Discrete chirp pchirp(L, s)(l) = exp(pi i s l^2 (L+1)/L) (Lemma meta_phases,
    U_{S_c}; Section 4.1).  Exponent reduced modulo 2L in exact integers."""
    twoL = 2 * L
    l = np.arange(L, dtype=np.int64)
    e = _mulmod(s, _mulmod(_mulmod(l, l, twoL), L + 1, twoL), twoL)
    return np.exp(1j * np.pi * e.astype(np.float64) / L)


# ----------------------------------------------------------------------------
# O1: direct sum
# ----------------------------------------------------------------------------
def dgt_direct(f, g, a, M, lam1=0, lam2=1) -> np.ndarray:
    """c(m,n) by the definition (eq. DGT), O(L M N).  Small L only."""
    f = np.asarray(f, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    L = f.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    l = np.arange(L, dtype=np.int64)
    den = lam2 * M
    c = np.empty((M, lat.N), dtype=np.complex128)
    for n in range(lat.N):
        win = np.conj(g[(l - a * n) % L])
        wn = lat.freq_offset_num(n)
        for m in range(M):
            # exponent l (m + wn/lam2) / M = l (lam2 m + wn) / (lam2 M)
            c[m, n] = np.sum(f * win * _cexp(l * (lam2 * m + wn), den))
    return c


def idgt_direct(c, gamma, a, M, lam1=0, lam2=1) -> np.ndarray:
    """Synthesis f(l) = sum_{m,n} c(m,n) gamma(l - a n) exp(2 pi i l (m + w(n))/M):
    the adjoint of dgt_direct with window gamma (Section 2.1).  Small L only."""
    gamma = np.asarray(gamma, dtype=np.complex128)
    L = gamma.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    l = np.arange(L, dtype=np.int64)
    den = lam2 * M
    f = np.zeros(L, dtype=np.complex128)
    for n in range(lat.N):
        win = gamma[(l - a * n) % L]
        wn = lat.freq_offset_num(n)
        for m in range(M):
            f += c[m, n] * win * _cexp(l * (lam2 * m + wn), den, sign=+1.0)
    return f


# ----------------------------------------------------------------------------
# O2: fold modulo M + FFT_M  (exact rearrangement of the sum over l)
# ----------------------------------------------------------------------------
def dgt_fold(f, g, a, M, lam1=0, lam2=1, cols=None) -> np.ndarray:
    """c(., n) = FFT_M of h_n(k) = sum_j f(k+jM) conj(g(k+jM-an)) e^{-2 pi i (k+jM) w(n)/M}.

    O(L) per time position.  ``cols`` restricts the computation to a subset of
    time positions n (returns shape (M, len(cols)))."""
    f = np.asarray(f, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    L = f.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    cols = range(lat.N) if cols is None else cols
    l = np.arange(L, dtype=np.int64)
    out = np.empty((M, len(cols)), dtype=np.complex128)
    for i, n in enumerate(cols):
        mod = _cexp(l * lat.freq_offset_num(n), lam2 * M)
        v = f * np.conj(g[(l - a * n) % L]) * mod
        h = v.reshape(L // M, M).sum(axis=0)
        out[:, i] = np.fft.fft(h)
    return out


def idgt_fold(c, gamma, a, M, lam1=0, lam2=1, cols=None) -> np.ndarray:
    """Adjoint of dgt_fold: unnormalised inverse FFT_M per column, unfold, window, sum.

    O(L) per time position.  ``cols`` lists the time positions n that ``c`` holds (shape
    (M, len(cols))): the synthesis of a coefficient array that is zero on every other
    column."""
    gamma = np.asarray(gamma, dtype=np.complex128)
    L = gamma.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    l = np.arange(L, dtype=np.int64)
    f = np.zeros(L, dtype=np.complex128)
    cols = list(range(lat.N)) if cols is None else list(cols)
    for i, n in enumerate(cols):
        h = np.fft.ifft(c[:, i]) * M
        mod = _cexp(l * lat.freq_offset_num(n), lam2 * M, sign=+1.0)
        f += np.tile(h, L // M) * gamma[(l - a * n) % L] * mod
    return f


# ----------------------------------------------------------------------------
# O3: separable lattice via the Zak / polyphase factorisation (eq. rect-flops)
# ----------------------------------------------------------------------------
def zak(x: np.ndarray, d: int) -> np.ndarray:
    """Zak transform used by the factorisation: Z[xi, col] = sum_{mu<d}
    x(col + K0 mu) e^{-2 pi i mu xi / d}, K0 = L/d, shape (d, K0)."""
    L = x.shape[-1]
    return np.fft.fft(np.asarray(x, dtype=np.complex128).reshape(d, L // d), axis=0)


def dgt_sep_zak(f, g, a, M) -> np.ndarray:
    """Separable DGT c(m,n) = sum_l f(l) conj(g(l - a n)) e^{-2 pi i l m / M}.

    With c, d, p, q of eqs. (cd, pq), K0 = L/d = c p q, and n = w + q nu
    (w < q, nu < d), the sum over l = k + jM, j = i + p mu becomes

      h_{w+q nu}(k) = (1/d) sum_xi e^{2 pi i nu xi/d}
                      sum_{i<p} ZF[xi, k+iM] conj(ZG~[xi, k+iM-aw])     (*)
      c(m, n)      = sum_{k<M} h_n(k) e^{-2 pi i k m / M}

    where ZF, ZG are the Zak transforms of f and g and ZG~ extends ZG to
    negative columns by quasi-periodicity ZG~[xi, col-K0] = e^{-2 pi i xi/d} ZG[xi, col].
    The three steps are the signal factorisation (4 L log d), the block
    products (8 L q) and the two FFT stages (4 MN log d + 4 MN log M) counted
    in eq. (rect-flops).
    """
    f = np.asarray(f, dtype=np.complex128)
    L = f.shape[0]
    k_ = sep_constants(L, a, M)
    p, q, d = k_["p"], k_["q"], k_["d"]
    K0 = L // d
    N = L // a
    ZF = zak(f, d)
    ZG = zak(g, d)
    xi = np.arange(d)
    unwrap = _cexp(xi, d, sign=+1.0)[:, None]        # conj(e^{-2 pi i xi/d})
    Y = np.empty((N, M), dtype=np.complex128)
    kk = np.arange(M)
    for w in range(q):
        X = np.zeros((d, M), dtype=np.complex128)
        for i in range(p):
            colF = kk + M * i
            colG = colF - a * w
            wrapped = colG < 0
            Gc = np.conj(ZG[:, colG % K0])
            Gc[:, wrapped] *= unwrap
            X += ZF[:, colF] * Gc
        Y[w::q, :] = np.fft.ifft(X, axis=0)             # rows nu -> n = w + q nu
    return np.fft.fft(Y, axis=1).T                      # c[m, n]


def idgt_sep_zak(c, gamma, a, M) -> np.ndarray:
    """Adjoint of dgt_sep_zak with window gamma: each step of (*) transposed
    in reverse order (unnormalised inverse FFT over m, forward FFT over nu
    with 1/d, multiplication by the window factor and sum over w, inverse Zak)."""
    gamma = np.asarray(gamma, dtype=np.complex128)
    L = gamma.shape[0]
    k_ = sep_constants(L, a, M)
    p, q, d = k_["p"], k_["q"], k_["d"]
    K0 = L // d
    ZG = zak(gamma, d)
    xi = np.arange(d)
    wrap = _cexp(xi, d)[:, None]                       # e^{-2 pi i xi/d}
    Y = np.fft.ifft(np.asarray(c).T, axis=1) * M       # [n][k]
    ZFt = np.zeros((d, K0), dtype=np.complex128)
    kk = np.arange(M)
    for w in range(q):
        Xt = np.fft.fft(Y[w::q, :], axis=0) / d        # adjoint of ifft over xi
        for i in range(p):
            colF = kk + M * i
            colG = colF - a * w
            wrapped = colG < 0
            Gw = ZG[:, colG % K0].copy()
            Gw[:, wrapped] *= wrap
            ZFt[:, colF] += Xt * Gw
    return (np.fft.ifft(ZFt, axis=0) * d).reshape(L)   # adjoint of the Zak DFT


# ----------------------------------------------------------------------------
# coset route (Prop. mwindec, eqs. mw_frop / mw_phases)
# ----------------------------------------------------------------------------
def coset_windows(g, a, M, lam1, lam2) -> list[np.ndarray]:
    """g_j = M_{sigma_j} T_{j a} g with sigma_j = j s mod b, j < lam2 (Prop. mw_frop)."""
    g = np.asarray(g, dtype=np.complex128)
    L = g.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    l = np.arange(L, dtype=np.int64)
    out = []
    for j in range(lam2):
        sigma = (j * lat.s) % lat.b
        out.append(_cexp(sigma * l, L, sign=+1.0) * np.roll(g, j * a))
    return out


def dgt_coset(f, g, a, M, lam1, lam2) -> np.ndarray:
    """c(m, lam2*nt + j) = e^{-2 pi i nt (lam2 a) sigma_j / L} c_j(m, nt) with c_j the
    separable DGT of f with window g_j on time step lam2*a (eq. mw_phases; the index
    relation printed as m = n - nt is read as j = n - lam2*nt)."""
    f = np.asarray(f, dtype=np.complex128)
    L = f.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    at = lam2 * a
    c = np.empty((M, lat.N), dtype=np.complex128)
    nt = np.arange(lat.N // lam2, dtype=np.int64)
    for j, gj in enumerate(coset_windows(g, a, M, lam1, lam2)):
        sigma = (j * lat.s) % lat.b
        cj = dgt_sep_zak(f, gj, at, M)
        c[:, j::lam2] = cj * _cexp(nt * at * sigma, L)[None, :]
    return c


def idgt_coset(c, gamma, a, M, lam1, lam2) -> np.ndarray:
    """Synthesis through the coset route: sum over j of the separable synthesis of the
    phase-corrected coset columns with the coset windows gamma_j (eq. mw_frop)."""
    L = np.asarray(gamma).shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    at = lam2 * a
    f = np.zeros(L, dtype=np.complex128)
    nt = np.arange(lat.N // lam2, dtype=np.int64)
    for j, gj in enumerate(coset_windows(gamma, a, M, lam1, lam2)):
        sigma = (j * lat.s) % lat.b
        cj = np.asarray(c)[:, j::lam2] * _cexp(nt * at * sigma, L, sign=+1.0)[None, :]
        f += idgt_sep_zak(cj, gj, at, M)
    return f


# ----------------------------------------------------------------------------
# shear route (Algorithm 1)
# ----------------------------------------------------------------------------
def _mulmod(x, y, m):
    """(x*y) mod m for int64 arrays whose reduced factors keep products below 2^62."""
    return (np.asarray(x, dtype=np.int64) % m) * (np.asarray(y, dtype=np.int64) % m) % m


def dgt_shear(f, g, a, M, lam1, lam2, shear=None) -> np.ndarray:
    """Algorithm 1 (dgtns) step by step: chirp by pchirp(L, s1) if s1 != 0; then either
    the separable DGT on (a, M) followed by the phase E and the column reindex
    (s0 = 0), or the frequency-domain DGT on (b_r, N_r) of pchirp(L,-s0) FFT(f)
    with the window pchirp(L,-s0) FFT(g)/L, followed by the phase E and the
    reindex of both indices (s0 != 0)."""
    f = np.asarray(f, dtype=np.complex128).copy()
    g = np.asarray(g, dtype=np.complex128).copy()
    L = f.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    sh = shearfind(L, a, M, lam1, lam2) if shear is None else shear
    b, N = lat.b, lat.N
    s0, s1 = sh.s0, sh.s1
    K = alg1_constants(L, a, M, sh)
    if s1 != 0:
        p = pchirp(L, s1)
        g = p * g
        f = p * f
    c = np.empty((M, N), dtype=np.complex128)
    if not sh.freq_shear:
        cr = dgt_sep_zak(f, g, a, M)
        k = np.arange(N, dtype=np.int64)
        E = np.exp(1j * np.pi * (_mulmod(K["C1"], _mulmod(k, k, 2 * N), 2 * N)).astype(np.float64) / N)
        m = np.arange(M, dtype=np.int64)
        for kk in range(N):
            rows = ((-(s1 * kk * a) + m * b) % L) // b
            c[rows, kk] = E[kk] * cr[:, kk]
        return c
    ar, Mr, Nr = K["ar"], K["Mr"], K["Nr"]
    C1, C2, C3, C4, C5, C6 = (K[x] for x in ("C1", "C2", "C3", "C4", "C5", "C6"))
    p0 = pchirp(L, -s0)
    g = p0 * np.fft.fft(g) / L
    f = p0 * np.fft.fft(f)
    cr = dgt_sep_zak(f, g, sh.b_r, Nr)                   # shape (Nr, Mr): channel, time
    twoN = 2 * N
    k = np.arange(Nr, dtype=np.int64)[:, None]
    m = np.arange(Mr, dtype=np.int64)[None, :]
    sq1 = (C1 * k + C2 * m) % twoN
    t1 = _mulmod(C3, _mulmod(sq1, sq1, twoN), twoN)
    t2 = _mulmod(m, (_mulmod(C4, m, twoN) + _mulmod(C5, k, twoN)) % twoN, twoN)
    E = np.exp(1j * np.pi * ((t1 - t2) % twoN).astype(np.float64) / N)
    mt = (C1 * k + C2 * m) % N
    kt = ((_mulmod(-s1 * ar, k, L) + _mulmod(C6, m, L)) % L) // b
    src = cr[(-k) % Nr, m]
    c[kt, mt] = E * src
    return c


def idgt_shear(c, gamma, a, M, lam1, lam2, shear=None) -> np.ndarray:
    """Synthesis through the shear route: the adjoint of dgt_shear, each step of
    Algorithm 1 transposed in reverse order (gather with conjugate phases,
    separable synthesis, inverse frequency shear and inverse chirp)."""
    c = np.asarray(c, dtype=np.complex128)
    gamma = np.asarray(gamma, dtype=np.complex128).copy()
    L = gamma.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    sh = shearfind(L, a, M, lam1, lam2) if shear is None else shear
    b, N = lat.b, lat.N
    s0, s1 = sh.s0, sh.s1
    K = alg1_constants(L, a, M, sh)
    p1 = pchirp(L, s1) if s1 != 0 else np.ones(L, dtype=np.complex128)
    gamma = p1 * gamma
    if not sh.freq_shear:
        k = np.arange(N, dtype=np.int64)
        E = np.exp(1j * np.pi * (_mulmod(K["C1"], _mulmod(k, k, 2 * N), 2 * N)).astype(np.float64) / N)
        m = np.arange(M, dtype=np.int64)
        cr = np.empty((M, N), dtype=np.complex128)
        for kk in range(N):
            rows = ((-(s1 * kk * a) + m * b) % L) // b
            cr[:, kk] = np.conj(E[kk]) * c[rows, kk]
        return np.conj(p1) * idgt_sep_zak(cr, gamma, a, M)
    ar, Mr, Nr = K["ar"], K["Mr"], K["Nr"]
    C1, C2, C3, C4, C5, C6 = (K[x] for x in ("C1", "C2", "C3", "C4", "C5", "C6"))
    twoN = 2 * N
    k = np.arange(Nr, dtype=np.int64)[:, None]
    m = np.arange(Mr, dtype=np.int64)[None, :]
    sq1 = (C1 * k + C2 * m) % twoN
    t1 = _mulmod(C3, _mulmod(sq1, sq1, twoN), twoN)
    t2 = _mulmod(m, (_mulmod(C4, m, twoN) + _mulmod(C5, k, twoN)) % twoN, twoN)
    E = np.exp(1j * np.pi * ((t1 - t2) % twoN).astype(np.float64) / N)
    mt = (C1 * k + C2 * m) % N
    kt = ((_mulmod(-s1 * ar, k, L) + _mulmod(C6, m, L)) % L) // b
    cr = np.empty((Nr, Mr), dtype=np.complex128)
    cr[(-k) % Nr, m] = np.conj(E) * c[kt, mt]
    p0 = pchirp(L, -s0)
    gh = p0 * np.fft.fft(gamma) / L
    fh = idgt_sep_zak(cr, gh, sh.b_r, Nr)               # adjoint of the separable step
    f = np.fft.ifft(np.conj(p0) * fh) * L                # adjoint of f -> p0 * FFT(f)
    return np.conj(p1) * f
