"""Frame operator, canonical dual and canonical tight windows (float64; test infrastructure only).

The frame operator of the Gabor system G(g, Lambda) is S = C* C (eq. frameop),
C the analysis operator of eq. (DGT).  For a lattice (a subgroup) the canonical
dual system is G(S^{-1} g, Lambda) and the canonical tight system G(S^{-1/2} g,
Lambda) (Section 2.1); the tight window makes the frame Parseval, ||C f|| = ||f||.

Three independent ways to the same windows:
  dense_*        S as an explicit L x L matrix (small L).
  zak_gram_*     block structure of S in the Zak domain of the separable lattice
                 (the factorisation used by the separable dual, Section 4.2), summed
                 over the coset windows for a nonseparable lattice (eq. mw_frop).
  shear_dual     Algorithm 2 (gabdualns), separable dual of the sheared window.
  fir_dual_diag  closed form when the window support is at most M long: S is
                 then diagonal, (S f)(l) = M sum_n |g(l - a n)|^2 f(l).
"""
from __future__ import annotations

import numpy as np

from .dgt import coset_windows, dgt_direct, pchirp, zak, _cexp
from .lattice import Lattice, sep_constants, shearfind


# ----------------------------------------------------------------------------
# dense frame operator (small L)
# ----------------------------------------------------------------------------
def analysis_matrix(g, a, M, lam1=0, lam2=1) -> np.ndarray:
    """Rows indexed (n, m) -> n*M + m: conj of the atom M_{mb+s(n)} T_{an} g (eq. DGT)."""
    g = np.asarray(g, dtype=np.complex128)
    L = g.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    l = np.arange(L, dtype=np.int64)
    rows = np.empty((lat.N * M, L), dtype=np.complex128)
    for n in range(lat.N):
        wn = lat.freq_offset_num(n)
        win = np.conj(g[(l - a * n) % L])
        for m in range(M):
            rows[n * M + m] = win * _cexp(l * (lam2 * m + wn), lam2 * M)
    return rows


def frame_operator(g, a, M, lam1=0, lam2=1) -> np.ndarray:
    C = analysis_matrix(g, a, M, lam1, lam2)
    return C.conj().T @ C


def dense_dual(g, a, M, lam1=0, lam2=1) -> np.ndarray:
    S = frame_operator(g, a, M, lam1, lam2)
    return np.linalg.solve(S, np.asarray(g, dtype=np.complex128))


def dense_tight(g, a, M, lam1=0, lam2=1) -> np.ndarray:
    S = frame_operator(g, a, M, lam1, lam2)
    ev, V = np.linalg.eigh(S)
    return V @ ((V.conj().T @ np.asarray(g, dtype=np.complex128)) / np.sqrt(ev))


# ----------------------------------------------------------------------------
# Zak-domain Gram blocks
# ----------------------------------------------------------------------------
def _phi_blocks(ZG, a, M, p, q, d, K0):
    """Phi[xi, k, i, w] = ZG~[xi, k + iM - a w] (quasi-periodic extension to negative
    columns, ZG~[xi, col - K0] = e^{-2 pi i xi/d} ZG[xi, col]).  Shape (d, M, p, q)."""
    xi = np.arange(d)
    wrap = _cexp(xi, d)[:, None]
    kk = np.arange(M)
    Phi = np.empty((d, M, p, q), dtype=np.complex128)
    for i in range(p):
        for w in range(q):
            col = kk + M * i - a * w
            blk = ZG[:, col % K0].copy()
            blk[:, col < 0] *= wrap
            Phi[:, :, i, w] = blk
    return Phi


def zak_gram(windows, at, M) -> tuple[np.ndarray, dict]:
    """Gram blocks G[xi, k] = M sum_j Phi_j Phi_j^H (p x p) of the frame operator of the
    union of separable systems G(g_j, at, M): in the Zak domain of that separable
    lattice, Z(S f)[xi, k + iM] = sum_i' G[xi, k][i, i'] Z f[xi, k + i'M]."""
    L = windows[0].shape[0]
    k_ = sep_constants(L, at, M)
    p, q, d = k_["p"], k_["q"], k_["d"]
    K0 = L // d
    G = np.zeros((d, M, p, p), dtype=np.complex128)
    for gj in windows:
        Phi = _phi_blocks(zak(gj, d), at, M, p, q, d, K0)
        G += M * np.einsum("xkiw,xkjw->xkij", Phi, Phi.conj())
    return G, dict(p=p, q=q, d=d, K0=K0)


def _apply_blocks(G, g, d, M, p, fn):
    """Apply fn(G) blockwise to the Zak transform of g and invert the Zak transform."""
    L = g.shape[0]
    K0 = L // d
    Zg = zak(g, d)
    vec = np.stack([Zg[:, np.arange(M) + M * i] for i in range(p)], axis=-1)   # (d, M, p)
    out = np.einsum("xkij,xkj->xki", fn(G), vec)
    Zo = np.empty((d, K0), dtype=np.complex128)
    for i in range(p):
        Zo[:, np.arange(M) + M * i] = out[..., i]
    return (np.fft.ifft(Zo, axis=0)).reshape(L)


def _inv(G):
    return np.linalg.inv(G)


def _inv_sqrt(G):
    ev, V = np.linalg.eigh(G)
    return np.einsum("...ij,...j,...kj->...ik", V, 1.0 / np.sqrt(ev), V.conj())


def zak_gram_dual(g, a, M, lam1=0, lam2=1) -> np.ndarray:
    """Canonical dual S^{-1} g through the Zak-domain Gram blocks of the coset
    decomposition (S = sum_j S_{g_j, tilde-Lambda}, eq. mw_frop)."""
    g = np.asarray(g, dtype=np.complex128)
    at = lam2 * a
    G, k_ = zak_gram(coset_windows(g, a, M, lam1, lam2), at, M)
    return _apply_blocks(G, g, k_["d"], M, k_["p"], _inv)


def zak_gram_tight(g, a, M, lam1=0, lam2=1) -> np.ndarray:
    """Canonical tight window S^{-1/2} g through the same Gram blocks."""
    g = np.asarray(g, dtype=np.complex128)
    at = lam2 * a
    G, k_ = zak_gram(coset_windows(g, a, M, lam1, lam2), at, M)
    return _apply_blocks(G, g, k_["d"], M, k_["p"], _inv_sqrt)


def gram_condition(g, a, M, lam1=0, lam2=1) -> float:
    """Ratio of the largest to the smallest eigenvalue of S (frame bound ratio)."""
    g = np.asarray(g, dtype=np.complex128)
    G, _ = zak_gram(coset_windows(g, a, M, lam1, lam2), lam2 * a, M)
    ev = np.linalg.eigvalsh(G)
    return float(ev.max() / ev.min())


# ----------------------------------------------------------------------------
# Algorithm 2 (dual through the shear)
# ----------------------------------------------------------------------------
def shear_dual(g, a, M, lam1, lam2, shear=None) -> np.ndarray:
    """Algorithm 2 (gabdualns): chirp by pchirp(L, s1); separable dual on (a_r, M_r)
    when s0 = 0, otherwise L * separable dual of pchirp(L,-s0) FFT(g) on (L/M_r, L/a_r)
    followed by IFFT(conj(pchirp(L,-s0)) .).  Reading: the listing stops there; the
    final step of the metaplectic conjugation, multiplication by conj(pchirp(L, s1)),
    is applied as well (S^{-1} = U S~^{-1} U^{-1} with U^{-1} the chirp, eq. shearframeop)."""
    g = np.asarray(g, dtype=np.complex128).copy()
    L = g.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    sh = shearfind(L, a, M, lam1, lam2) if shear is None else shear
    p1 = pchirp(L, sh.s1) if sh.s1 != 0 else np.ones(L, dtype=np.complex128)
    g = p1 * g
    Mr = L // sh.b_r
    ar = a * lat.b // sh.b_r
    if not sh.freq_shear:
        gd = zak_gram_dual(g, ar, Mr)
    else:
        p0 = pchirp(L, -sh.s0)
        gh = p0 * np.fft.fft(g)
        gd = L * zak_gram_dual(gh, L // Mr, L // ar)
        gd = np.fft.ifft(np.conj(p0) * gd)
    return np.conj(p1) * gd


# ----------------------------------------------------------------------------
# short windows: diagonal frame operator
# ----------------------------------------------------------------------------
def fir_dual_diag(g, a, M) -> np.ndarray:
    """gamma(l) = g(l) / (M sum_n |g(l - a n)|^2), exact when supp g fits in M samples
    (then only the m-sum's diagonal survives: painless nonorthogonal expansion),
    for every lattice with time step a and M channels."""
    g = np.asarray(g, dtype=np.complex128)
    L = g.shape[0]
    N = L // a
    # sum_n |g(l - a n)|^2 depends on l mod a only: the rows of |g|^2 viewed as [N][a], summed
    per = (np.abs(g) ** 2).reshape(N, a).sum(axis=0)
    den = np.tile(per, N)
    return g / (M * den)
