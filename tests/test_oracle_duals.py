"""Pins for the oracle's dual and tight windows (no GPU): perfect reconstruction,
Parseval, dense frame operator, the diagonal closed form for short windows, and
Algorithm 2 (with the reading that its final un-chirp is required)."""
import numpy as np
import pytest

from oracle import dgt as D
from oracle import duals as U
from oracle import lattice as La
from workloads import gaussian_window, hann_window

RNG = np.random.default_rng(77)

FRAMES = [(36, 3, 6, 1, 2), (16, 2, 4, 1, 2), (48, 4, 8, 1, 2), (96, 4, 8, 1, 3), (120, 4, 10, 1, 2),
          (144, 4, 12, 1, 3), (144, 4, 12, 3, 4), (240, 4, 12, 1, 4), (288, 6, 18, 1, 2)]


def _crand(n):
    return RNG.standard_normal(n) + 1j * RNG.standard_normal(n)


@pytest.mark.parametrize("params", FRAMES)
def test_zak_and_shear_duals_equal_dense(params):
    L, a, M, l1, l2 = params
    g = gaussian_window(L)
    gd = U.dense_dual(g, a, M, l1, l2)
    gt = U.dense_tight(g, a, M, l1, l2)
    assert np.linalg.norm(U.zak_gram_dual(g, a, M, l1, l2) - gd) <= 1e-12 * np.linalg.norm(gd)
    assert np.linalg.norm(U.zak_gram_tight(g, a, M, l1, l2) - gt) <= 1e-12 * np.linalg.norm(gt)
    assert np.linalg.norm(U.shear_dual(g, a, M, l1, l2) - gd) <= 1e-12 * np.linalg.norm(gd)


@pytest.mark.parametrize("params", FRAMES + [(1440, 16, 48, 1, 2)])
def test_perfect_reconstruction_and_parseval(params):
    """C_gamma^* C_g f = f for gamma = S^{-1} g; ||C_{g_t} f|| = ||f|| for g_t = S^{-1/2} g."""
    L, a, M, l1, l2 = params
    g = gaussian_window(L)
    gd = U.zak_gram_dual(g, a, M, l1, l2)
    gt = U.zak_gram_tight(g, a, M, l1, l2)
    f = _crand(L)
    c = D.dgt_coset(f, g, a, M, l1, l2)
    fr = D.idgt_shear(c, gd, a, M, l1, l2)
    assert np.linalg.norm(fr - f) <= 1e-12 * np.linalg.norm(f)
    ct = D.dgt_shear(f, gt, a, M, l1, l2)
    assert abs(np.linalg.norm(ct) ** 2 / np.linalg.norm(f) ** 2 - 1) <= 1e-12
    # tight system: C_{g_t}^* C_{g_t} = I
    assert np.linalg.norm(D.idgt_coset(ct, gt, a, M, l1, l2) - f) <= 1e-12 * np.linalg.norm(f)


def test_frame_operator_diagonal_for_short_windows():
    """supp g within M samples: S = diag(M sum_n |g(l - an)|^2) for any lambda (the
    m-sum of the atoms' products vanishes off the diagonal)."""
    L, a, M = 96, 4, 16
    g = hann_window(L, 16)
    for (l1, l2) in ((0, 1), (1, 2), (1, 3), (3, 4)):
        if not La.feasible(L, a, M, l1, l2):
            continue
        S = U.frame_operator(g, a, M, l1, l2)
        diag = np.diag(S).real
        assert np.abs(S - np.diag(np.diag(S))).max() <= 1e-13 * diag.max()
        gd = U.fir_dual_diag(g, a, M)
        assert np.allclose(U.zak_gram_dual(g, a, M, l1, l2), gd, atol=1e-13)


def test_fir_dual_closed_form_at_workload_scale():
    """Hann window of length M on the quincunx audio lattice (scaled to L = 16384):
    the Zak-Gram dual equals the diagonal closed form."""
    L, a, M = 16384, 128, 1024
    g = hann_window(L, 1024)
    gd = U.fir_dual_diag(g, a, M)
    z = U.zak_gram_dual(g, a, M, 1, 2)
    assert np.linalg.norm(z - gd) <= 1e-12 * np.linalg.norm(gd)


def test_algorithm2_needs_final_unchirp():
    """Reading of Algorithm 2: when s1 != 0 the listing's output is the dual of the
    chirped window; undoing the chirp recovers S^{-1} g, skipping it does not."""
    L, a, M, l1, l2 = 36, 3, 6, 1, 2
    sh = La.shearfind(L, a, M, l1, l2)
    assert sh.s1 != 0
    g = gaussian_window(L)
    gd = U.dense_dual(g, a, M, l1, l2)
    with_unchirp = U.shear_dual(g, a, M, l1, l2)
    listing_only = with_unchirp * D.pchirp(L, sh.s1)
    assert np.linalg.norm(with_unchirp - gd) <= 1e-12 * np.linalg.norm(gd)
    assert np.linalg.norm(listing_only - gd) > 0.1 * np.linalg.norm(gd)
