"""Pins for the oracle's transform (no GPU): brute force through explicit
time-frequency shift operators, closed forms, covariance, library special
cases, route equality and adjoint identities."""
from math import gcd

import numpy as np
import pytest

from oracle import dgt as D
from oracle import lattice as La
from workloads import gaussian_window, hann_window

RNG = np.random.default_rng(1234)


def _crand(n):
    return RNG.standard_normal(n) + 1j * RNG.standard_normal(n)


def _tf_shift(g, x, omega):
    """pi(x, omega) g = M_omega T_x g built from the operator definitions of Section 2.1:
    T_x g(l) = g(l - x) (a roll), M_omega h(l) = exp(2 pi i l omega / L) h(l)."""
    L = g.shape[0]
    return np.exp(2j * np.pi * np.arange(L) * omega / L) * np.roll(g, x)


def _brute_coefficients(f, g, a, M, l1, l2):
    """<f, pi(lambda) g> for every lambda of the lattice, generated as the point set of
    the normal-form matrix, then arranged at (m, n) by x = a n, omega = m b + (n s mod b)."""
    L = f.shape[0]
    lat = La.Lattice(L, a, M, l1, l2)
    out = np.full((M, lat.N), np.nan + 0j)
    for (x, om) in lat.points():
        n = x // a
        m = (om - (n * lat.s) % lat.b) // lat.b
        assert (om - (n * lat.s) % lat.b) % lat.b == 0
        out[m, n] = np.vdot(_tf_shift(g, x, om), f)
    assert not np.isnan(out).any()
    return out


@pytest.mark.parametrize("params", [(36, 6, 6, 0, 1), (36, 6, 6, 1, 2), (36, 6, 6, 1, 3), (36, 6, 6, 2, 3),
                                    (48, 4, 8, 1, 2), (24, 2, 6, 1, 4), (60, 5, 10, 1, 2)])
def test_direct_sum_equals_operator_brute_force(params):
    L, a, M, l1, l2 = params
    f, g = _crand(L), _crand(L)
    ref = _brute_coefficients(f, g, a, M, l1, l2)
    c = D.dgt_direct(f, g, a, M, l1, l2)
    assert np.linalg.norm(c - ref) <= 1e-13 * np.linalg.norm(ref)


def _all_routes(f, g, a, M, l1, l2):
    out = {"fold": D.dgt_fold(f, g, a, M, l1, l2), "coset": D.dgt_coset(f, g, a, M, l1, l2),
           "shear": D.dgt_shear(f, g, a, M, l1, l2)}
    if l2 == 1:
        out["sep_zak"] = D.dgt_sep_zak(f, g, a, M)
    return out


def test_routes_equal_direct_on_every_small_lattice():
    """Coset (Prop. mwindec), shear (Algorithm 1, both branches), fold and the separable
    Zak factorisation all reproduce the definition on every feasible lattice, L <= 40."""
    count = 0
    for L in range(2, 41):
        for a in range(1, L + 1):
            if L % a:
                continue
            for M in range(1, L + 1):
                if L % M:
                    continue
                for l2 in range(1, 5):
                    for l1 in range(l2):
                        if gcd(l1, l2) != 1 or not La.feasible(L, a, M, l1, l2):
                            continue
                        f, g = _crand(L), _crand(L)
                        ref = D.dgt_direct(f, g, a, M, l1, l2)
                        for name, c in _all_routes(f, g, a, M, l1, l2).items():
                            assert np.linalg.norm(c - ref) <= 1e-12 * np.linalg.norm(ref), (name, L, a, M, l1, l2)
                        count += 1
    assert count > 900


def test_shear_result_independent_of_shear_pair():
    """Several valid (s0, s1) give the same coefficients (the result is unique)."""
    L, a, M, l1, l2 = 48, 4, 8, 1, 2
    lat = La.Lattice(L, a, M, l1, l2)
    f, g = _crand(L), _crand(L)
    ref = D.dgt_direct(f, g, a, M, l1, l2)
    found = 0
    for s1 in range(0, 12):
        v = s1 * a + lat.s
        X, k1, _ = La.ext_gcd(v, lat.b)
        mod = a * lat.b // X
        for s0 in range(1, mod):
            if (s0 * X + a * k1) % mod == 0:
                sh = La.Shear(s0, s1, X, L)
                c = D.dgt_shear(f, g, a, M, l1, l2, shear=sh)
                assert np.linalg.norm(c - ref) <= 1e-12 * np.linalg.norm(ref), (s0, s1)
                found += 1
                break
    assert found >= 3


@pytest.mark.parametrize("params", [(1440, 16, 48, 1, 2), (1440, 16, 48, 0, 1), (1440, 15, 45, 1, 2),
                                    (2160, 30, 60, 1, 3), (4096, 64, 512, 1, 2), (4096, 32, 256, 3, 4)])
def test_closed_forms_impulses(params):
    """g = delta_0 gives c(m,n) = f(an) e^{-2 pi i a n (m + w(n))/M}; f = delta_{l0} gives
    c(m,n) = conj(g(l0 - an)) e^{-2 pi i l0 (m + w(n))/M}, at any size, every route."""
    L, a, M, l1, l2 = params
    lat = La.Lattice(L, a, M, l1, l2)
    n = np.arange(lat.N)
    m = np.arange(M)[:, None]
    wn = (n * l1) % l2
    f = _crand(L)
    delta = np.zeros(L, complex)
    delta[0] = 1
    ref = f[a * n][None, :] * np.exp(-2j * np.pi * (((a * n)[None, :] * (l2 * m + wn[None, :])) % (l2 * M)) / (l2 * M))
    for name, c in _all_routes(f, delta, a, M, l1, l2).items():
        assert np.abs(c - ref).max() <= 1e-12 * np.abs(ref).max(), name
    l0 = 7 % L
    g = _crand(L)
    fd = np.zeros(L, complex)
    fd[l0] = 1
    ref = np.conj(g[(l0 - a * n) % L])[None, :] * np.exp(-2j * np.pi * ((l0 * (l2 * m + wn[None, :])) % (l2 * M)) / (l2 * M))
    for name, c in _all_routes(fd, g, a, M, l1, l2).items():
        assert np.abs(c - ref).max() <= 1e-12 * np.abs(ref).max(), name


def test_special_case_is_the_dft():
    """a = L (one time position), constant window: c(., 0) is numpy's unnormalised FFT."""
    L = 60
    f = _crand(L)
    c = D.dgt_direct(f, np.ones(L), L, L)
    assert np.allclose(c[:, 0], np.fft.fft(f), atol=1e-12)
    c2 = D.dgt_sep_zak(f, np.ones(L), L, L)
    assert np.allclose(c2[:, 0], np.fft.fft(f), atol=1e-12)


@pytest.mark.parametrize("params", [(1440, 16, 48, 1, 2), (2160, 30, 60, 1, 3), (480, 8, 24, 3, 4)])
def test_covariance(params):
    """T_{lam2 a j} f shifts columns by lam2 j with phase e^{-2 pi i x (m + w(n))/M};
    M_b f shifts rows by one (consequences of the TF-shift definitions)."""
    L, a, M, l1, l2 = params
    lat = La.Lattice(L, a, M, l1, l2)
    f, g = _crand(L), gaussian_window(L)
    c = D.dgt_coset(f, g, a, M, l1, l2)
    x = l2 * a
    cs = D.dgt_shear(np.roll(f, x), g, a, M, l1, l2)
    n = np.arange(lat.N)
    m = np.arange(M)[:, None]
    ph = np.exp(-2j * np.pi * ((x * (l2 * m + ((n * l1) % l2)[None, :])) % (l2 * M)) / (l2 * M))
    assert np.allclose(cs, ph * np.roll(c, l2, axis=1), atol=1e-11)
    fm = np.exp(2j * np.pi * np.arange(L) * lat.b / L) * f
    cm = D.dgt_fold(fm, g, a, M, l1, l2)
    assert np.allclose(cm, np.roll(c, 1, axis=0), atol=1e-11)


@pytest.mark.parametrize("params", [(1440, 16, 48, 1, 2), (2160, 30, 60, 1, 3), (480, 8, 24, 3, 4),
                                    (4096, 64, 512, 1, 2)])
def test_adjoint_identities(params):
    """<C f, c> = <f, C* c> for each route's synthesis (synthesis is the adjoint)."""
    L, a, M, l1, l2 = params
    N = L // a
    f, g = _crand(L), _crand(L)
    cc = RNG.standard_normal((M, N)) + 1j * RNG.standard_normal((M, N))
    for fw, bw in ((D.dgt_fold, D.idgt_fold), (D.dgt_coset, D.idgt_coset), (D.dgt_shear, D.idgt_shear)):
        lhs = np.vdot(cc, fw(f, g, a, M, l1, l2))
        rhs = np.vdot(bw(cc, g, a, M, l1, l2), f)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_synthesis_matches_direct_small():
    L, a, M, l1, l2 = 48, 4, 8, 1, 2
    g = _crand(L)
    cc = RNG.standard_normal((M, L // a)) + 1j * RNG.standard_normal((M, L // a))
    ref = D.idgt_direct(cc, g, a, M, l1, l2)
    for bw in (D.idgt_fold, D.idgt_coset, D.idgt_shear):
        assert np.linalg.norm(bw(cc, g, a, M, l1, l2) - ref) <= 1e-12 * np.linalg.norm(ref)


def test_synthesis_of_selected_columns_matches_direct():
    """idgt_fold(cols=S) on the columns S equals the direct synthesis (Section 2.1, inversion
    formula) of the full array that is zero outside S, for every lambda2 and column mix
    (first, last, both parities of w(n))."""
    for L, a, M, l1, l2 in ((48, 4, 8, 1, 2), (72, 6, 12, 1, 3), (64, 4, 16, 0, 1)):
        N = L // a
        g = _crand(L)
        cols = [0, 1, N // 2 + 1, N - 1]
        cc = np.zeros((M, N), dtype=np.complex128)
        cc[:, cols] = RNG.standard_normal((M, len(cols))) + 1j * RNG.standard_normal((M, len(cols)))
        ref = D.idgt_direct(cc, g, a, M, l1, l2)
        got = D.idgt_fold(cc[:, cols], g, a, M, l1, l2, cols=cols)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_pchirp_is_second_degree_character():
    """pchirp(L, s)(l + x) = pchirp(L, s)(l) pchirp(L, s)(x) e^{2 pi i s l x / L}: the
    identity used in Lemma meta_phases for U_{S_c}; with (L+1) it holds for odd and even L."""
    for L in (36, 37, 1440):
        for s in (1, 3, L - 2):
            p = D.pchirp(L, s)
            l = np.arange(L)
            for x in (1, 5, L - 1):
                lhs = p[(l + x) % L]
                rhs = p * p[x] * np.exp(2j * np.pi * ((s * l * x) % L) / L)
                assert np.allclose(lhs, rhs, atol=1e-12)


def test_hann_window_is_fir():
    L, Lg = 4096, 256
    h = hann_window(L, Lg)
    nz = np.nonzero(h)[0]
    assert len(nz) == Lg - 1                      # first periodic-Hann tap is 0
    assert abs(np.linalg.norm(h) - 1) < 1e-14
    assert np.allclose(h[1:Lg // 2], h[L - 1:L - Lg // 2:-1])   # even about 0
