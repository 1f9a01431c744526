"""Pins for the oracle's integer lattice algebra (no GPU)."""
import os
from math import gcd

import pytest

from oracle import lattice as La

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [list(map(int, ln.split())) for ln in fh if ln.strip() and not ln.startswith("#")]


def _normal_form_by_construction(pts, L):
    """Prop. lattNF's existence proof: b = min nonzero omega with (0, omega) in the
    lattice, a = min nonzero x of any point, s = min omega with (a, omega) in it."""
    b = min([w for (x, w) in pts if x == 0 and w != 0] or [L])
    a = min([x for (x, w) in pts if x != 0] or [L])
    s = min(w for (x, w) in pts if x == a % L)
    return a, s, b


@pytest.mark.parametrize("row", _rows("fig1_lattices.txt"))
def test_fig1_lattices_are_subgroups_in_normal_form(row):
    L, a, M, l1, l2, npts = row
    lat = La.Lattice(L, a, M, l1, l2)
    pts = lat.points()
    assert len(pts) == npts
    # closed under addition and negation: a subgroup of Z_L^2
    for (x1, w1) in list(pts)[:12]:
        for (x2, w2) in pts:
            assert ((x1 + x2) % L, (w1 + w2) % L) in pts
        assert ((-x1) % L, (-w1) % L) in pts
    assert _normal_form_by_construction(pts, L) == (a, lat.s, lat.b)
    # lambda = s / b in lowest terms (Section 2.1)
    g = gcd(lat.b, lat.s) if lat.s else lat.b
    assert (lat.s // g, lat.b // g) == ((l1, l2) if l1 else (0, 1))


def test_minimal_length_matches_lattice_conditions():
    """Prop. minsig: a|L, M|L, (L/a) lam and (L/M) lam integral  <=>  lam2 lcm(a,M) | L."""
    for a in range(1, 9):
        for M in range(1, 9):
            for l2 in range(1, 6):
                for l1 in range(l2):
                    if gcd(l1, l2) != 1:
                        continue
                    for L in range(1, 241):
                        cond = (L % a == 0 and L % M == 0
                                and ((L // a) * l1) % l2 == 0 and ((L // M) * l1) % l2 == 0)
                        assert cond == La.feasible(L, a, M, l1, l2), (L, a, M, l1, l2)


@pytest.mark.parametrize("row", _rows("fig2_lengths.txt"))
def test_fig2_lengths(row):
    a, M, L = row
    for l2 in range(1, 11):
        for l1 in range(l2):
            if gcd(l1, l2) == 1:
                assert La.feasible(L, a, M, l1, l2)
    # minimal: no proper divisor of L is legal for every lambda2 <= 10
    for div in range(1, L):
        if L % div == 0 and all(La.feasible(div, a, M, 1 if k > 1 else 0, k) for k in range(1, 11)):
            pytest.fail("smaller common legal length %d" % div)


@pytest.mark.parametrize("row", _rows("remark_noshear_lengths.txt"))
def test_remark_noshear_lengths(row):
    a, M, l1, l2, value = row
    assert La.min_length(a, M, l2) * La.noshear_length_factor(a, M, l1, l2) == value


def _all_small_lattices(Lmax):
    for L in range(2, Lmax + 1):
        for a in range(1, L + 1):
            if L % a:
                continue
            for M in range(1, L + 1):
                if L % M:
                    continue
                for l2 in range(1, 5):
                    for l1 in range(l2):
                        if gcd(l1, l2) == 1 and La.feasible(L, a, M, l1, l2):
                            yield L, a, M, l1, l2


def test_shearfind_yields_separable_lattice_small():
    """Theorem shearform: U^{-1}_{s0,s1} Lambda is the product lattice diag(a b/b_r, b_r),
    checked by enumerating the point sets (independent of eq. modcond)."""
    count = 0
    for (L, a, M, l1, l2) in _all_small_lattices(40):
        sh = La.shearfind(L, a, M, l1, l2)
        assert La.sheared_is_separable(L, a, M, l1, l2, sh), (L, a, M, l1, l2, sh)
        count += 1
    assert count > 500


def test_shearfind_prefers_time_shear_exactly_when_possible():
    """Prop. noshearlength: s0 = 0 is possible iff a | s + k b for some k; lengths
    n L_min c/c1 are always of that kind."""
    for (L, a, M, l1, l2) in _all_small_lattices(96):
        sh = La.shearfind(L, a, M, l1, l2)
        lat = La.Lattice(L, a, M, l1, l2)
        possible = any((lat.s + k * lat.b) % a == 0 for k in range(M))
        assert (not sh.freq_shear) == possible
        if L % (La.min_length(a, M, l2) * La.noshear_length_factor(a, M, l1, l2)) == 0:
            assert not sh.freq_shear


def test_workload_lattices():
    """The five workload lattices: feasibility and the shear branch used."""
    expect = {
        (1440, 16, 48, 1, 2): (True, 16, 0, 15),
        (1 << 20, 128, 1024, 1, 2): (False, 0, (1 << 20) - 4, 1024),
        (172800, 60, 720, 1, 3): (True, 6, 0, 80),
        (1 << 18, 256, 2048, 1, 2): (True, 4, 0, 64),
    }
    for (L, a, M, l1, l2), (fs, s0, s1, br) in expect.items():
        sh = La.shearfind(L, a, M, l1, l2)
        assert (sh.freq_shear, sh.s0, sh.s1, sh.b_r) == (fs, s0, s1, br)
    # lambda2 = 3 is never legal for power-of-two lengths (serving stream redraws it)
    for L in (16384, 65536, 262144, 1048576):
        for a in (L // 1024, L // 512):
            assert not La.feasible(L, a, 8 * a, 1, 3)
            assert La.feasible(L, a, 8 * a, 1, 2) and La.feasible(L, a, 8 * a, 1, 4)


def test_alg1_constants_integral():
    for (L, a, M, l1, l2) in _all_small_lattices(72):
        sh = La.shearfind(L, a, M, l1, l2)
        if sh.freq_shear:
            K = La.alg1_constants(L, a, M, sh)
            assert K["ar"] * sh.b_r == a * (L // M)
            assert K["Mr"] * sh.b_r == L and K["Nr"] * K["ar"] == L
