"""Oracle pins for the blockwise (overlap-add) DGT: it must reproduce the full-length DGT with
the FIR window exactly (the direct sum on small lattices, the coset route on larger ones),
its synthesis must be the adjoint, and with the canonical dual taps it must reconstruct."""
import numpy as np
import pytest

from oracle import dgt as D
from oracle import duals as U
from oracle import ola as O
from workloads import hann_taps


def _taps(kind, Lg, seed):
    if kind == "hann":
        t, center = hann_taps(Lg)
        return t / np.linalg.norm(t), center
    rng = np.random.default_rng(seed)
    t = rng.standard_normal(Lg) + 1j * rng.standard_normal(Lg)
    return t / np.linalg.norm(t), 3          # off-centre placement: tap 0 at time -3


def _full(taps, center, L):
    return O.local_window(taps, center, L)


CASES = [
    # L, a, M, lam1, lam2, window kind, Lg, Lb
    (1152, 16, 48, 1, 2, "hann", 48, 192),
    (720, 8, 24, 1, 3, "hann", 20, 144),
    (720, 8, 24, 2, 3, "rand", 17, 144),
    (1024, 8, 16, 1, 4, "rand", 40, 128),     # window longer than M
    (2048, 16, 64, 0, 1, "hann", 64, 256),
]


@pytest.mark.parametrize("case", CASES)
def test_ola_equals_full_length_dgt(case):
    L, a, M, l1, l2, kind, Lg, Lb = case
    taps, center = _taps(kind, Lg, L)
    rng = np.random.default_rng(L + l2)
    f = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    g = _full(taps, center, L)
    ref = D.dgt_coset(f, g, a, M, l1, l2)
    c = O.dgt_ola(f, taps, center, a, M, l1, l2, Lb)
    assert np.linalg.norm(c - ref) / np.linalg.norm(ref) <= 1e-12
    if L <= 1152:
        direct = D.dgt_direct(f, g, a, M, l1, l2)
        assert np.linalg.norm(c - direct) / np.linalg.norm(direct) <= 1e-12


@pytest.mark.parametrize("case", CASES)
def test_ola_synthesis_is_the_adjoint(case):
    L, a, M, l1, l2, kind, Lg, Lb = case
    taps, center = _taps(kind, Lg, L)
    rng = np.random.default_rng(7 * L)
    f = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    u = rng.standard_normal((M, L // a)) + 1j * rng.standard_normal((M, L // a))
    lhs = np.vdot(u, O.dgt_ola(f, taps, center, a, M, l1, l2, Lb))
    rhs = np.vdot(O.idgt_ola(u, taps, center, a, M, l1, l2, Lb), f)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # and it equals the full-length synthesis with the same window
    ref = D.idgt_coset(u, _full(taps, center, L), a, M, l1, l2)
    got = O.idgt_ola(u, taps, center, a, M, l1, l2, Lb)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12


@pytest.mark.parametrize("case", [c for c in CASES if c[6] <= c[2]])
def test_ola_reconstruction_with_the_dual_taps(case):
    L, a, M, l1, l2, kind, Lg, Lb = case
    taps, center = _taps(kind, Lg, L)
    gam = U.fir_dual_diag(_full(taps, center, L), a, M)
    gtaps = gam[(np.arange(Lg) - center) % L]
    rng = np.random.default_rng(3 * L)
    f = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    fr = O.idgt_ola(O.dgt_ola(f, taps, center, a, M, l1, l2, Lb), gtaps, center, a, M, l1, l2, Lb)
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) <= 1e-12


def test_ola_length_and_cost_factor():
    # eq. (OLA-eff): the blocks are transformed at length Lx >= Lb + Lg, a cost factor
    # rho = Lx / Lb >= (Lg + Lb) / Lb; Lx is the next admissible length
    for a, M, l2, Lg, Lb in [(16, 48, 2, 48, 192), (128, 1024, 2, 1024, 16384), (8, 24, 3, 20, 144)]:
        Lx = O.ola_length(a, M, l2, Lg, Lb)
        q = l2 * np.lcm(a, M)
        assert Lx % q == 0 and Lb + Lg <= Lx < Lb + Lg + q
        assert Lx / Lb >= (Lg + Lb) / Lb
    with pytest.raises(ValueError):
        O.dgt_ola(np.zeros(1152), np.ones(48), 24, 16, 48, 1, 2, 100)      # Lb not admissible
