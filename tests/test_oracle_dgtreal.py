"""Oracle pins for the real-signal DGT: the conjugate symmetry of the full coefficients of a
real signal and window (against the direct sum), the stored channels, reconstruction from
them with the canonical dual, and the refusal outside lambda2 <= 2."""
import numpy as np
import pytest

from oracle import dgt as D
from oracle import dgtreal as R
from oracle import duals as U

CASES = [(96, 4, 8, 0, 1), (96, 4, 8, 1, 2), (144, 6, 12, 1, 2), (256, 8, 16, 1, 2)]


@pytest.mark.parametrize("case", CASES)
def test_symmetry_of_real_coefficients(case):
    L, a, M, l1, l2 = case
    rng = np.random.default_rng(L + M)
    f, g = rng.standard_normal(L), rng.standard_normal(L)
    c = D.dgt_direct(f, g, a, M, l1, l2)
    m = np.arange(M)[:, None]
    n = np.arange(L // a)[None, :]
    assert np.allclose(np.conj(c), c[R.partner(m, n, M, l1, l2), n], atol=1e-12 * np.abs(c).max())
    ch = R.dgtreal(f, g, a, M, l1, l2)
    assert ch.shape == (M // 2 + 1, L // a)
    assert np.abs(ch - c[:M // 2 + 1]).max() <= 1e-12 * np.abs(c).max()
    assert np.abs(R.expand(ch, a, M, l1, l2) - c).max() <= 1e-12 * np.abs(c).max()


@pytest.mark.parametrize("case", CASES)
def test_real_reconstruction(case):
    L, a, M, l1, l2 = case
    rng = np.random.default_rng(3 * L + M)
    f = rng.standard_normal(L)
    g = np.exp(-np.pi * ((np.arange(L) + L // 2) % L - L // 2) ** 2 / (L / 4))
    gam = U.zak_gram_dual(g, a, M, l1, l2).real
    fr = R.idgtreal(R.dgtreal(f, g, a, M, l1, l2), gam, a, M, l1, l2)
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) <= 1e-12


def test_refused_outside_the_symmetry():
    with pytest.raises(ValueError):
        R.dgtreal(np.zeros(72), np.zeros(72), 2, 12, 1, 3)
    # lambda2 = 3: the symmetry maps channels to non-integer offsets, so it fails
    L, a, M = 72, 2, 12
    rng = np.random.default_rng(1)
    c = D.dgt_direct(rng.standard_normal(L), rng.standard_normal(L), a, M, 1, 3)
    n = np.arange(L // a)
    assert not np.allclose(np.conj(c[1]), c[(-1) % M], atol=1e-6)
