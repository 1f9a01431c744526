"""Oracle pins for the two-dimensional tensor-product DGT: the per-dimension algorithm equals
the two-dimensional definition, its synthesis is the adjoint, and the tensor product of the
one-dimensional canonical duals reconstructs."""
import numpy as np
import pytest

from oracle import dgt2 as T
from oracle import duals as U

CASES = [
    # (L1, (a1, M1, lam1, lam2)), (L2, (a2, M2, lam1, lam2))
    ((24, (4, 6, 1, 2)), (36, (6, 6, 1, 3))),
    ((12, (2, 6, 1, 2)), (16, (2, 4, 0, 1))),
]


def _win(L, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(L) + 1j * rng.standard_normal(L)


@pytest.mark.parametrize("case", CASES)
def test_per_dimension_equals_definition(case):
    (L1, lat1), (L2, lat2) = case
    rng = np.random.default_rng(L1 * L2)
    f = rng.standard_normal((L1, L2)) + 1j * rng.standard_normal((L1, L2))
    g1, g2 = _win(L1, 1), _win(L2, 2)
    ref = T.dgt2_direct(f, g1, g2, lat1, lat2)
    got = T.dgt2(f, g1, g2, lat1, lat2)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12


@pytest.mark.parametrize("case", CASES)
def test_adjoint_and_reconstruction(case):
    (L1, lat1), (L2, lat2) = case
    rng = np.random.default_rng(L1 + L2)
    f = rng.standard_normal((L1, L2)) + 1j * rng.standard_normal((L1, L2))
    g1, g2 = _win(L1, 3), _win(L2, 4)
    c = T.dgt2(f, g1, g2, lat1, lat2)
    u = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
    assert abs(np.vdot(u, c) - np.vdot(T.idgt2(u, g1, g2, lat1, lat2), f)) <= 1e-12 * abs(np.vdot(u, c))
    d1 = U.dense_dual(g1, *lat1)
    d2 = U.dense_dual(g2, *lat2)
    fr = T.idgt2(c, d1, d2, lat1, lat2)
    assert np.linalg.norm(fr - f) / np.linalg.norm(f) <= 1e-10
