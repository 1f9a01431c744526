"""Two-dimensional DGT on a tensor-product lattice, float64, CPU.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the CPU legs of
bench.py; shares no code with the CUDA path.

Section 3.5 (extension to higher dimensions): with a separable window g1 (x) g2 and a lattice
Lambda1 x Lambda2 (each nonseparable on its own axis), the transform of f(l1, l2) is

    c(m1, n1, m2, n2) = sum_{l1, l2} f(l1, l2) conj(g1(l1 - a1 n1)) conj(g2(l2 - a2 n2))
                        exp(-2 pi i l1 (m1 + w1(n1)) / M1) exp(-2 pi i l2 (m2 + w2(n2)) / M2),

which factors into the one-dimensional transform along l2 followed by the one along l1 (the
paper's per-dimension algorithm).  Coefficient arrays are indexed c[m1, n1, m2, n2].
"""
from __future__ import annotations

import numpy as np

from .dgt import dgt_coset, dgt_direct, idgt_coset
from .lattice import Lattice


def dgt2_direct(f, g1, g2, lat1, lat2) -> np.ndarray:
    """The definition, as a sum over both axes for every coefficient (small sizes only).
    lat = (a, M, lam1, lam2)."""
    f = np.asarray(f, dtype=np.complex128)
    L1, L2 = f.shape
    a1, M1, p1, q1 = lat1
    a2, M2, p2, q2 = lat2
    la1, la2 = Lattice(L1, a1, M1, p1, q1), Lattice(L2, a2, M2, p2, q2)
    N1, N2 = la1.N, la2.N
    l1 = np.arange(L1)
    l2 = np.arange(L2)
    g1 = np.asarray(g1, dtype=np.complex128)
    g2 = np.asarray(g2, dtype=np.complex128)
    c = np.empty((M1, N1, M2, N2), dtype=np.complex128)
    for n1 in range(N1):
        w1 = ((n1 * p1) % q1) / q1
        for m1 in range(M1):
            e1 = np.conj(g1[(l1 - a1 * n1) % L1]) * np.exp(-2j * np.pi * l1 * (m1 + w1) / M1)
            fx = e1 @ f                                     # sum over l1, a function of l2
            for n2 in range(N2):
                w2 = ((n2 * p2) % q2) / q2
                e2 = np.conj(g2[(l2 - a2 * n2) % L2]) * np.exp(-2j * np.pi * l2[None, :] * (np.arange(M2)[:, None] + w2) / M2)
                c[m1, n1, :, n2] = e2 @ fx
    return c


def dgt2(f, g1, g2, lat1, lat2) -> np.ndarray:
    """Per-dimension algorithm: the transform along l2 of every row, then along l1."""
    f = np.asarray(f, dtype=np.complex128)
    L1, L2 = f.shape
    # along l2: rows f[l1, :] -> (M2, N2) each
    r = np.stack([dgt_coset(f[i], g2, *lat2) for i in range(L1)])          # (L1, M2, N2)
    # along l1: columns r[:, m2, n2] -> (M1, N1) each
    M2, N2 = r.shape[1], r.shape[2]
    c = np.empty((lat1[1], L1 // lat1[0], M2, N2), dtype=np.complex128)
    for m2 in range(M2):
        for n2 in range(N2):
            c[:, :, m2, n2] = dgt_coset(r[:, m2, n2], g1, *lat1)
    return c


def idgt2(c, gamma1, gamma2, lat1, lat2) -> np.ndarray:
    """Synthesis with gamma1 (x) gamma2: the adjoint of dgt2 with those windows."""
    c = np.asarray(c, dtype=np.complex128)
    M1, N1, M2, N2 = c.shape
    L1, L2 = N1 * lat1[0], N2 * lat2[0]
    r = np.empty((L1, M2, N2), dtype=np.complex128)
    for m2 in range(M2):
        for n2 in range(N2):
            r[:, m2, n2] = idgt_coset(c[:, :, m2, n2], gamma1, *lat1)
    return np.stack([idgt_coset(r[i], gamma2, *lat2) for i in range(L1)])
