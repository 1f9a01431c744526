"""Real-signal DGT (coefficients of the non-negative channels only), float64, CPU.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the CPU legs of
bench.py; shares no code with the CUDA path.

For a real signal f and a real window g, eq. DGT gives
    conj(c(m, n)) = sum_l f(l) g(l - a n) exp(+2 pi i l (m + w(n))/M) = c(-m - 2 w(n), n)
(indices modulo M).  With lambda2 <= 2, 2 w(n) = (n lambda1) mod lambda2 is an integer, so
every channel is the conjugate of a channel at most M/2 ... the channels 0..M/2 (M even)
determine c.  This is the real-signal variant of the library interface the paper uses
(LTFAT's dgtreal, Section 4.4); the symmetry holds for lambda2 <= 2 only.
"""
from __future__ import annotations

import numpy as np

from .dgt import dgt_coset, idgt_coset


def _check(M, lam2):
    if lam2 > 2 or M % 2:
        raise ValueError("the real-signal DGT needs lambda2 <= 2 and an even M")


def partner(m, n, M, lam1, lam2):
    """Channel whose conjugate is channel m of column n: (-m - 2 w(n)) mod M."""
    return (-np.asarray(m) - ((np.asarray(n) * lam1) % lam2) * (2 // lam2)) % M


def dgtreal(f, g, a, M, lam1, lam2) -> np.ndarray:
    """Channels 0..M/2 of c (shape (M/2 + 1, N)) for a real f and a real g."""
    _check(M, lam2)
    return dgt_coset(np.asarray(f, dtype=np.float64), np.asarray(g, dtype=np.float64), a, M, lam1, lam2)[:M // 2 + 1]


def expand(ch, a, M, lam1, lam2) -> np.ndarray:
    """The full coefficient array (M, N) from channels 0..M/2 by the symmetry."""
    _check(M, lam2)
    ch = np.asarray(ch, dtype=np.complex128)
    Mh, N = ch.shape
    c = np.empty((M, N), dtype=np.complex128)
    c[:Mh] = ch
    m = np.arange(Mh, M)[:, None]
    n = np.arange(N)[None, :]
    c[Mh:] = np.conj(ch[partner(m, n, M, lam1, lam2), n])
    return c


def idgtreal(ch, gamma, a, M, lam1, lam2) -> np.ndarray:
    """Real synthesis from channels 0..M/2: the real part of the synthesis of the expanded
    coefficients (exactly real when they come from a real signal and window)."""
    return idgt_coset(expand(ch, a, M, lam1, lam2), np.asarray(gamma, dtype=np.float64), a, M, lam1, lam2).real
