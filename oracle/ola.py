"""Blockwise (overlap-add) DGT with an FIR window, float64, CPU.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the CPU legs of
bench.py; shares no code with the CUDA path.

The OLA algorithm (Section 4, and the shear-OLA algorithm of Section 4.1): the signal of
length L = Lb Nb is cut into Nb blocks of Lb samples; every block, zero-extended to a length
Lx >= Lb + Lg (Lg the window support), is transformed with the same lattice and window on
Z_Lx, and the coefficient columns of the short transforms are added into the columns of the
long one.  The cost grows by the factor rho = (Lg + Lb) / Lb of eq. (OLA-eff) (rho = Lx/Lb
here, Lx rounded up to an admissible length).

Column map.  Block beta sits at the start of its buffer (samples 0..Lb-1).  A column nu of
the block's own time axis (global column n = beta Lb / a + nu) sees the block iff its window
support [a nu - center, a nu - center + Lg) meets [0, Lb), i.e. nu_lo <= nu <= nu_hi with
nu_hi = floor((Lb - 1 + center) / a); on Z_Lx such a column is column nu mod Nx (Nx = Lx/a),
and no two of them share a local column because Lx >= Lb + Lg.  Local columns beyond nu_hi
therefore stand for nu - Nx (windows that start before the block).  The lattice phase and
w(n) agree between the two axes because Lb and Lx are multiples of lam2 lcm(a, M).

Synthesis (the adjoint): gather each block's Nx columns from the global coefficients with the
same map, synthesise on Z_Lx, keep the block's Lb samples.
"""
from __future__ import annotations

import numpy as np

from .dgt import dgt_coset, idgt_coset
from .lattice import min_length


def ola_length(a: int, M: int, lam2: int, Lg: int, Lb: int) -> int:
    """Smallest admissible local length Lx >= Lb + Lg (a multiple of lam2 lcm(a, M))."""
    q = min_length(a, M, lam2)
    return -(-(Lb + Lg) // q) * q


def local_window(taps, center: int, Lx: int) -> np.ndarray:
    """Zero-centred FIR taps (tap t at time t - center) as a window on Z_Lx."""
    taps = np.asarray(taps)
    g = np.zeros(Lx, dtype=np.result_type(taps.dtype, np.float64))
    g[(np.arange(taps.shape[0]) - center) % Lx] = taps
    return g


def column_map(beta: int, Lb: int, Lx: int, a: int, center: int, N: int) -> np.ndarray:
    """Global column of every local column of block beta."""
    Nx = Lx // a
    nu = np.arange(Nx, dtype=np.int64)
    nu_hi = (Lb - 1 + center) // a
    nu = np.where(nu <= nu_hi, nu, nu - Nx)
    return (beta * (Lb // a) + nu) % N


def _check(L, a, M, lam2, Lg, Lb, Lx):
    q = min_length(a, M, lam2)
    if L % Lb or Lb % q or Lx % q or Lx < Lb + Lg or Lx > L:
        raise ValueError("OLA needs Lb | L, Lb and Lx multiples of lam2 lcm(a, M), Lb + Lg <= Lx <= L")


def dgt_ola(f, taps, center, a, M, lam1, lam2, Lb, Lx=None) -> np.ndarray:
    """c (shape (M, N)) of f with the FIR window, block by block (OLA)."""
    f = np.asarray(f, dtype=np.complex128)
    L = f.shape[0]
    Lg = np.asarray(taps).shape[0]
    Lx = Lx or ola_length(a, M, lam2, Lg, Lb)
    _check(L, a, M, lam2, Lg, Lb, Lx)
    N = L // a
    gx = local_window(taps, center, Lx)
    c = np.zeros((M, N), dtype=np.complex128)
    for beta in range(L // Lb):
        x = np.zeros(Lx, dtype=np.complex128)
        x[:Lb] = f[beta * Lb:(beta + 1) * Lb]
        c[:, column_map(beta, Lb, Lx, a, center, N)] += dgt_coset(x, gx, a, M, lam1, lam2)
    return c


def idgt_ola(c, taps, center, a, M, lam1, lam2, Lb, Lx=None) -> np.ndarray:
    """Synthesis with the FIR window `taps`: the adjoint of dgt_ola."""
    c = np.asarray(c, dtype=np.complex128)
    M_, N = c.shape
    L = N * a
    Lg = np.asarray(taps).shape[0]
    Lx = Lx or ola_length(a, M, lam2, Lg, Lb)
    _check(L, a, M, lam2, Lg, Lb, Lx)
    gx = local_window(taps, center, Lx)
    f = np.zeros(L, dtype=np.complex128)
    for beta in range(L // Lb):
        cx = c[:, column_map(beta, Lb, Lx, a, center, N)]
        f[beta * Lb:(beta + 1) * Lb] = idgt_coset(cx, gx, a, M, lam1, lam2)[:Lb]
    return f
