"""Gradients of the log-magnitude loss through the DGT (float64; test infrastructure only).

Loss  l(f, g) = sum_{m,n} log(|c(m,n)|^2 + eps),  c = C_g f  (eq. DGT).

With u = c / (|c|^2 + eps), dl = 2 Re sum u* dc.  Hence (gradients in the
convention d/dRe + i d/dIm, which is also PyTorch's for complex leaves):

  signal:  grad_f = 2 C_g^* u                 (C_g^* = synthesis with window g)
           real f: 2 Re(C_g^* u)
  window:  grad_g(j) = 2 sum_n f(j + a n) conj(U_n(j + a n)),
           U_n(l) = sum_m u(m, n) exp(+2 pi i l (m + w(n)) / M)
           real g: the real part.

Not in the paper (the paper has no differentiation); derived from eq. (DGT)
and pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

from .dgt import _cexp, dgt_fold, idgt_fold
from .lattice import Lattice


def loss(f, g, a, M, lam1, lam2, eps=1e-6) -> float:
    c = dgt_fold(f, g, a, M, lam1, lam2)
    return float(np.sum(np.log(np.abs(c) ** 2 + eps)))


def grads(f, g, a, M, lam1, lam2, eps=1e-6, coefs=None):
    """Return (loss, grad_f, grad_g) for one signal.  ``coefs`` (shape (M, N)) stands in for
    c = C_g f in every later step (to measure how the gradients respond to an error in c)."""
    f = np.asarray(f)
    g = np.asarray(g)
    L = f.shape[0]
    lat = Lattice(L, a, M, lam1, lam2)
    c = dgt_fold(f, g, a, M, lam1, lam2) if coefs is None else np.asarray(coefs, dtype=np.complex128)
    u = c / (np.abs(c) ** 2 + eps)
    lval = float(np.sum(np.log(np.abs(c) ** 2 + eps)))
    v = idgt_fold(u, g, a, M, lam1, lam2)
    gf = 2 * v.real if np.isrealobj(f) else 2 * v
    l = np.arange(L, dtype=np.int64)
    wsum = np.zeros(L, dtype=np.complex128)
    fc = np.asarray(f, dtype=np.complex128)
    for n in range(lat.N):
        Un = np.tile(np.fft.ifft(u[:, n]) * M, L // M) * _cexp(l * lat.freq_offset_num(n), lam2 * M, sign=+1.0)
        # term(j) = f(j + a n) conj(U_n(j + a n)), j = l - a n
        wsum += np.roll(fc * np.conj(Un), -a * n)
    gg = 2 * wsum.real if np.isrealobj(g) else 2 * wsum
    return lval, gf, gg
