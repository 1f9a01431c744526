"""Pins for the oracle's gradients (no GPU): central finite differences in float64.

The loss sum log(|c|^2 + 1e-6) is stiff where |c| is small; central differences
with h = 1e-3 carry truncation errors up to ~1e-2 there, so the tight check uses
h = 1e-6 (rounding error ~1e-9 relative) and the h = 1e-3 check runs on the
smooth eps = 1 loss."""
import numpy as np

from oracle import grads as Gr
from workloads import noisy_gaussian_window

L, A, M, L1, L2 = 2048, 16, 128, 1, 2


def _setup():
    f = np.random.default_rng(3).standard_normal(L)
    g = noisy_gaussian_window(L, 3)
    return f, g


def _fd(fun, x, v, h):
    return (fun(x + h * v) - fun(x - h * v)) / (2 * h)


def test_gradients_match_finite_differences_tight():
    f, g = _setup()
    _, gf, gg = Gr.grads(f, g, A, M, L1, L2)
    rng = np.random.default_rng(11)
    lf = lambda x: Gr.loss(x, g, A, M, L1, L2)
    lg = lambda x: Gr.loss(f, x, A, M, L1, L2)
    for _ in range(16):
        v = rng.standard_normal(L)
        v /= np.linalg.norm(v)
        assert abs(_fd(lf, f, v, 1e-6) - gf @ v) <= 1e-5 * abs(gf @ v)
        assert abs(_fd(lg, g, v, 1e-6) - gg @ v) <= 1e-5 * abs(gg @ v)
    for i in rng.integers(0, L, 16):
        e = np.zeros(L)
        e[i] = 1
        assert abs(_fd(lf, f, e, 1e-6) - gf[i]) <= 1e-5 * max(abs(gf[i]), 1e-3)
        assert abs(_fd(lg, g, e, 1e-6) - gg[i]) <= 1e-5 * max(abs(gg[i]), 1e-3)


def test_gradients_smooth_loss_h1e3():
    f, g = _setup()
    eps = 1.0
    _, gf, gg = Gr.grads(f, g, A, M, L1, L2, eps)
    rng = np.random.default_rng(12)
    for _ in range(8):
        v = rng.standard_normal(L)
        v /= np.linalg.norm(v)
        d1 = _fd(lambda x: Gr.loss(x, g, A, M, L1, L2, eps), f, v, 1e-3)
        d2 = _fd(lambda x: Gr.loss(f, x, A, M, L1, L2, eps), g, v, 1e-3)
        assert abs(d1 - gf @ v) <= 1e-5 * abs(gf @ v)
        assert abs(d2 - gg @ v) <= 1e-3 * abs(gg @ v)


def test_complex_signal_gradient():
    """Complex f: gradient 2 C* u in the d/dRe + i d/dIm convention."""
    rng = np.random.default_rng(13)
    f = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    g = noisy_gaussian_window(L, 3)
    _, gf, _ = Gr.grads(f, g, A, M, L1, L2)
    lf = lambda x: Gr.loss(x, g, A, M, L1, L2)
    for _ in range(4):
        v = rng.standard_normal(L)
        v /= np.linalg.norm(v)
        dre = _fd(lf, f, v, 1e-6)
        dim = _fd(lf, f, 1j * v, 1e-6)
        assert abs(dre - gf.real @ v) <= 1e-5 * abs(gf.real @ v)
        assert abs(dim - gf.imag @ v) <= 1e-5 * abs(gf.imag @ v)
