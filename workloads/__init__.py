"""Seeded synthetic inputs for the nonseparable-lattice DGT workloads.

This module is the only code shared by the CUDA path's tests/bench and the
CPU oracle.  It produces signals and windows (the *inputs* of the transform)
and the lattice parameter sets of the five workloads; it contains none of the
transform's arithmetic.  Every generator is deterministic in its seed
(``numpy.random.default_rng``), returns float64 / complex128 numpy arrays, and
the caller rounds to float32 where a single-precision run is wanted.

Windows
-------
* ``gaussian_window(L)`` -- periodised Gaussian of width sqrt(L),
  g(l) = sum_k exp(-pi (l + kL)^2 / L) with l taken in (-L/2, L/2], l2-normalised.
* ``hann_window(L, Lg)`` -- zero-centred periodic Hann of length Lg,
  h(x) = 0.5 + 0.5 cos(2 pi x / Lg) for x in [-Lg/2, Lg/2), placed at index
  x mod L, l2-normalised.  ``hann_taps(Lg)`` returns the same taps as a short
  array together with the index of tap x = 0.

Signals
-------
* ``complex_normal(L, seed)`` -- re and im i.i.d. N(0, 1).
* ``real_normal(L, seed)`` -- i.i.d. N(0, 1).
* ``pink_noise(L, seed)`` -- white N(0,1) shaped to a 1/f power spectrum
  (rfft bins k >= 1 scaled by k^-1/2, DC removed), unit RMS.
* ``linear_chirp(L, seed, noise_db=-60)`` -- exp(i pi (l^2 mod 4L) / (2L)),
  instantaneous frequency sweeping 0 -> L/2 bins, plus complex white noise of
  total power 10^(noise_db/10).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(*key) -> np.random.Generator:
    return np.random.default_rng([int(k) for k in key])


# ----------------------------------------------------------------------------
# windows
# ----------------------------------------------------------------------------
def gaussian_window(L: int, periods: int = 4) -> np.ndarray:
    """Periodised Gaussian of width sqrt(L) (time-frequency symmetric), ||g||_2 = 1."""
    l = np.arange(L, dtype=np.int64)
    lc = np.where(l > L // 2, l - L, l).astype(np.float64)
    g = np.zeros(L)
    for k in range(-periods, periods + 1):
        g += np.exp(-math.pi * (lc + k * L) ** 2 / L)
    return g / np.linalg.norm(g)


def hann_taps(Lg: int) -> tuple[np.ndarray, int]:
    """Zero-centred periodic Hann taps for x = -Lg/2 .. Lg/2-1 (unnormalised),
    and the index of the tap at x = 0.  Lg must be even."""
    if Lg % 2:
        raise ValueError("Hann length must be even")
    x = np.arange(-Lg // 2, Lg // 2, dtype=np.float64)
    h = 0.5 + 0.5 * np.cos(2 * math.pi * x / Lg)
    return h, Lg // 2


def hann_window(L: int, Lg: int) -> np.ndarray:
    """Full-length array of the zero-centred Hann FIR window of length Lg, ||h||_2 = 1."""
    h, center = hann_taps(Lg)
    g = np.zeros(L)
    idx = (np.arange(Lg) - center) % L
    g[idx] = h
    return g / np.linalg.norm(g)


def noisy_gaussian_window(L: int, seed: int, rel: float = 0.01) -> np.ndarray:
    """Gaussian window plus rel * N(0,1) white noise (a learnable-window initialisation)."""
    g = gaussian_window(L)
    return g + rel * _rng(seed, 10**6).standard_normal(L)


# ----------------------------------------------------------------------------
# signals
# ----------------------------------------------------------------------------
def complex_normal(L: int, *seed) -> np.ndarray:
    r = _rng(*seed)
    return r.standard_normal(L) + 1j * r.standard_normal(L)


def real_normal(L: int, *seed) -> np.ndarray:
    return _rng(*seed).standard_normal(L)


def pink_noise(L: int, *seed) -> np.ndarray:
    x = _rng(*seed).standard_normal(L)
    X = np.fft.rfft(x)
    k = np.arange(X.shape[0], dtype=np.float64)
    scale = np.zeros_like(k)
    scale[1:] = k[1:] ** -0.5
    y = np.fft.irfft(X * scale, n=L)
    return y / np.sqrt(np.mean(y * y))


def linear_chirp(L: int, *seed, noise_db: float = -60.0) -> np.ndarray:
    l = np.arange(L, dtype=np.int64)
    ph = (l * l) % (4 * L)                       # exact integer reduction of l^2
    s = np.exp(1j * math.pi * ph.astype(np.float64) / (2 * L))
    r = _rng(*seed)
    sigma = math.sqrt(10 ** (noise_db / 10) / 2)
    return s + sigma * (r.standard_normal(L) + 1j * r.standard_normal(L))


# ----------------------------------------------------------------------------
# the five workloads (lattice parameters and batch recipes)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    a: int
    M: int
    lam1: int
    lam2: int
    batch: int
    real_signal: bool
    windows: tuple = field(default=("gauss",))

    @property
    def N(self) -> int:
        return self.L // self.a

    @property
    def b(self) -> int:
        return self.L // self.M

    @property
    def coefs(self) -> int:
        return self.M * self.N


QUINCUNX_FP64 = Workload("quincunx-L1440-a16-M48", 1440, 16, 48, 1, 2, 1, False, ("gauss",))
AUDIO_BATCH = Workload("audio-L1048576-a128-M1024-quincunx-b64", 1 << 20, 128, 1024, 1, 2, 64, True,
                       ("hann1024", "gauss"))
DENSE_THIRD = Workload("L172800-a60-M720-lambda1_3-b128", 172800, 60, 720, 1, 3, 128, False,
                       ("gauss", "gauss_tight"))
DIFFERENTIABLE = Workload("diff-L262144-a256-M2048-quincunx-b32", 1 << 18, 256, 2048, 1, 2, 32, True,
                          ("gauss_noisy",))
DIFF_SUBCASE = Workload("diff-sub-L2048-a16-M128-quincunx", 2048, 16, 128, 1, 2, 4, True, ("gauss_noisy",))

WORKLOADS = {w.name: w for w in (QUINCUNX_FP64, AUDIO_BATCH, DENSE_THIRD, DIFFERENTIABLE, DIFF_SUBCASE)}


def window_for(L: int, kind: str, seed: int = 0) -> np.ndarray:
    """Full-length float64 window of the given kind."""
    if kind in ("gauss", "gauss_tight"):
        return gaussian_window(L)
    if kind.startswith("hann"):
        return hann_window(L, int(kind[4:]))
    if kind == "gauss_noisy":
        return noisy_gaussian_window(L, seed)
    raise ValueError(kind)


def signal_batch(w: Workload, count: int | None = None, cfg_id: int = 0, start: int = 0) -> np.ndarray:
    """Batch of `count` signals (default: the whole batch) of workload `w`, [B][L]."""
    B = w.batch if count is None else count
    out = np.empty((B, w.L), dtype=np.float64 if w.real_signal else np.complex128)
    for i in range(B):
        idx = start + i
        if w is AUDIO_BATCH:
            out[i] = pink_noise(w.L, cfg_id, idx)
        elif w is DENSE_THIRD:
            out[i] = complex_normal(w.L, cfg_id, idx) if idx < w.batch // 2 else linear_chirp(w.L, cfg_id, idx)
        elif w.real_signal:
            out[i] = real_normal(w.L, cfg_id, idx)
        else:
            out[i] = complex_normal(w.L, cfg_id, idx)
    return out


# ----------------------------------------------------------------------------
# serving-loop request stream (Poisson arrivals over the four lengths)
# ----------------------------------------------------------------------------
SERVE_LENGTHS = (16384, 65536, 262144, 1048576)


@dataclass(frozen=True)
class Request:
    t_arrival: float
    L: int
    a: int
    M: int
    lam1: int
    lam2: int
    window: str
    kind: str          # "dgt" or "idgt"
    feasible: bool
    redraws: int


def serve_requests(rate: float, seconds: float, seed: int = 4, infeasible_every: int = 0) -> list[Request]:
    """Poisson request stream: L uniform on SERVE_LENGTHS, a in {L/1024, L/512},
    M = 8a, lambda2 drawn from {1,2,3,4} (lambda1 = 1, or 0 when lambda2 = 1) and
    redrawn while L is not divisible by lambda2 * lcm(a, M).  Every
    `infeasible_every`-th request (if > 0) keeps an infeasible lambda2 = 3 on purpose."""
    r = _rng(seed, 2000)
    t = 0.0
    out = []
    i = 0
    while True:
        t += r.exponential(1.0 / rate)
        if t >= seconds:
            break
        L = int(r.choice(SERVE_LENGTHS))
        a = L // int(r.choice((1024, 512)))
        M = 8 * a
        lcm = a * M // math.gcd(a, M)
        redraws = 0
        lam2 = int(r.choice((1, 2, 3, 4)))
        force_bad = infeasible_every > 0 and i % infeasible_every == infeasible_every - 1
        if force_bad:
            lam2 = 3
        else:
            while L % (lam2 * lcm):
                lam2 = int(r.choice((1, 2, 3, 4)))
                redraws += 1
        lam1 = 0 if lam2 == 1 else 1
        window = "gauss" if r.random() < 0.5 else "hann%d" % M
        kind = "dgt" if r.random() < 0.7 else "idgt"
        out.append(Request(t, L, a, M, lam1, lam2, window, kind, L % (lam2 * lcm) == 0, redraws))
        i += 1
    return out
