"""Seeded synthetic waveforms and workload recipes.

This module generates inputs only: it holds none of the correction method's
arithmetic (no resampling, no ionospheric phase).  Both the CUDA library's
tests/benchmark and the FP64 oracle draw their inputs from here, so the two
sides see identical samples.

Waveforms follow the shapes used in the paper's experiments (LFM chirps,
arbitrary band-limited waveforms, tones); workloads follow the five published
configurations: a plain single pulse, a Doppler bank, an uneven batch, a
split-precision exact-sinc bank and a Poisson serving stream.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 20250807


def rng_for(config_index: int, salt: int = 0) -> np.random.Generator:
    """PCG64 generator seeded with SEED_BASE + config index (+ salt)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(config_index) + 1000 * int(salt)))


# ---------------------------------------------------------------------------
# Waveforms (complex128; cast with .astype(np.complex64) for the device).

def lfm(n: int, fs: float, bandwidth: float) -> np.ndarray:
    """Baseband LFM chirp exp(i pi k (t - T/2)^2), k = B/T, T = n/fs: sweeps
    -B/2 .. +B/2 about the carrier."""
    T = n / fs
    k = bandwidth / T
    t = np.arange(n, dtype=np.float64) / fs
    return np.exp(1j * np.pi * k * (t - T / 2.0) ** 2)


def rf_lfm(n: int, fs: float, f0: float, bandwidth: float, T: float) -> np.ndarray:
    """Complex RF samples of an LFM of duration T centred at f0: the phase
    2 pi (f0 - B/2) t + pi (B/T) t^2 at t = i / fs, i < n (the sweep f0 - B/2
    .. f0 + B/2 over T; past T the formula extends)."""
    t = np.arange(n, dtype=np.float64) / fs
    return np.exp(1j * (2 * np.pi * (f0 - bandwidth / 2) * t + np.pi * (bandwidth / T) * t * t))


def bandlimited_noise(n: int, rng: np.random.Generator, frac: float = 0.8) -> np.ndarray:
    """Unit-variance complex Gaussian noise low-passed to |f| <= frac * fs/2:
    draw CN(0,1) samples, zero the DFT bins above the cut-off, transform back
    and rescale to unit mean power."""
    w = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2.0)
    W = np.fft.fft(w)
    nu = np.fft.fftfreq(n)                       # cycles/sample in [-0.5, 0.5)
    W[np.abs(nu) > frac * 0.5] = 0.0
    x = np.fft.ifft(W)
    return x / np.sqrt(np.mean(np.abs(x) ** 2))


def bandlimited_noise_batch(p: int, n: int, rng: np.random.Generator, frac: float = 0.8) -> np.ndarray:
    """p pulses of band-limited noise at once, each by the recipe of
    ``bandlimited_noise`` (rows of one (p, n) draw; complex128)."""
    import os
    import scipy.fft as sfft
    w = np.empty((p, n), dtype=np.complex128)
    w.real = rng.standard_normal((p, n))
    w.imag = rng.standard_normal((p, n))
    w *= 1.0 / np.sqrt(2.0)
    W = sfft.fft(w, axis=-1, workers=os.cpu_count() or 1)
    nu = np.fft.fftfreq(n)
    W[:, np.abs(nu) > frac * 0.5] = 0.0
    x = sfft.ifft(W, axis=-1, workers=os.cpu_count() or 1)
    return x / np.sqrt(np.mean(np.abs(x) ** 2, axis=-1, keepdims=True))


def tone(n: int, f_norm: float) -> np.ndarray:
    """exp(2 pi i f_norm m), f_norm in cycles/sample."""
    return np.exp(2j * np.pi * f_norm * np.arange(n, dtype=np.float64))


def gaussian_tone(n: int, center: float, sigma: float, f_norm: float) -> np.ndarray:
    """Gaussian-envelope tone exp(-(m-c)^2/(2 s^2)) exp(2 pi i f m): band-limited
    and time-limited to double precision when s*(0.5-|f|) and (n/2)/s are large."""
    m = np.arange(n, dtype=np.float64)
    return np.exp(-((m - center) ** 2) / (2.0 * sigma * sigma)) * np.exp(2j * np.pi * f_norm * m)


# ---------------------------------------------------------------------------
# Workload recipes.

@dataclass
class PlainPulse:
    """Config 1: one LFM pulse, N=4096, fs=10 MHz, B=5 MHz, fc=1 GHz,
    v_r=+7.5 km/s, TEC=50 TECU."""
    n: int = 4096
    fs: float = 10e6
    bandwidth: float = 5e6
    fc: float = 1e9
    v_r: float = 7500.0
    tec: float = 50.0

    def pulse(self) -> np.ndarray:
        return lfm(self.n, self.fs, self.bandwidth)


@dataclass
class DopplerBank:
    """Config 2: one band-limited noise pulse (N=65536, fs=20 MHz, fc=1 GHz)
    corrected for n_v range rates U[-8,8] km/s x n_tec TECs U[5,150] TECU."""
    n: int = 65536
    n_v: int = 256
    n_tec: int = 16
    fs: float = 20e6
    fc: float = 1e9
    seed_index: int = 2

    def draw(self):
        rng = rng_for(self.seed_index)
        x = bandlimited_noise(self.n, rng)
        v = rng.uniform(-8000.0, 8000.0, self.n_v)
        tec = rng.uniform(5.0, 150.0, self.n_tec)
        return x, v, tec


@dataclass
class UnevenBatch:
    """Config 3: n_pulses pulses, lengths log-uniform in [n_min, n_max], half
    LFM (B ~ U[1,10] MHz) and half band-limited noise, fs=20 MHz, fc=1 GHz,
    per-pulse v_r ~ U[-8,8] km/s and TEC ~ U[5,150] TECU."""
    n_pulses: int = 4096
    n_min: int = 1024
    n_max: int = 262144
    fs: float = 20e6
    fc: float = 1e9
    seed_index: int = 3

    def lengths(self, rng) -> np.ndarray:
        u = rng.uniform(np.log(self.n_min), np.log(self.n_max), self.n_pulses)
        return np.clip(np.round(np.exp(u)).astype(np.int64), self.n_min, self.n_max)

    def draw(self):
        """Returns (lengths, concatenated complex64 samples, offsets, v, tec)."""
        rng = rng_for(self.seed_index)
        lens = self.lengths(rng)
        kinds = rng.integers(0, 2, self.n_pulses)
        bws = rng.uniform(1e6, 10e6, self.n_pulses)
        v = rng.uniform(-8000.0, 8000.0, self.n_pulses)
        tec = rng.uniform(5.0, 150.0, self.n_pulses)
        offs = np.zeros(self.n_pulses + 1, dtype=np.int64)
        offs[1:] = np.cumsum(lens)
        x = np.empty(int(offs[-1]), dtype=np.complex64)
        for i in range(self.n_pulses):
            n = int(lens[i])
            if kinds[i] == 0:
                s = lfm(n, self.fs, bws[i])
            else:
                s = bandlimited_noise(n, rng)
            x[offs[i]:offs[i + 1]] = s.astype(np.complex64)
        return lens, x, offs[:-1], v, tec


@dataclass
class SplitPrecisionBank:
    """Config 4: exact-sinc resampling as a dense contraction; n_alpha range
    rates U[-8,8] km/s, each applied to n_pulses band-limited noise pulses of
    N=8192 samples at fs=20 MHz."""
    n: int = 8192
    n_alpha: int = 64
    n_pulses: int = 512
    fs: float = 20e6
    seed_index: int = 4

    def draw(self, n_pulses: int | None = None):
        rng = rng_for(self.seed_index)
        v = rng.uniform(-8000.0, 8000.0, self.n_alpha)
        p = self.n_pulses if n_pulses is None else n_pulses
        x = np.stack([bandlimited_noise(self.n, rng) for _ in range(p)])
        return x, v

    def draw_distinct(self):
        """The stated workload: n_pulses distinct pulses per range rate.
        Returns (x complex64 [n_alpha][n_pulses][n], v)."""
        rng = rng_for(self.seed_index, salt=1)
        v = rng.uniform(-8000.0, 8000.0, self.n_alpha)
        x = np.empty((self.n_alpha, self.n_pulses, self.n), dtype=np.complex64)
        for i in range(self.n_alpha):
            x[i] = bandlimited_noise_batch(self.n_pulses, self.n, rng).astype(np.complex64)
        return x, v


@dataclass
class ServingStream:
    """Config 5: Poisson arrivals at `rate` pulses/s for `duration` s, lengths
    log-uniform in [n_min, n_max], mixed LFM/noise, per-request v_r and TEC,
    admitted against an HBM budget."""
    rate: float = 20000.0
    duration: float = 60.0
    n_min: int = 2048
    n_max: int = 1048576
    fs: float = 20e6
    fc: float = 1e9
    budget_bytes: int = 64 << 30
    seed_index: int = 5

    def arrivals(self, rng=None, duration: float | None = None) -> np.ndarray:
        rng = rng_for(self.seed_index) if rng is None else rng
        d = self.duration if duration is None else duration
        gaps = rng.exponential(1.0 / self.rate, int(self.rate * d * 1.2) + 16)
        t = np.cumsum(gaps)
        return t[t < d]

    def request(self, rng, i: int):
        """One request: (samples complex64, v_r, tec)."""
        u = rng.uniform(np.log(self.n_min), np.log(self.n_max))
        n = int(np.clip(round(np.exp(u)), self.n_min, self.n_max))
        if rng.integers(0, 2) == 0:
            s = lfm(n, self.fs, rng.uniform(1e6, 10e6))
        else:
            s = bandlimited_noise(n, rng)
        return s.astype(np.complex64), rng.uniform(-8000.0, 8000.0), rng.uniform(5.0, 150.0)
