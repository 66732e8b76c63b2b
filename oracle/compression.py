"""FP64 oracle: pulse compression bundled with the FFT ionospheric correction.

TEST INFRASTRUCTURE (see the package docstring).  Sec. II-B (the paragraph
after Eq. 16 and the figure of the pulse-compression path) proposes running
the correction inside the frequency-domain pass that pulse compression
(matched filtering against the transmitted replica) already makes: forward
DFT, multiply by exp(-i phi_k) of Eq. 16 and by the conjugate spectrum of the
replica, inverse DFT.  The result is the cross-correlation of the corrected
pulse with the replica; this module states it that way, in the time domain,
so that it shares nothing with the frequency-domain product it checks.
"""

from __future__ import annotations

import numpy as np

from .core import fft_length, iono_correct, resample


def corrected_buffer(x, fs: float, fc: float, v_r: float, tec_tecu: float,
                     mode: str = "windowed", taps: int = 32, beta: float = 8.0,
                     carrier_shift: bool = False, freq_ref: float = 0.0, n_out: int | None = None):
    """The whole corrected L-buffer of Eq. 16 before truncation: the pulse
    resampled by alpha(v_r) (Eq. 2), zero-padded to L = the next power of two
    of its length, transformed, multiplied by exp(-i phi_k) and transformed
    back (all L samples kept: the dispersion may carry energy past the
    pulse's samples).  n_out: samples of the resampled pulse (default n)."""
    y = resample(x, fs, fc, v_r, mode, n_out, taps, beta, carrier_shift, freq_ref)
    n = y.shape[-1]
    L = fft_length(n)
    yp = np.zeros(L, dtype=np.complex128)
    yp[:n] = y
    return iono_correct(yp, fs, fc, tec_tecu)          # n = L: nothing truncated


def cross_correlate(z, h, lags):
    """r[m] = sum_j z[(m + j) mod L] conj(h[j]) for each lag m (an int n means
    lags 0 .. n-1): the circular cross-correlation of the L-periodic buffer z
    with the replica h (len(h) <= L), written as the matched filter's sum over
    the replica."""
    z = np.asarray(z, dtype=np.complex128)
    h = np.asarray(h, dtype=np.complex128)
    L = z.shape[-1]
    if h.shape[-1] > L:
        raise ValueError("replica longer than the transform")
    lags = np.arange(int(lags)) if np.ndim(lags) == 0 else np.asarray(lags, dtype=np.int64)
    r = np.zeros(lags.shape[0], dtype=np.complex128)
    idx = np.arange(h.shape[-1])
    hc = np.conj(h)
    for i, m in enumerate(lags):
        r[i] = np.sum(z[(m + idx) % L] * hc)
    return r


def correct_compress(x, replica, fs: float, fc: float, v_r: float, tec_tecu: float,
                     mode: str = "windowed", taps: int = 32, beta: float = 8.0,
                     carrier_shift: bool = False, freq_ref: float = 0.0, n_out: int | None = None,
                     lags=None):
    """Pulse compression with the ionospheric correction (Sec. II-B): the
    matched-filter output of the resampled, corrected pulse against the
    replica at the given lags (default 0 .. n_out-1, n_out the resampled
    pulse's samples, default its input's n).  Lag
    m is the replica's inner product with the corrected buffer starting at
    sample m; lags up to L - len(replica) are the linear correlation (the
    buffer is zero-padded), later ones wrap around the L-buffer, as the DFT
    product does."""
    z = corrected_buffer(x, fs, fc, v_r, tec_tecu, mode, taps, beta, carrier_shift, freq_ref, n_out)
    if lags is None:
        lags = np.asarray(x).shape[-1] if n_out is None else int(n_out)
    return cross_correlate(z, replica, lags)


def correct_compress_bank(x, replica, fs: float, fc: float, v_list, tec_list, mode: str = "windowed",
                          carrier_shift: bool = False, freq_ref: float = 0.0):
    """correct_compress for every (v_r, TEC) pair: out[v][tec][lag]."""
    n = np.asarray(x).shape[-1]
    out = np.zeros((len(v_list), len(tec_list), n), dtype=np.complex128)
    for i, v in enumerate(v_list):
        for t, tec in enumerate(tec_list):
            out[i, t] = correct_compress(x, replica, fs, fc, v, tec, mode,
                                         carrier_shift=carrier_shift, freq_ref=freq_ref)
    return out
