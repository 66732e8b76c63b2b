"""FP64 oracle: LFM predistortion comparators and the SNR-loss metric.

TEST INFRASTRUCTURE (see the package docstring).  These are the waveforms the
paper compares its FFT correction against (Sec. II-A, II-C, Appendix B): an
LFM whose frequency solves the Halpin cubic exactly (CUBIC), the
pseudo-Chebyshev quadratic approximation (POLY, corrected and original
coefficients), and the correlation-peak SNR loss used to compare them.
They pin the sign, the factor 4*pi and kappa of the oracle's Eq. 16.
"""

from __future__ import annotations

import numpy as np

from .core import C_LIGHT, KAPPA, TECU

A_CHEB = np.sqrt(3.0) / 2.0        # a = sqrt(3)/2 (Sec. II-A, after Eq. 8)


def cubic_coefficients(t, f0, B, T, K2):
    """Eq. 4 written as f^3 - P f^2 - Q = 0:
    P = f0 + B t/T - 2 K2 B/(c f0^2 T),  Q = 2 K2 B/(c T)."""
    t = np.asarray(t, dtype=np.float64)
    P = f0 + B * t / T - 2.0 * K2 * B / (C_LIGHT * f0 * f0 * T)
    Q = 2.0 * K2 * B / (C_LIGHT * T)
    return P, Q


def cubic_frequency(t, f0, B, T, K2):
    """Eqs. 11-14: the real root of Eq. 4,
    f = (P - omega - chi/omega)/3, chi = P^2, psi = -2 P^3 - 27 Q,
    omega = cbrt((psi + sqrt(psi^2 - 4 chi^3))/2).
    The radicand equals 108 P^3 Q + 729 Q^2 >= 0 for P, Q >= 0; a negative
    value can only be rounding (it is exactly 0 at Q = 0) and is taken as 0."""
    P, Q = cubic_coefficients(t, f0, B, T, K2)
    chi = P * P
    psi = -2.0 * P ** 3 - 27.0 * Q
    omega = np.cbrt((psi + np.sqrt(np.maximum(psi * psi - 4.0 * chi ** 3, 0.0))) / 2.0)
    return (P - omega - chi / omega) / 3.0


def chebyshev_nodes(f0, B, T, K2, factor=2.0):
    """The three-node data of the pseudo-Chebyshev expansion.

    Node frequencies f1,f2,f3 = f0 + B(1-a)/2, f0 + B/2, f0 + B(1+a)/2.
    With g = factor*K2/c (factor 2: Eqs. 9-10; factor 4: the original
    coefficients of Eqs. 23-24):
      T1 = -aT/2 + g[f2^-2 - f1^-2]                      (Eq. 9 / Eq. 23)
      T3 = +aT/2 + g[f2^-2 - f3^-2]                      (reading, see below)
      T2 = g[2 f2^-2 - f1^-2 - f3^-2]                    (Eq. 10 / Eq. 24)
    T1 and T3 are the transmit times of f1 and f3 relative to that of f2
    under the inverse relation of Eq. 4, t(f) = T(f-f0)/B + g(f0^-2 - f^-2);
    the paper uses T3 in Eqs. 7-8 without printing it, and T3 is the mirror
    of Eq. 9 at the third node (so T2 = T1 + T3)."""
    a = A_CHEB
    f1 = f0 + B * (1.0 - a) / 2.0
    f2 = f0 + B / 2.0
    f3 = f0 + B * (1.0 + a) / 2.0
    g = factor * K2 / C_LIGHT
    T1 = -a * T / 2.0 + g * (f2 ** -2 - f1 ** -2)
    T3 = a * T / 2.0 + g * (f2 ** -2 - f3 ** -2)
    T2 = g * (2.0 * f2 ** -2 - f1 ** -2 - f3 ** -2)
    t2 = T / 2.0 + g * (f0 ** -2 - f2 ** -2)      # transmit time of f2
    return dict(f2=f2, T1=T1, T2=T2, T3=T3, t2=t2)


def chebyshev_coefficients(f0, B, T, K2, factor=2.0):
    """Slope and curvature of the pseudo-Chebyshev quadratic about node 2.

    gamma = (aB/2) T2 / (T1 T3 (T3 - T1))                       (Eq. 8)
    slope = -(aB/2) (T1^2 + T3^2) / (T1 T3 (T3 - T1))           (Eq. 7 reading)
    These are the coefficients of the quadratic through the three nodes
    (T1, -aB/2), (0, 0), (T3, +aB/2) in (time, frequency) relative to node 2.
    Eq. 7 prints the denominator as T1 T2 (T3 - T1); with T2 = T1 + T3 -> 0
    as K2 -> 0 that would diverge instead of reducing to mu0 = B/T (Eq. 6),
    so the interpolating form is taken.  Returns (mu0, delta_mu, gamma)."""
    nd = chebyshev_nodes(f0, B, T, K2, factor)
    a = A_CHEB
    T1, T2, T3 = nd["T1"], nd["T2"], nd["T3"]
    gamma = (a * B / 2.0) * T2 / (T1 * T3 * (T3 - T1))
    slope = -(a * B / 2.0) * (T1 ** 2 + T3 ** 2) / (T1 * T3 * (T3 - T1))
    mu0 = B / T                                                  # Eq. 6
    return mu0, slope - mu0, gamma


def chebyshev_frequency(t, f0, B, T, K2, factor=2.0):
    """Eq. 5 about node 2: f(t) = f2 + (mu0 + dmu)(t - t2) + gamma (t - t2)^2."""
    nd = chebyshev_nodes(f0, B, T, K2, factor)
    mu0, dmu, gamma = chebyshev_coefficients(f0, B, T, K2, factor)
    s = np.asarray(t, dtype=np.float64) - nd["t2"]
    return nd["f2"] + (mu0 + dmu) * s + gamma * s * s


def chebyshev_phase(t, f0, B, T, K2, factor=2.0):
    """phi(t) = 2 pi int_0^t f(t') dt' of ``chebyshev_frequency``, integrated
    in closed form."""
    nd = chebyshev_nodes(f0, B, T, K2, factor)
    mu0, dmu, gamma = chebyshev_coefficients(f0, B, T, K2, factor)
    t = np.asarray(t, dtype=np.float64)
    t2 = nd["t2"]
    s, s0 = t - t2, -t2
    integral = (nd["f2"] * t + (mu0 + dmu) * (s * s - s0 * s0) / 2.0
                + gamma * (s ** 3 - s0 ** 3) / 3.0)
    return 2.0 * np.pi * integral


def trapezoid_phase(f, dt):
    """phi(t) = 2 pi int_0^t f dt' by the trapezoidal rule on a uniform grid
    (Sec. II-A, the CUBIC waveform of Sec. II-C)."""
    f = np.asarray(f, dtype=np.float64)
    phi = np.zeros_like(f)
    phi[1:] = 2.0 * np.pi * np.cumsum(0.5 * (f[1:] + f[:-1]) * dt)
    return phi


def lfm_phase(t, f0, B, T):
    """Undistorted LFM from f0 to f0+B over T: phi = 2 pi (f0 t + B t^2/(2T))."""
    t = np.asarray(t, dtype=np.float64)
    return 2.0 * np.pi * (f0 * t + B * t * t / (2.0 * T))


def correlation_peak(a, b):
    """max over lags of |sum_n a[n] conj(b[n - lag])| (linear correlation by a
    zero-padded FFT)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    n = len(a) + len(b)
    L = 1
    while L < n:
        L *= 2
    r = np.fft.ifft(np.fft.fft(a, L) * np.conj(np.fft.fft(b, L)))
    return float(np.max(np.abs(r)))


def snr_loss_db(a, b):
    """Correlation-peak SNR loss of b against a, relative to the energy of
    both (the LFM autocorrelation peak of Fig. 2): -20 log10(peak/(|a||b|))."""
    peak = correlation_peak(a, b)
    return -20.0 * np.log10(peak / (np.linalg.norm(a) * np.linalg.norm(b)))


def predistorted_lfm(n: int, fs: float, f0: float, B: float, T: float, tec_tecu: float,
                     kind: str = "cubic", f_mix: float = 0.0):
    """The transmit waveforms compared in Sec. II-C, sampled at t_m = m / fs,
    m = 0 .. n-1, as s[m] = exp(i (phi(t_m) - 2 pi f_mix t_m)):

    * "lfm"   -- the undistorted LFM from f0 over B in T (``lfm_phase``);
    * "cubic" -- the frequency solving Eq. 4 (Eqs. 11-14), its phase by the
                 trapezoidal rule (Sec. II-A; the CUBIC waveform of Fig. 2);
    * "poly"  -- the pseudo-Chebyshev expansion, Eqs. 5-10, phase in closed
                 form (POLY);
    * "poly4" -- the same with the original factor-4 coefficients of
                 Appendix B (Eqs. 23-24), the negative control.

    K2 = kappa E with E = tec_tecu TECU.  f_mix mixes the waveform down
    (f_mix = 0: RF samples)."""
    t = np.arange(int(n), dtype=np.float64) / fs
    K2 = KAPPA * tec_tecu * TECU
    if kind == "lfm":
        phi = lfm_phase(t, f0, B, T)
    elif kind == "cubic":
        phi = trapezoid_phase(cubic_frequency(t, f0, B, T, K2), 1.0 / fs)
    elif kind == "poly":
        phi = chebyshev_phase(t, f0, B, T, K2, 2.0)
    elif kind == "poly4":
        phi = chebyshev_phase(t, f0, B, T, K2, 4.0)
    else:
        raise ValueError(kind)
    return np.exp(1j * (phi - 2.0 * np.pi * f_mix * t))
