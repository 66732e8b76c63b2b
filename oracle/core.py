"""FP64 oracle: Doppler resampling and FFT ionospheric correction.

TEST INFRASTRUCTURE (see the package docstring): plain numpy, float64 and
complex128 throughout, written for a reader to check against the paper by eye.
No blocking, fusion or reordering beyond what each definition states; library
primitives used as single steps are ``numpy.fft`` (the DFT), ``numpy.sin``,
``numpy.exp`` and ``@`` (a matrix product).

Notation follows the paper: ``x`` sampled pulse, ``fs`` sample rate, ``fc``
carrier, ``v_r`` range rate (positive when approaching), ``alpha`` the
two-way relativistic factor, ``E`` total electron content, ``K2 = kappa*E``.
"""

from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Physical constants (SI).  CODATA 2018: e and c are exact by definition, m_e
# and eps0 are the recommended values.
C_LIGHT = 299792458.0
E_CHARGE = 1.602176634e-19
M_ELECTRON = 9.1093837015e-31
EPS0 = 8.8541878128e-12
# Eq. 3: tau(f) = e^2 E / (8 pi^2 m_e eps0 c f^2) = K2 / (c f^2), so
# K2 = kappa * E with kappa = e^2 / (8 pi^2 m_e eps0)  (= 40.308193... m^3/s^2).
KAPPA = E_CHARGE ** 2 / (8.0 * np.pi ** 2 * M_ELECTRON * EPS0)
# One TEC unit is 1e16 electrons per square metre.
TECU = 1.0e16


# ---------------------------------------------------------------------------
# Doppler factor.

def alpha(v_r: float) -> float:
    """Eq. 1: alpha = (1 + v_r/c) / (1 - v_r/c), v_r > 0 approaching."""
    b = v_r / C_LIGHT
    return (1.0 + b) / (1.0 - b)


def alpha_minus_one(v_r: float) -> float:
    """alpha - 1 = (2 v_r/c) / (1 - v_r/c): Eq. 1 rearranged, no cancellation."""
    b = v_r / C_LIGHT
    return (2.0 * b) / (1.0 - b)


# ---------------------------------------------------------------------------
# Kaiser-windowed sinc kernel for windowed Whittaker-Shannon interpolation
# (Sec. I method list, Sec. III-A Table I "Windowed Whittaker-Shannon").  The
# paper leaves the taper open; the kernel here is the Kaiser window of half
# width R = taps/2 and shape beta.

def i0(x):
    """Modified Bessel function of the first kind, order 0, by its power
    series I0(x) = sum_k ((x/2)^2)^k / (k!)^2, summed until a term falls below
    1e-17 of the partial sum (all terms are positive)."""
    x = np.asarray(x, dtype=np.float64)
    q = 0.25 * x * x
    term = np.ones_like(x)
    total = np.ones_like(x)
    k = 1
    while True:
        term = term * q / float(k * k)
        total = total + term
        if np.all(term <= 1e-17 * total):
            return total
        k += 1


def kaiser(u, half_width: float, beta: float):
    """Kaiser window w(u) = I0(beta*sqrt(1-(u/R)^2)) / I0(beta) on |u| <= R,
    zero outside."""
    u = np.asarray(u, dtype=np.float64)
    r = u / half_width
    inside = np.abs(r) <= 1.0
    arg = beta * np.sqrt(np.maximum(0.0, 1.0 - r * r))
    return np.where(inside, i0(arg) / i0(np.float64(beta)), 0.0)


def kernel_windowed(u, taps: int = 32, beta: float = 8.0):
    """h(u) = sinc(u) * w(u): the windowed interpolation kernel, with
    sinc(u) = sin(pi u)/(pi u) (Eq. 17) and w the Kaiser window of half width
    taps/2.  h vanishes for |u| >= taps/2."""
    u = np.asarray(u, dtype=np.float64)
    return np.sinc(u) * kaiser(u, taps / 2.0, beta)


# ---------------------------------------------------------------------------
# Resampling y[n] = x(alpha * n * Ts)  (Eq. 2), positions in units of Ts.

def _as_pulses(x):
    x = np.asarray(x, dtype=np.complex128)
    return x, x.ndim == 1


def resample_windowed(x, a: float, n_out: int | None = None,
                      taps: int = 32, beta: float = 8.0):
    """Windowed Whittaker-Shannon interpolation (Eq. 17 truncated to the
    kernel support, Table I row 2, Algorithm 1's per-output sum).

        y[n] = sum_i x[i] * h(t_n - i),   t_n = a * n,

    with h the Kaiser-windowed sinc of half width R = taps/2 and x[i] = 0
    outside [0, N).  h is zero for |t - i| >= R, so with m = floor(t_n) and
    frac = t_n - m the sum runs over i = m + j, j = -R+1 .. R.

    sin(pi (frac - j)) is written (-1)^j sin(pi frac) -- the same number -- so
    that an integer position gives exact zeros off the centre tap.
    ``x`` is one pulse (N,) or a stack (P, N); the output has n_out samples
    (default N) per pulse."""
    if taps % 2 or taps < 2:
        raise ValueError("taps must be even and >= 2")
    x, single = _as_pulses(x)
    xs = x[None, :] if single else x
    n_in = xs.shape[1]
    n_out = n_in if n_out is None else int(n_out)
    half = taps // 2
    n = np.arange(n_out, dtype=np.float64)
    t = a * n
    m = np.floor(t)
    frac = t - m
    m = m.astype(np.int64)
    s = np.sin(np.pi * frac)
    y = np.zeros((xs.shape[0], n_out), dtype=np.complex128)
    for j in range(-half + 1, half + 1):
        u = frac - j
        sign = 1.0 if j % 2 == 0 else -1.0
        with np.errstate(divide="ignore", invalid="ignore"):
            sinc = np.where(u == 0.0, 1.0, sign * s / (np.pi * u))
        h = sinc * kaiser(u, float(half), beta)
        idx = m + j
        valid = (idx >= 0) & (idx < n_in)
        xv = np.where(valid[None, :], xs[:, np.clip(idx, 0, n_in - 1)], 0.0)
        y += xv * h[None, :]
    return y[0] if single else y


def _exact_sinc_rows(t, n_in):
    """Rows S[r, m] = sinc(t_r - m), m = 0..n_in-1 (Eq. 17 kernel).
    sin(pi (t - m)) is written (-1)^m sin(pi t) with sin(pi t) taken from the
    fractional part of t, exact at integer t."""
    fl = np.floor(t)
    fr = t - fl
    s = np.sin(np.pi * fr) * (1.0 - 2.0 * np.mod(fl, 2.0))      # sin(pi t)
    mm = np.arange(n_in, dtype=np.float64)
    sign = 1.0 - 2.0 * np.mod(mm, 2.0)                           # (-1)^m
    u = t[:, None] - mm[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        S = np.where(u == 0.0, 1.0, sign[None, :] * s[:, None] / (np.pi * u))
    return S


def resample_exact(x, a: float, n_out: int | None = None, block: int = 512):
    """Exact Whittaker-Shannon interpolation (Eq. 17, Table I row 1) over the
    N available samples:  y[n] = sum_{m=0}^{N-1} x[m] sinc(a n - m).
    ``x`` is (N,) or (P, N); rows of S are built ``block`` at a time."""
    x, single = _as_pulses(x)
    xs = x[None, :] if single else x
    n_in = xs.shape[1]
    n_out = n_in if n_out is None else int(n_out)
    t_all = a * np.arange(n_out, dtype=np.float64)
    y = np.zeros((xs.shape[0], n_out), dtype=np.complex128)
    for b0 in range(0, n_out, block):
        S = _exact_sinc_rows(t_all[b0:b0 + block], n_in)
        y[:, b0:b0 + block] = xs @ S.T
    return y[0] if single else y


def resample_exact_rows(x, a: float, rows):
    """Selected outputs y[rows] of ``resample_exact`` (same definition), for
    sampled checks of full-size problems."""
    x, single = _as_pulses(x)
    xs = x[None, :] if single else x
    t = a * np.asarray(rows, dtype=np.float64)
    S = _exact_sinc_rows(t, xs.shape[1])
    y = xs @ S.T
    return y[0] if single else y


# ---------------------------------------------------------------------------
# Ionospheric correction (Sec. II-B).

def fft_length(n: int) -> int:
    """Transform length: the smallest power of two >= n (zero padding)."""
    n = int(n)
    if n < 1:
        raise ValueError("n must be >= 1")
    L = 1
    while L < n:
        L *= 2
    return L


def bin_frequencies(L: int, fs: float, fc: float):
    """Absolute frequency of each DFT bin, f_k = fc + fs * kt / L with kt = k
    for k < L/2 and k - L otherwise (bin L/2 is -fs/2).  fc = 0 means the
    samples are taken at RF, so f_k is the RF frequency itself."""
    k = np.arange(L, dtype=np.float64)
    kt = np.where(k < L // 2, k, k - L)
    return fc + fs * kt / L


def iono_phase(L: int, fs: float, fc: float, tec_tecu: float):
    """phi_k = 4 pi K2 / (c f_k), the two-way dispersive phase of Eqs. 15-16
    (K2 = kappa * E, E = tec_tecu * 1e16 el/m^2).  A bin at f_k = 0 gets 0."""
    K2 = KAPPA * tec_tecu * TECU
    f = bin_frequencies(L, fs, fc)
    with np.errstate(divide="ignore"):
        phi = np.where(f != 0.0, 4.0 * np.pi * K2 / (C_LIGHT * f), 0.0)
    return phi


def _iono(y, fs, fc, tec_tecu, sign, L=None):
    y = np.asarray(y, dtype=np.complex128)
    n = y.shape[-1]
    L = fft_length(n) if L is None else int(L)
    Y = np.fft.fft(y, n=L, axis=-1)                  # forward, exp(-2 pi i k n / L)
    Y = Y * np.exp(sign * 1j * iono_phase(L, fs, fc, tec_tecu))
    return np.fft.ifft(Y, axis=-1)[..., :n]          # inverse with 1/L, truncate


def iono_correct(y, fs: float, fc: float, tec_tecu: float, L: int | None = None):
    """Eq. 16: s_trans = F^-1[ F(s_rec) * exp(-4 pi i K2 / (c f)) ].
    The pulse (last axis, n samples) is zero-padded to L (default the next
    power of two >= n) and the inverse transform is truncated back to n."""
    return _iono(y, fs, fc, tec_tecu, -1.0, L)


def iono_distort(s, fs: float, fc: float, tec_tecu: float, L: int | None = None):
    """Eq. 15: s_rec = F^-1[ F(s_trans) * exp(+4 pi i K2 / (c f)) ]."""
    return _iono(s, fs, fc, tec_tecu, +1.0, L)


# ---------------------------------------------------------------------------
# Carrier term of a passband dilation, and frequency conversion.

def carrier_term(n_out: int, delta: float, fs: float, f: float):
    """exp(2 pi i f delta n Ts), n = 0 .. n_out-1, delta = alpha - 1.

    A passband signal x(t) exp(2 pi i fc t) dilated by alpha (Eq. 2) is
    x(alpha t) exp(2 pi i fc alpha t); taken back to baseband about fc it is
    x(alpha t) times this term with f = fc.  The phase f delta n / fs is
    formed in cycles and reduced to [-1/2, 1/2] before the exponential."""
    n = np.arange(int(n_out), dtype=np.float64)
    cyc = f * delta * n / fs
    cyc = cyc - np.round(cyc)
    return np.exp(2j * np.pi * cyc)


def frequency_conversion(x, delta: float, fs: float, f_ref: float, n_out: int | None = None):
    """Frequency conversion (Sec. I method list; Table I): the dilation
    approximated by a tone multiply, y[n] = x[n] exp(2 pi i f_ref delta n Ts)
    with x = 0 beyond its N samples.  Exact for a tone at f_ref (whose
    frequency Eq. 2 scales by alpha); for other frequencies f the tone misses
    (f - f_ref) delta, so for an LFM the error grows with its bandwidth."""
    x, single = _as_pulses(x)
    xs = x[None, :] if single else x
    n_in = xs.shape[1]
    n_out = n_in if n_out is None else int(n_out)
    y = np.zeros((xs.shape[0], n_out), dtype=np.complex128)
    k = min(n_in, n_out)
    y[:, :k] = xs[:, :k]
    y = y * carrier_term(n_out, delta, fs, f_ref)[None, :]
    return y[0] if single else y


def resample(x, fs: float, fc: float, v_r: float, mode: str = "windowed",
             n_out: int | None = None, taps: int = 32, beta: float = 8.0,
             carrier_shift: bool = False, freq_ref: float = 0.0):
    """The Doppler step y[n] = x(alpha n Ts) (Eq. 2) by one of Table I's
    methods -- "windowed" or "exact" Whittaker-Shannon interpolation (Eq. 17)
    or "freqconv" (frequency conversion with reference frequency freq_ref).
    With carrier_shift the samples are baseband about fc and the passband
    dilation's carrier term carrier_term(.., fc) is applied as well (for
    "freqconv": a tone at freq_ref + fc)."""
    dl = alpha_minus_one(v_r)
    if mode == "freqconv":
        f = freq_ref + (fc if carrier_shift else 0.0)
        return frequency_conversion(x, dl, fs, f, n_out)
    a = alpha(v_r)
    if mode == "windowed":
        y = resample_windowed(x, a, n_out, taps, beta)
    elif mode == "exact":
        y = resample_exact(x, a, n_out)
    else:
        raise ValueError(mode)
    if carrier_shift:
        y = y * carrier_term(y.shape[-1], dl, fs, fc)
    return y


# ---------------------------------------------------------------------------
# The corrected pulse: Doppler resampling, then ionospheric correction.

def correct(x, fs: float, fc: float, v_r: float, tec_tecu: float,
            mode: str = "windowed", n_out: int | None = None,
            taps: int = 32, beta: float = 8.0, carrier_shift: bool = False,
            freq_ref: float = 0.0):
    """Resample by alpha(v_r) (Eq. 2 via Eq. 17, or frequency conversion)
    then apply Eq. 16."""
    y = resample(x, fs, fc, v_r, mode, n_out, taps, beta, carrier_shift, freq_ref)
    return iono_correct(y, fs, fc, tec_tecu)


def correct_bank(x, fs: float, fc: float, v_list, tec_list,
                 n_out: int | None = None, taps: int = 32, beta: float = 8.0,
                 mode: str = "windowed", carrier_shift: bool = False, freq_ref: float = 0.0):
    """One pulse corrected for every (v_r, TEC) pair: out[v][tec][n]."""
    x = np.asarray(x, dtype=np.complex128)
    n_out = x.shape[0] if n_out is None else int(n_out)
    out = np.zeros((len(v_list), len(tec_list), n_out), dtype=np.complex128)
    for iv, v in enumerate(v_list):
        y = resample(x, fs, fc, v, mode, n_out, taps, beta, carrier_shift, freq_ref)
        for it, tec in enumerate(tec_list):
            out[iv, it] = iono_correct(y, fs, fc, tec)
    return out
