"""Pins for the oracle's range-rate factor and resampling (CPU only).

Each check ties the oracle to something other than itself: exact rational
arithmetic, library routines (scipy/numpy Bessel and Kaiser, numpy sinc),
brute-force sums over every input sample, closed forms of band-limited
signals, the paper's printed accuracy (Sec. III-B, Table I) and invariants.
"""

import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import predistortion as pdist
import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


# --------------------------------------------------------------------- alpha

@pytest.mark.parametrize("v", [-8000.0, -1.5, 0.0, 3.0, 7500.0, 1.2e7])
def test_alpha_exact_rational(v):
    b = Fraction(v) / Fraction(oracle.C_LIGHT)
    exact = (1 + b) / (1 - b)
    assert abs(oracle.alpha(v) - float(exact)) <= 1e-15 * float(exact)
    assert abs(oracle.alpha_minus_one(v) - float(exact - 1)) <= 1e-15 * abs(float(exact - 1)) + 1e-300


@pytest.mark.parametrize("v", [1.0, 7500.0, 8000.0, 3e6])
def test_alpha_two_way_invariants(v):
    # Eq. 1 is the two-way relativistic factor: alpha(v) alpha(-v) = 1, alpha(0) = 1,
    # alpha > 1 when approaching, and alpha = 1 + 2b + 2b^2 + O(b^3).
    a, am = oracle.alpha(v), oracle.alpha(-v)
    assert abs(a * am - 1.0) < 1e-15
    assert oracle.alpha(0.0) == 1.0
    assert a > 1.0 > am
    b = v / oracle.C_LIGHT
    assert abs(oracle.alpha_minus_one(v) - (2 * b + 2 * b * b)) <= 4 * abs(b) ** 3 + 1e-300


def test_alpha_config1_value():
    # v_r = +7.5 km/s  ->  alpha - 1 = 5.0036e-5
    assert abs(oracle.alpha_minus_one(7500.0) - 5.00359e-5) < 1e-9


# ------------------------------------------------------------ kaiser kernel

def test_i0_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    x = np.linspace(0.0, 30.0, 301)
    np.testing.assert_allclose(oracle.i0(x), sp.i0(x), rtol=1e-14)
    np.testing.assert_allclose(oracle.i0(x), np.i0(x), rtol=1e-14)


@pytest.mark.parametrize("M,beta", [(33, 8.0), (17, 5.0), (65, 12.0)])
def test_kaiser_matches_numpy_window(M, beta):
    R = (M - 1) / 2.0
    u = np.arange(M) - R
    np.testing.assert_allclose(oracle.kaiser(u, R, beta), np.kaiser(M, beta), rtol=1e-13, atol=1e-16)


def test_kernel_support_and_nodes():
    h = oracle.kernel_windowed
    assert h(0.0) == 1.0
    ints = np.arange(-15, 16)
    ints = ints[ints != 0]
    assert np.max(np.abs(h(ints.astype(float)))) < 1e-15       # sinc zeros
    assert np.all(np.abs(h(np.array([16.0, -16.0]))) < 1e-18)       # sinc(16) w(16)
    assert np.all(h(np.array([16.5, -20.0, 16.0001])) == 0.0)       # outside the support
    u = np.linspace(-15.9, 15.9, 101)
    np.testing.assert_allclose(h(u), h(-u), rtol=0, atol=0)     # even
    np.testing.assert_allclose(oracle.kaiser(np.array([16.0]), 16.0, 8.0),
                               1.0 / oracle.i0(8.0), rtol=1e-15)


# -------------------------------------------------------- windowed resample

def _brute_windowed(x, a, n_out, taps, beta):
    """Every input sample, every output, scalar loops: y[n] = sum_i x[i] h(a n - i)."""
    y = np.zeros(n_out, dtype=np.complex128)
    for n in range(n_out):
        t = a * n
        acc = 0j
        for i in range(len(x)):
            acc += x[i] * float(np.sinc(t - i)) * float(oracle.kaiser(t - i, taps / 2, beta))
        y[n] = acc
    return y


@pytest.mark.parametrize("a,taps,n_out", [(1.37, 8, 30), (0.81, 8, 33), (1.0004, 32, 40), (0.93, 32, 48)])
def test_windowed_matches_brute_force(a, taps, n_out):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(24) + 1j * rng.standard_normal(24)
    y = oracle.resample_windowed(x, a, n_out, taps=taps, beta=8.0)
    ref = _brute_windowed(x, a, n_out, taps, 8.0)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n_out", [4096, 1000, 5000])
def test_windowed_identity_at_alpha_one(n_out):
    x = synth.bandlimited_noise(4096, synth.rng_for(1, salt=3))
    y = oracle.resample_windowed(x, oracle.alpha(0.0), n_out)
    m = min(n_out, 4096)
    assert np.array_equal(y[:m], x[:m])                          # bitwise
    assert np.all(y[m:] == 0)


def test_windowed_gaussian_tone_closed_form():
    # A Gaussian-envelope tone is band- and time-limited to double precision,
    # so its dilation x(a t) is known in closed form at every output.
    n, c, s, f = 512, 256.0, 20.0, 0.15
    a = oracle.alpha(7500.0 * 40)                               # visible dilation
    x = synth.gaussian_tone(n, c, s, f)
    t = a * np.arange(n)
    exact = np.exp(-((t - c) ** 2) / (2 * s * s)) * np.exp(2j * np.pi * f * t)
    y = oracle.resample_windowed(x, a, n)
    assert np.max(np.abs(y - exact)) < 1e-4
    errs = [np.max(np.abs(oracle.resample_windowed(x, a, n, taps=k) - exact)) for k in (4, 8, 16)]
    assert errs[0] > errs[1] > errs[2]                          # Table I: error falls with N_window


def test_windowed_tone_frequency_scales_by_alpha():
    # Eq. 2: x(a t) of a tone at f has frequency a*f.
    n, f = 4096, 0.1
    a = oracle.alpha(7500.0)
    y = oracle.resample_windowed(synth.tone(n, f), a, n)
    exact = synth.tone(n, f * a)
    sl = slice(32, int((n - 1) / a) - 32)
    assert np.max(np.abs(y[sl] - exact[sl])) < 1e-4


def test_windowed_lfm_matches_dilated_analytic():
    # A resampled sampled LFM matches the analytically generated LFM with the
    # dilated slope on interior samples (Sec. I, analytic resampling).
    cfg = synth.PlainPulse()
    x = cfg.pulse()
    a = oracle.alpha(cfg.v_r)
    T = cfg.n / cfg.fs
    k = cfg.bandwidth / T
    t = a * np.arange(cfg.n) / cfg.fs
    analytic = np.exp(1j * np.pi * k * (t - T / 2.0) ** 2)
    y = oracle.resample_windowed(x, a, cfg.n)
    sl = slice(64, int((cfg.n - 1) / a) - 64)
    assert np.max(np.abs(y[sl] - analytic[sl])) < 2e-4


def test_windowed_snr_loss_against_analytic_e5():
    # Sec. III-B: windowed sinc vs analytic resampling of an RF-sampled LFM loses
    # about 1e-4 dB with the paper's LUT kernel; exact evaluation must do no worse.
    g = GOLDEN["E5_fig_sinc_snr_loss"]
    fs, T, fcen, B, v = g["fs_hz"], g["T_s"], g["fc_hz"], g["bandwidth_hz"], g["v_m_s"]
    n = int(round(T * fs))
    t = np.arange(n) / fs
    x = np.exp(1j * pdist.lfm_phase(t, fcen - B / 2, B, T))
    a = oracle.alpha(v)
    nin = int(np.floor((n - 1) / a))
    ref = np.exp(1j * pdist.lfm_phase(a * t[:nin], fcen - B / 2, B, T))
    y = oracle.resample_windowed(x, a, nin, taps=40)
    assert pdist.snr_loss_db(ref, y) <= g["loss_db_about"]


def test_windowed_error_falls_with_taps_table1():
    # Table I: the windowed-sinc error against the exact sum shrinks as the
    # window widens (a trend, not a bound); interior samples of a band-limited
    # pulse, the same pulse and range rate for every tap count.
    rng = np.random.default_rng(21)
    n = 1024
    X = np.fft.fft(rng.standard_normal(n) + 1j * rng.standard_normal(n))
    k = np.fft.fftfreq(n)
    X[np.abs(k) > 0.4] = 0
    x = np.fft.ifft(X)
    a = oracle.alpha(6000.0)
    ref = oracle.resample_exact(x, a, n)
    inner = slice(200, n - 200)
    errs = []
    for taps in (8, 16, 32, 64):
        y = oracle.resample_windowed(x, a, n, taps=taps)
        errs.append(np.linalg.norm(y[inner] - ref[inner]) / np.linalg.norm(ref[inner]))
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:])), errs


# ----------------------------------------------------------- exact resample

def test_exact_matches_numpy_sinc_matrix():
    rng = np.random.default_rng(11)
    x = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    for a, n_out in ((1.01, 80), (0.97, 50), (1.0, 64)):
        S = np.sinc(a * np.arange(n_out)[:, None] - np.arange(64)[None, :])
        np.testing.assert_allclose(oracle.resample_exact(x, a, n_out), S @ x, rtol=0, atol=1e-12)


def test_exact_identity_at_alpha_one():
    x = synth.bandlimited_noise(1024, synth.rng_for(1, salt=4))
    assert np.array_equal(oracle.resample_exact(x, 1.0), x)


def test_exact_gaussian_tone_is_exact():
    # Whittaker-Shannon reconstruction is exact for band-limited signals
    # (Sec. III-A, Table I "Exact"): a Gaussian tone dilated by alpha.
    n, c, s, f = 512, 256.0, 20.0, 0.15
    a = oracle.alpha(-7500.0 * 40)
    x = synth.gaussian_tone(n, c, s, f)
    t = a * np.arange(n)
    exact = np.exp(-((t - c) ** 2) / (2 * s * s)) * np.exp(2j * np.pi * f * t)
    assert np.max(np.abs(oracle.resample_exact(x, a, n) - exact)) < 1e-11


def test_exact_rows_and_stacks_agree():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, 300)) + 1j * rng.standard_normal((3, 300))
    a = oracle.alpha(5000.0)
    Y = oracle.resample_exact(X, a, 310)
    rows = np.array([0, 7, 150, 299, 309])
    np.testing.assert_allclose(oracle.resample_exact_rows(X, a, rows), Y[:, rows], rtol=0, atol=1e-14)
    np.testing.assert_allclose(Y[1], oracle.resample_exact(X[1], a, 310), rtol=0, atol=1e-13)
