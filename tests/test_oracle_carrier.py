"""Pins for the oracle's frequency conversion and the passband carrier term
(CPU only): the cheap O(N) Doppler method of Sec. I / Table I ("Frequency
Conversion") and the term exp(2 pi i fc (alpha - 1) n Ts) that a passband
dilation adds to a baseband pulse.

Each check ties the oracle to something other than itself: the closed form of
a dilated tone, the analytic dilation of an LFM (Table I's error growth with
bandwidth), and the identity between dilating a passband signal and dilating
its baseband envelope with the carrier term applied.
"""

import numpy as np
import pytest

import oracle
from oracle import predistortion as pdist
import synth


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("v,f_ref", [(7500.0, 2.3e6), (-8000.0, -4.1e6), (1000.0, 413e6)])
def test_freqconv_exact_for_a_tone_at_the_reference(v, f_ref):
    # Eq. 2 turns exp(2 pi i f0 t) into exp(2 pi i f0 alpha t): a tone at the
    # reference frequency is dilated exactly by the tone multiply.
    fs = 2.048e9 if f_ref > 1e8 else 20e6
    n = 50000
    m = np.arange(n, dtype=np.float64)
    x = np.exp(2j * np.pi * f_ref * m / fs)
    y = oracle.frequency_conversion(x, oracle.alpha_minus_one(v), fs, f_ref)
    want = np.exp(2j * np.pi * f_ref * oracle.alpha(v) * m / fs)
    assert np.max(np.abs(y - want)) < 1e-8


def test_freqconv_misses_other_frequencies_by_f_delta():
    # a tone at f != f_ref comes out at f + f_ref delta instead of f alpha:
    # the output's phase slope against the dilated tone is (f - f_ref) delta.
    fs, n, v = 20e6, 4096, 8000.0
    f, f_ref = 3e6, 1e6
    dl = oracle.alpha_minus_one(v)
    m = np.arange(n, dtype=np.float64)
    y = oracle.frequency_conversion(np.exp(2j * np.pi * f * m / fs), dl, fs, f_ref)
    ph = np.unwrap(np.angle(y * np.exp(-2j * np.pi * f * oracle.alpha(v) * m / fs)))
    slope = np.polyfit(m, ph, 1)[0] * fs / (2 * np.pi)            # Hz
    assert abs(slope - (-(f - f_ref) * dl)) < 1e-6 * abs((f - f_ref) * dl) + 1e-9


def test_freqconv_error_grows_as_bandwidth_squared():
    # Table I: frequency conversion's error for LFMs scales as B^2.  An RF
    # LFM from f0 over T is dilated analytically (Eq. 2, the LFM regenerated
    # with the dilated time axis) and by a tone multiply at the band centre;
    # the error energy quadruples when B doubles.
    fs, T, f0, v = 2.048e9, 100e-6, 413e6, 1000.0
    n = int(T * fs)
    t = np.arange(n) / fs
    a, dl = oracle.alpha(v), oracle.alpha_minus_one(v)
    errs = []
    for B in (9e6, 18e6, 36e6):
        x = np.exp(1j * pdist.lfm_phase(t, f0, B, T))
        y = np.where(a * t < T, np.exp(1j * pdist.lfm_phase(a * t, f0, B, T)), 0.0)
        z = oracle.frequency_conversion(x, dl, fs, f0 + B / 2.0)
        errs.append(rel(z, y) ** 2)
    assert 3.4 < errs[1] / errs[0] < 4.4
    assert 3.6 < errs[2] / errs[1] < 4.2


def test_freqconv_zero_delta_and_truncation():
    x = synth.bandlimited_noise(1000, synth.rng_for(7))
    assert np.array_equal(oracle.frequency_conversion(x, 0.0, 20e6, 5e6), x)
    y = oracle.frequency_conversion(x, 1e-5, 20e6, 5e6, n_out=1200)
    assert np.all(y[1000:] == 0)
    np.testing.assert_allclose(np.abs(y[:1000]), np.abs(x), rtol=1e-14)


@pytest.mark.parametrize("mode", ["exact", "windowed"])
def test_carrier_term_matches_passband_dilation(mode):
    # Dilating a passband signal p = x exp(2 pi i fc n/fs) and mixing it back
    # down equals dilating x and applying the carrier term (c4 reading of
    # Eq. 2 on complex baseband).  A Gaussian-envelope tone keeps both x and p
    # band-limited and time-limited, so interior samples agree to the
    # interpolation's accuracy.
    fs, fc, n, v = 20e6, 3e6, 4096, 8000.0 * 40      # large delta makes the term visible
    x = synth.gaussian_tone(n, n / 2, 300.0, 0.05)
    m = np.arange(n, dtype=np.float64)
    p = x * np.exp(2j * np.pi * fc * m / fs)
    a, dl = oracle.alpha(v), oracle.alpha_minus_one(v)
    rs = oracle.resample_exact if mode == "exact" else oracle.resample_windowed
    lhs = rs(p, a) * np.exp(-2j * np.pi * fc * m / fs)
    rhs = oracle.resample(x, fs, fc, v, mode=mode, carrier_shift=True)
    tol = 1e-9 if mode == "exact" else 2e-4
    assert rel(lhs, rhs) < tol
    # without the term the two differ by the carrier's phase drift
    plain = oracle.resample(x, fs, fc, v, mode=mode)
    assert rel(lhs, plain) > 0.1
    # mutations: alpha instead of alpha - 1, or the opposite sign
    wrong = plain * oracle.carrier_term(n, a, fs, fc)
    assert rel(lhs, wrong) > 0.1
    wrong = plain * np.conj(oracle.carrier_term(n, dl, fs, fc))
    assert rel(lhs, wrong) > 0.1


def test_carrier_term_reduces_large_phases():
    # the phase reaches thousands of cycles (fc = 1 GHz, 8 km/s, 2^20 samples):
    # the reduced form equals the unreduced exponential
    n, dl, fs, fc = 1 << 20, oracle.alpha_minus_one(8000.0), 20e6, 1e9
    c = oracle.carrier_term(n, dl, fs, fc)
    k = np.array([0, 1, 12345, n - 1])
    want = np.exp(2j * np.pi * (fc * dl * k / fs))
    np.testing.assert_allclose(c[k], want, atol=1e-9)
    assert abs(fc * dl * (n - 1) / fs) > 2000
