"""Pins for the oracle's FFT ionospheric correction (CPU only).

The DFT convention is pinned to a brute-force sum and to the shift theorem the
paper states (Sec. II-B); the phase law to the physical group delay of Eq. 3
measured on a pulse envelope; the correction to the exact inverse of the
distortion (Eqs. 15-16); the constant kappa to the textbook GNSS figure.
"""

import numpy as np
import pytest

import oracle
import synth


def test_kappa_textbook_value():
    # kappa = e^2/(8 pi^2 m_e eps0) ~ 40.3 m^3/s^2; one TECU delays GPS L1
    # (1575.42 MHz) by 0.162 m of range (one way).
    assert abs(oracle.KAPPA - 40.3082) < 1e-3
    assert abs(oracle.KAPPA * 1e16 / 1575.42e6 ** 2 - 0.1624) < 5e-4


@pytest.mark.parametrize("L", [8, 16, 64])
def test_dft_convention_brute_force(L):
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    n = np.arange(L)
    F = np.exp(-2j * np.pi * np.outer(n, n) / L)
    np.testing.assert_allclose(np.fft.fft(x), F @ x, atol=1e-12)
    np.testing.assert_allclose(np.fft.ifft(F @ x), x, atol=1e-13)


def test_shift_theorem_sign():
    # Sec. II-B: if h(t) = g(t - t0) then h^ = g^ exp(-2 pi i t0 f).
    L, d = 256, 5
    rng = np.random.default_rng(1)
    g = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    f = np.fft.fftfreq(L)
    h = np.fft.ifft(np.fft.fft(g) * np.exp(-2j * np.pi * d * f))
    np.testing.assert_allclose(h, np.roll(g, d), atol=1e-12)


def test_bin_frequencies_match_fftfreq():
    for L in (8, 1024, 4096):
        np.testing.assert_array_equal(oracle.bin_frequencies(L, 20e6, 1e9),
                                      1e9 + np.fft.fftfreq(L, d=1 / 20e6))


def test_zero_tec_is_identity():
    x = synth.bandlimited_noise(3000, synth.rng_for(1, salt=5))
    np.testing.assert_allclose(oracle.iono_correct(x, 20e6, 1e9, 0.0), x, atol=1e-14)


@pytest.mark.parametrize("tec", [5.0, 50.0, 150.0])
def test_distort_then_correct_is_identity(tec):
    # Eq. 16 is the exact inverse of Eq. 15 on the transform buffer.
    x = synth.bandlimited_noise(4096, synth.rng_for(1, salt=6))
    d = oracle.iono_distort(x, 20e6, 1e9, tec)
    assert np.max(np.abs(d - x)) > 0.1                          # it does something
    np.testing.assert_allclose(oracle.iono_correct(d, 20e6, 1e9, tec), x, atol=1e-12)
    np.testing.assert_allclose(oracle.iono_correct(x, 20e6, 1e9, -tec), d, atol=1e-12)


@pytest.mark.parametrize("tec,f1", [(50.0, 0.0), (150.0, 3e6), (100.0, -4e6)])
def test_group_delay_matches_eq3(tec, f1):
    # Distortion (Eq. 15) delays a narrowband pulse centred on RF frequency f by
    # the two-way group delay 2 tau(f) = 2 K2/(c f^2) (Eq. 3).  Measured here as
    # the shift of the energy centroid of the envelope.
    fs, fc, L = 20e6, 1e9, 8192
    m = np.arange(L)
    c, s = 4096.0, 60.0
    x = np.exp(-((m - c) ** 2) / (2 * s * s)) * np.exp(2j * np.pi * f1 / fs * m)
    z = oracle.iono_distort(x, fs, fc, tec)
    centroid = lambda v: np.sum(m * np.abs(v) ** 2) / np.sum(np.abs(v) ** 2)
    delay_s = (centroid(z) - centroid(x)) / fs
    expect = 2 * oracle.KAPPA * tec * oracle.TECU / (oracle.C_LIGHT * (fc + f1) ** 2)
    assert abs(delay_s - expect) < 2e-3 * expect
    back = oracle.iono_correct(x, fs, fc, tec)
    assert abs((centroid(back) - centroid(x)) / fs + expect) < 2e-3 * expect


def test_truncation_matches_full_buffer():
    x = synth.bandlimited_noise(3000, synth.rng_for(1, salt=7))
    full = np.zeros(4096, dtype=np.complex128)
    full[:3000] = x
    a = oracle.iono_correct(x, 20e6, 1e9, 80.0)
    b = oracle.iono_correct(full, 20e6, 1e9, 80.0)[:3000]
    np.testing.assert_allclose(a, b, atol=1e-14)
    assert a.shape == (3000,)


def test_rf_mode_dc_bin_has_zero_phase():
    phi = oracle.iono_phase(1024, 2.048e9, 0.0, 100.0)
    assert phi[0] == 0.0 and np.all(np.isfinite(phi))
    assert np.all(phi[1:512] > 0) and np.all(phi[512:] < 0)


def test_correct_is_resample_then_iono():
    cfg = synth.PlainPulse()
    x = cfg.pulse()
    z = oracle.correct(x, cfg.fs, cfg.fc, cfg.v_r, cfg.tec)
    y = oracle.resample_windowed(x, oracle.alpha(cfg.v_r), cfg.n)
    np.testing.assert_array_equal(z, oracle.iono_correct(y, cfg.fs, cfg.fc, cfg.tec))
    bank = oracle.correct_bank(x[:512], cfg.fs, cfg.fc, [cfg.v_r, -100.0], [5.0, cfg.tec])
    np.testing.assert_allclose(bank[1, 0], oracle.correct(x[:512], cfg.fs, cfg.fc, -100.0, 5.0), atol=0)
