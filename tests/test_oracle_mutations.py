"""Planted mistakes in the oracle must trip its pins (CPU only).

Each case patches one oracle function with a plausible error -- a flipped sign,
a one-way instead of two-way factor, a wrong window width, a dropped factor --
and re-runs a pin from the other test files, which must now fail.
"""

import numpy as np
import pytest

import oracle
import oracle.core as core
from tests import test_oracle_iono as ti
from tests import test_oracle_resample as tr


def _expect_failure(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_flipped_phase_sign_is_caught(monkeypatch):
    good = core.iono_phase
    monkeypatch.setattr(core, "iono_phase", lambda *a: -good(*a))
    _expect_failure(ti.test_group_delay_matches_eq3, 50.0, 0.0)


def test_half_phase_is_caught(monkeypatch):
    good = core.iono_phase
    monkeypatch.setattr(core, "iono_phase", lambda *a: 0.5 * good(*a))   # 2 pi instead of 4 pi
    _expect_failure(ti.test_group_delay_matches_eq3, 150.0, 3e6)


def test_one_way_doppler_is_caught(monkeypatch):
    monkeypatch.setattr(core, "alpha", lambda v: 1.0 + v / core.C_LIGHT)
    monkeypatch.setattr(oracle, "alpha", core.alpha)
    _expect_failure(tr.test_alpha_two_way_invariants, 7500.0)


def test_wrong_window_width_is_caught(monkeypatch):
    good = core.kaiser
    monkeypatch.setattr(core, "kaiser", lambda u, R, b: good(u, 2 * R, b))
    _expect_failure(tr.test_windowed_gaussian_tone_closed_form)


def test_dropped_bin_offset_is_caught(monkeypatch):
    # f_k without the carrier term
    monkeypatch.setattr(core, "bin_frequencies",
                        lambda L, fs, fc: fs * np.fft.fftfreq(L))
    _expect_failure(ti.test_group_delay_matches_eq3, 50.0, 0.0)


def test_wrong_frequency_conversion_sign_is_caught(monkeypatch):
    from tests import test_oracle_carrier as tc
    good = core.carrier_term
    monkeypatch.setattr(core, "carrier_term", lambda n, d, fs, f: np.conj(good(n, d, fs, f)))
    _expect_failure(tc.test_freqconv_exact_for_a_tone_at_the_reference, 7500.0, 2.3e6)


def test_carrier_term_with_alpha_instead_of_delta_is_caught(monkeypatch):
    from tests import test_oracle_carrier as tc
    good = core.carrier_term
    monkeypatch.setattr(core, "carrier_term", lambda n, d, fs, f: good(n, d + 1.0, fs, f))
    _expect_failure(tc.test_carrier_term_matches_passband_dilation, "exact")


def test_correlation_lag_reversed_is_caught(monkeypatch):
    # z[m - j] instead of z[m + j]: a convolution, not the matched filter
    import oracle.compression as pc
    from tests import test_oracle_compression as tcmp

    def reversed_lag(z, h, lags):
        z = np.asarray(z, dtype=np.complex128)
        L = z.shape[-1]
        lags = np.arange(int(lags)) if np.ndim(lags) == 0 else np.asarray(lags)
        idx = np.arange(len(h))
        return np.array([np.sum(z[(m - idx) % L] * np.conj(h)) for m in lags])
    monkeypatch.setattr(pc, "cross_correlate", reversed_lag)
    _expect_failure(tcmp.test_peak_at_the_delay_with_the_replica_energy)


def test_predistortion_factor_four_is_caught(monkeypatch):
    # the corrected pseudo-Chebyshev expansion replaced by Appendix B's
    # original factor-4 coefficients: Fig. 2's CUBIC-vs-POLY bound fails
    import oracle.predistortion as pd
    from tests import test_oracle_predistortion as tp
    good = pd.chebyshev_phase
    e1 = tp.E1
    n = int(round(e1["T_s"] * e1["fs_hz"]))
    args = (n, e1["fs_hz"], e1["f0_hz"], e1["bandwidth_hz"], e1["T_s"], e1["tec_el_m2"] / oracle.TECU)

    def pin():
        loss = pd.snr_loss_db(pd.predistorted_lfm(*args, kind="cubic"), pd.predistorted_lfm(*args, kind="poly"))
        assert loss < e1["max_loss_cubic_vs_poly_db"]
    pin()                                        # the pin holds for the correct oracle
    monkeypatch.setattr(pd, "chebyshev_phase",
                        lambda t, f0, B, T, K2, factor=2.0: good(t, f0, B, T, K2, 4.0))
    _expect_failure(pin)
