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
