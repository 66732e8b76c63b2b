"""Pins for the oracle's pulse compression bundled with the ionospheric
correction (Sec. II-B, the paragraph after Eq. 16 and the pulse-compression
figure): the matched filter's output of the corrected pulse against a replica.

Each check ties the oracle to something other than itself: the matched
filter's peak (Cauchy-Schwarz: the replica's energy, at the true delay), the
distortion/correction identity of Eqs. 15-16, the group delay of Eq. 3 seen as
a shift of the compressed peak when the correction is skipped, and the
convolution theorem (a DFT product, a different computation of the same
correlation).
"""

import numpy as np
import pytest

import oracle
from oracle import compression as pc
import synth

FS, FC = 20e6, 1e9


def placed(replica, n, d):
    x = np.zeros(n, dtype=np.complex128)
    x[d:d + len(replica)] = replica
    return x


def lfm_replica(n_rep, bw):
    return synth.lfm(n_rep, FS, bw)


def test_peak_at_the_delay_with_the_replica_energy():
    h = lfm_replica(1000, 5e6)
    n, d = 4096, 1234
    r = pc.correct_compress(placed(h, n, d), h, FS, FC, 0.0, 0.0)
    e = np.sum(np.abs(h) ** 2)
    assert np.argmax(np.abs(r)) == d
    assert abs(r[d] - e) < 1e-9 * e
    assert np.all(np.abs(r) <= e * (1 + 1e-12))


def test_correction_undoes_the_distortion_at_the_peak():
    # Eq. 15 applied to the received window, Eq. 16 in the compression pass:
    # the peak is the replica's energy again, at the true delay
    h = lfm_replica(2000, 8e6)
    L, d, tec = 8192, 3000, 120.0
    x = oracle.iono_distort(placed(h, L, d), FS, FC, tec)
    r = pc.correct_compress(x, h, FS, FC, 0.0, tec)
    e = np.sum(np.abs(h) ** 2)
    assert np.argmax(np.abs(r)) == d
    assert abs(r[d] - e) < 1e-9 * e


@pytest.mark.parametrize("tec", [50.0, 150.0])
def test_uncorrected_peak_moves_by_the_group_delay(tec):
    # Eq. 3: the two-way group delay 2 K2 / (c f^2) at the carrier, in samples;
    # compressing without the correction finds the peak that much later
    h = lfm_replica(2048, 2e6)
    L, d = 16384, 4000
    x = oracle.iono_distort(placed(h, L, d), FS, FC, tec)
    r = np.abs(pc.correct_compress(x, h, FS, FC, 0.0, 0.0))
    m = int(np.argmax(r))
    y0, y1, y2 = r[m - 1], r[m], r[m + 1]
    peak = m + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    want = 2.0 * oracle.KAPPA * tec * oracle.TECU / (oracle.C_LIGHT * FC ** 2) * FS
    assert want > 2.0
    assert abs((peak - d) - want) < 0.05, (peak - d, want)
    # with the correction the peak is back at the delay
    rc = np.abs(pc.correct_compress(x, h, FS, FC, 0.0, tec))
    assert int(np.argmax(rc)) == d


def test_cross_correlation_equals_the_dft_product():
    # convolution theorem: the time-domain matched-filter sum equals the
    # inverse DFT of Z conj(H) (the product the fused pass computes)
    rng = synth.rng_for(9)
    z = synth.bandlimited_noise(4096, rng)
    h = synth.bandlimited_noise(700, rng)
    lags = np.concatenate([np.arange(50), np.arange(4000, 4096)])   # incl. wrap-around lags
    r = pc.cross_correlate(z, h, lags)
    want = np.fft.ifft(np.fft.fft(z) * np.conj(np.fft.fft(h, 4096)))[lags]
    np.testing.assert_allclose(r, want, atol=1e-10)


def test_equals_correct_then_correlate_with_guard_zeros():
    # with the pulse's energy well inside its window, compressing the
    # corrected L-buffer is correlating the (truncated) corrected pulse with
    # the replica, linearly
    h = lfm_replica(500, 4e6)
    n, d = 6000, 2500
    x = placed(h, n, d) + 0.1 * placed(synth.bandlimited_noise(1000, synth.rng_for(10)), n, 2300)
    v, tec = -6000.0, 80.0
    lags = np.arange(2000, 3200)
    r = pc.correct_compress(x, h, FS, FC, v, tec, lags=lags)
    z = oracle.correct(x, FS, FC, v, tec)
    want = np.array([np.sum(z[m:m + len(h)] * np.conj(h)) for m in lags])
    np.testing.assert_allclose(r, want, atol=1e-9 * np.max(np.abs(want)))


def test_mutation_unconjugated_replica_fails():
    # multiplying by the replica spectrum without the conjugate (a convolution)
    # loses the peak: the pin above would catch that mistake
    h = lfm_replica(1000, 5e6)
    x = placed(h, 4096, 1234)
    z = pc.corrected_buffer(x, FS, FC, 0.0, 0.0)
    bad = np.fft.ifft(np.fft.fft(z) * np.fft.fft(h, 4096))
    e = np.sum(np.abs(h) ** 2)
    assert np.max(np.abs(bad)) < 0.2 * e
