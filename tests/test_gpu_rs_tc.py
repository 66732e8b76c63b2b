"""GPU parity of the Doppler bank's windowed-sinc resampling on tensor cores
(tcgen05 GEMM of the pulse's Hankel tiles with each range rate's tap weights
and their first two derivatives at the tile centre, fp16 hi/lo operands)
against the FP64 oracle.

With TEC = 0 the bank's correction is the identity up to FFT round-off, so
correct_bank returns the resampled pulses themselves.  Tolerance: rel-L2 <=
1e-5 per range rate (the FP32 paths' bar); the same calls through the
CUDA-core kernel (forced by the schedule) must meet it too.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
FS, FC = 20e6, 1e9


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def dcg():
    import paper_2508_04951_gb300 as m
    m.build.build()
    m.load()
    return m


@pytest.fixture(scope="module")
def ctx(dcg):
    c = dcg.Context(0)
    yield c
    c.close()


def noise(n, salt):
    return synth.bandlimited_noise(n, synth.rng_for(11, salt=salt)).astype(np.complex64)


def bank_resampled(dcg, ctx, x, v, n_out=0):
    import torch
    n = x.size
    no = n_out or n
    out = torch.full((len(v) * no,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    dcg.dc_profile_enable(ctx, True)
    dcg.correct_bank(ctx, torch.from_numpy(x).cuda(), v, [0.0], out, FS, FC, n_out=n_out)
    dcg.dc_check(ctx)
    prof = dcg.dc_profile_read(ctx)
    dcg.dc_profile_enable(ctx, False)
    return out.view(len(v), no).cpu().numpy(), prof


CASES = [
    (65536, np.random.default_rng(1).uniform(-8000, 8000, 64), 0),   # the bank's shape, 2 groups
    (1000, np.array([-8000.0, 0.0, 5.0, 7999.0]), 0),                # one partial tile
    (4097, np.random.default_rng(2).uniform(-8000, 8000, 33), 0),    # ragged tile, partial group
    (70001, np.array([3000.0, -3000.0, 100.0]), 70100),              # n_out > n
    (200000, np.random.default_rng(3).uniform(-4000, 4000, 40), 0),  # long pulse
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_tensor_core_bank_resampling_matches_oracle(dcg, ctx, case):
    n, v, n_out = CASES[case]
    x = noise(n, case)
    got, prof = bank_resampled(dcg, ctx, x, v, n_out)
    assert "resample_tc" in prof                     # the tensor-core kernel ran
    x64 = x.astype(np.complex128)
    idx = range(len(v)) if len(v) <= 8 else np.random.default_rng(case).choice(len(v), 8, replace=False)
    for i in idx:
        ref = oracle.resample_windowed(x64, oracle.alpha(v[i]), n_out or n)
        assert rel(got[i], ref) <= TOL, (i, v[i])


def test_cuda_core_schedule_agrees(dcg, ctx):
    n, v = 65536, np.array([-7777.0, -10.0, 4321.0])
    x = noise(n, 9)
    tc, _ = bank_resampled(dcg, ctx, x, v)
    dcg.dc_tuning_set(ctx, {"resample_tc": 2})
    try:
        cc, prof = bank_resampled(dcg, ctx, x, v)
        assert "resample_tc" not in prof and "resample_tiled" in prof
    finally:
        dcg.dc_tuning_set(ctx, None)
    for i in range(len(v)):
        ref = oracle.resample_windowed(x.astype(np.complex128), oracle.alpha(v[i]))
        assert rel(cc[i], ref) <= TOL
        assert rel(tc[i], ref) <= TOL
        assert rel(tc[i], cc[i]) <= 2 * TOL


@pytest.mark.parametrize("scale", [1e-6, 3e4])
def test_input_scale_is_handled(dcg, ctx, scale):
    # the operands are scaled per tile before the fp16 split: tiny and large
    # pulses resample as accurately as unit-power ones
    n, v = 8192, np.array([-8000.0, 6000.0])
    x = (noise(n, 4) * scale).astype(np.complex64)
    got, prof = bank_resampled(dcg, ctx, x, v)
    assert "resample_tc" in prof
    for i in range(len(v)):
        ref = oracle.resample_windowed(x.astype(np.complex128), oracle.alpha(v[i]))
        assert rel(got[i], ref) <= TOL


def test_far_apart_range_rates_fall_back(dcg, ctx):
    # delays 2e-3 n apart: more than one tensor-core tile's tap span, so the
    # bank resamples on CUDA cores, still to the oracle's result
    n, v = 65536, np.array([-3e5, 3e5])
    x = noise(n, 5)
    got, prof = bank_resampled(dcg, ctx, x, v)
    assert "resample_tc" not in prof
    for i in range(len(v)):
        ref = oracle.resample_windowed(x.astype(np.complex128), oracle.alpha(v[i]))
        assert rel(got[i], ref) <= TOL


def test_lfm_dilated_slope_through_the_tensor_core_bank(dcg, ctx):
    # Table I / Sec. I: an LFM resampled by the bank matches the analytically
    # dilated LFM (chirp rate k alpha^2 about T/(2 alpha)) on interior samples
    n, B = 16384, 6e6
    x = synth.lfm(n, FS, B)
    v = np.array([-8000.0, 8000.0])
    got, prof = bank_resampled(dcg, ctx, x.astype(np.complex64), v)
    assert "resample_tc" in prof
    T = n / FS
    k = B / T
    t = np.arange(n) / FS
    for i in range(len(v)):
        a = oracle.alpha(v[i])
        want = np.exp(1j * np.pi * k * (a * t - T / 2) ** 2)
        sl = slice(64, n - 64)
        assert np.max(np.abs(got[i][sl] - want[sl])) < 2e-4
