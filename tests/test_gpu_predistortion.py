"""GPU parity of the predistorted LFM transmit waveforms (Sec. II-A, II-C,
Appendix B) against the FP64 oracle, and the paper's Fig. 2 comparison run
entirely on the GPU: the cubic-predistorted LFM (Eqs. 4, 11-14, trapezoidal
phase) against the LFM predistorted by the FFT method (Eq. 16 through
iono_correct at RF sampling) within the printed 0.01 dB.
"""

import json
import os

import numpy as np
import pytest

import oracle
from oracle import predistortion as pdist

pytestmark = pytest.mark.gpu

TOL = 1e-5
E1 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))["E1_fig2"]
F0, B, FS, T = E1["f0_hz"], E1["bandwidth_hz"], E1["fs_hz"], E1["T_s"]
TEC = E1["tec_el_m2"] / oracle.TECU
N = int(round(T * FS))


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


KINDS = {"lfm": 0, "cubic": 1, "poly": 2, "poly4": 3}


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("f_mix", [0.0, F0])
def test_waveform_matches_oracle(dcg, ctx, kind, f_mix):
    import torch
    y = torch.full((N,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    dcg.predistort_lfm(ctx, y, FS, F0, B, T, TEC, f_mix=f_mix, kind=KINDS[kind])
    dcg.dc_check(ctx)
    ref = pdist.predistorted_lfm(N, FS, F0, B, T, TEC, kind, f_mix)
    assert rel(y.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("n,tec", [(1, 100.0), (1025, 0.0), (1 << 22, 60.0)])
def test_cubic_lengths_and_zero_tec(dcg, ctx, n, tec):
    # lengths around the scan's 1024-sample blocks and the largest allowed;
    # the waveform runs past T where n / fs > T (the formulas extend)
    import torch
    y = torch.empty(n, dtype=torch.complex64, device="cuda")
    dcg.predistort_lfm(ctx, y, FS, F0, B, T, tec, kind=dcg.DC_LFM_CUBIC)
    dcg.dc_check(ctx)
    ref = pdist.predistorted_lfm(n, FS, F0, B, T, tec, "cubic")
    assert rel(y.cpu().numpy(), ref) <= TOL


def test_fig2_cubic_against_fft_predistortion_on_gpu(dcg, ctx):
    # Fig. 2: the LFM predistorted by the FFT method (Eq. 16 with fc = 0: RF
    # samples, guard zeros on both sides) against the cubic waveform: loss
    # below 0.01 dB; both computed by the library
    import torch
    L, off = 1 << 19, 1 << 16
    lfm = torch.empty(N, dtype=torch.complex64, device="cuda")
    dcg.predistort_lfm(ctx, lfm, FS, F0, B, T, TEC, kind=dcg.DC_LFM_PLAIN)
    buf = torch.zeros(L, dtype=torch.complex64, device="cuda")
    buf[off:off + N] = lfm
    fft_pre = torch.empty_like(buf)
    dcg.iono_correct(ctx, buf, fft_pre, FS, 0.0, TEC)
    cubic = torch.empty(N, dtype=torch.complex64, device="cuda")
    dcg.predistort_lfm(ctx, cubic, FS, F0, B, T, TEC, kind=dcg.DC_LFM_CUBIC)
    poly = torch.empty_like(cubic)
    dcg.predistort_lfm(ctx, poly, FS, F0, B, T, TEC, kind=dcg.DC_LFM_POLY)
    poly4 = torch.empty_like(cubic)
    dcg.predistort_lfm(ctx, poly4, FS, F0, B, T, TEC, kind=dcg.DC_LFM_POLY_ORIGINAL)
    dcg.dc_check(ctx)
    c = cubic.cpu().numpy().astype(np.complex128)
    assert pdist.snr_loss_db(c, fft_pre.cpu().numpy().astype(np.complex128)) < E1["max_loss_cubic_vs_fft_db"]
    assert pdist.snr_loss_db(c, poly.cpu().numpy().astype(np.complex128)) < E1["max_loss_cubic_vs_poly_db"]
    assert pdist.snr_loss_db(c, poly4.cpu().numpy().astype(np.complex128)) > 0.5


def test_bad_arguments_launch_nothing(dcg, ctx):
    import torch
    y = torch.full((64,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    for kw in (dict(kind=7), dict(kind=1, tec=-1.0), dict(kind=1, T=0.0), dict(kind=2, tec=float("nan"))):
        with pytest.raises(dcg.DcError) as e:
            dcg.predistort_lfm(ctx, y, FS, F0, B, kw.get("T", T), kw.get("tec", TEC), kind=kw["kind"])
        assert e.value.status == 1
    dcg.dc_check(ctx)
    assert np.all(y.cpu().numpy() == np.complex64(7 - 7j))
