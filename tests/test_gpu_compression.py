"""GPU parity of pulse compression bundled with the ionospheric correction
(Sec. II-B, the pulse-compression path): correct_compress (one pulse) and
correct_compress_bank (one pulse x every (v_r, TEC) pair, the replica's
conjugate spectrum folded into each TEC's factor table) against the FP64
oracle's time-domain matched filter, on every transform schedule (one row
pass, cluster-fused, three passes) and resampling mode.  Tolerance: rel-L2 <=
1e-5 over the lags checked (FP32 path).
"""

import numpy as np
import pytest

import oracle
from oracle import compression as pc
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
    return synth.bandlimited_noise(n, synth.rng_for(9, salt=salt)).astype(np.complex64)


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def lag_sample(n, k, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([np.arange(min(n, 64)), np.arange(max(0, n - 64), n),
                                     rng.integers(0, n, k)]))


# n, n_rep, mode: L = 1024 (one row pass), 4096 (one CTA), 65536 (16-CTA
# clusters), 2^17 (three passes); replica shorter than, equal to and
# (n < L) longer than the pulse
@pytest.mark.parametrize("n,n_rep,mode", [(1000, 300, "windowed"), (1000, 1024, "exact"),
                                          (4096, 4096, "windowed"), (3000, 3500, "freqconv"),
                                          (40000, 2048, "windowed"), (65536, 9000, "windowed"),
                                          (100000, 5000, "windowed"), (200000, 1, "windowed")])
def test_correct_compress_matches_oracle(dcg, ctx, n, n_rep, mode):
    import torch
    x, h = noise(n, n % 101), noise(n_rep, 7) if n_rep > 1 else np.array([0.5 - 1j], np.complex64)
    y = torch.full((n,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    m = {"windowed": dcg.DC_WINDOWED, "exact": dcg.DC_EXACT_FP32, "freqconv": dcg.DC_FREQCONV}[mode]
    v, tec = -7000.0, 130.0
    dcg.correct_compress(ctx, dev(x), dev(h), y, FS, FC, v, tec, mode=m, freq_ref=1e6)
    dcg.dc_check(ctx)
    lags = np.arange(n) if n <= 4096 else lag_sample(n, 1500, n)
    ref = pc.correct_compress(x.astype(np.complex128), h.astype(np.complex128), FS, FC, v, tec,
                              mode=mode, freq_ref=1e6, lags=lags)
    got = y.cpu().numpy()[lags]
    assert rel(got, ref) <= TOL


def test_compressed_peak_recovers_the_replica(dcg, ctx):
    # a replica placed at a known delay and distorted by the ionosphere
    # (Eq. 15): the bundled correction + matched filter peaks at the delay
    # with the replica's energy
    import torch
    n, d, tec = 16384, 5000, 140.0
    h = synth.lfm(2048, FS, 4e6)
    x = np.zeros(n, dtype=np.complex128)
    x[d:d + len(h)] = h
    xd = oracle.iono_distort(x, FS, FC, tec).astype(np.complex64)
    y = torch.empty(n, dtype=torch.complex64, device="cuda")
    dcg.correct_compress(ctx, dev(xd), dev(h.astype(np.complex64)), y, FS, FC, 0.0, tec)
    dcg.dc_check(ctx)
    r = np.abs(y.cpu().numpy())
    e = np.sum(np.abs(h) ** 2)
    assert int(np.argmax(r)) == d
    assert abs(r[d] - e) < 1e-5 * e
    # without the correction the peak sits a group delay later (Eq. 3)
    dcg.correct_compress(ctx, dev(xd), dev(h.astype(np.complex64)), y, FS, FC, 0.0, 0.0)
    r0 = np.abs(y.cpu().numpy())
    shift = 2.0 * oracle.KAPPA * tec * oracle.TECU / (oracle.C_LIGHT * FC ** 2) * FS
    assert abs(int(np.argmax(r0)) - d - shift) <= 0.6


@pytest.mark.parametrize("n,n_rep,n_v,n_tec", [(1000, 200, 3, 2), (4096, 1000, 3, 2),
                                               (65536, 4096, 4, 3), (200000, 3000, 2, 2)])
def test_correct_compress_bank_matches_oracle(dcg, ctx, n, n_rep, n_v, n_tec):
    import torch
    x, h = noise(n, 40 + n % 7), noise(n_rep, 41)
    rng = np.random.default_rng(n)
    v, tec = rng.uniform(-8000, 8000, n_v), rng.uniform(5, 150, n_tec)
    out = torch.empty(n_v * n_tec * n, dtype=torch.complex64, device="cuda")
    dcg.correct_compress_bank(ctx, dev(x), dev(h), v, tec, out, FS, FC)
    dcg.dc_check(ctx)
    got = out.view(n_v, n_tec, n).cpu().numpy()
    lags = np.arange(n) if n <= 4096 else lag_sample(n, 800, n + 1)
    x64, h64 = x.astype(np.complex128), h.astype(np.complex128)
    for i in range(n_v):
        for t in range(n_tec):
            ref = pc.correct_compress(x64, h64, FS, FC, v[i], tec[t], lags=lags)
            assert rel(got[i, t][lags], ref) <= TOL, (i, t)


def test_compress_rejects_bad_replicas(dcg, ctx):
    import torch
    x = dev(noise(1000, 1))
    y = torch.full((1000,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    too_long = dev(noise(1025, 2))                     # L = 1024 for n = 1000
    with pytest.raises(dcg.DcError):
        dcg.correct_compress(ctx, x, too_long, y, FS, FC, 0.0, 10.0)
    with pytest.raises(dcg.DcError):
        dcg.correct_compress_bank(ctx, x, too_long, [0.0], [10.0], y, FS, FC)
    dcg.dc_check(ctx)
    assert np.all(y.cpu().numpy() == np.complex64(7 - 7j))
