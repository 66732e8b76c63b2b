"""GPU parity at the longest pulses the library takes (2^20 samples, the top
of the serving stream's length range) and at the largest Doppler range rate
of the workloads (|v_r| = 8 km/s, delta n up to ~56 samples at the end of the
pulse), through every entry point a 2^20-sample pulse can reach: resampling
alone, the full correction in a ragged batch, and one served request.  Each
result is checked whole against the FP64 oracle.  Also: a context whose HBM
budget is too small for a call refuses it with DC_EBUSY and launches nothing.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
N20 = 1 << 20
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


def lfm(n, salt):
    rng = synth.rng_for(6, salt=salt)
    return synth.lfm(n, FS, rng.uniform(1e6, 10e6)).astype(np.complex64)


def noise(n, salt):
    return synth.bandlimited_noise(n, synth.rng_for(6, salt=salt)).astype(np.complex64)


@pytest.mark.parametrize("v", [8000.0, -8000.0])
def test_resample_2p20_at_8kms(dcg, ctx, v):
    import torch
    x = noise(N20, salt=1 if v > 0 else 2)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    dcg.doppler_resample(ctx, xd, yd, FS, FC, v)
    dcg.dc_check(ctx)
    ref = oracle.resample_windowed(x.astype(np.complex128), oracle.alpha(v))
    assert rel(yd.cpu().numpy(), ref) <= TOL


def test_correct_batch_with_2p20_pulses(dcg, ctx):
    import torch
    lens = [N20, 3000, N20 - 777, 70000]
    vs = [8000.0, -8000.0, -8000.0, 5000.0]
    tecs = [150.0, 150.0, 60.0, 20.0]
    xs = [lfm(lens[0], 3), noise(lens[1], 4), noise(lens[2], 5), lfm(lens[3], 6)]
    items = np.zeros(len(lens), dtype=dcg.ITEM_DTYPE)
    off = 0
    for i, n in enumerate(lens):
        items[i] = (off, n, off, n, FS, FC, vs[i], tecs[i])
        off += n
    xd = torch.from_numpy(np.concatenate(xs)).cuda()
    od = torch.full_like(xd, complex(7.0, -7.0))
    dcg.correct_batch(ctx, xd, od, items)
    dcg.dc_check(ctx)
    out = od.cpu().numpy()
    off = 0
    for i, n in enumerate(lens):
        ref = oracle.correct(xs[i].astype(np.complex128), FS, FC, vs[i], tecs[i])
        assert rel(out[off:off + n], ref) <= TOL, i
        off += n


def test_served_2p20_request(dcg):
    x = noise(N20, salt=7)
    y = np.zeros_like(x)
    srv = dcg.dc_serve_start(0, 1 << 30, slots=2)
    rid = srv.submit(x, y, FS, FC, -8000.0, 150.0)
    srv.wait(rid, 60000)
    srv.stop()
    ref = oracle.correct(x.astype(np.complex128), FS, FC, -8000.0, 150.0)
    assert rel(y, ref) <= TOL


def test_budget_too_small_is_busy_and_launches_nothing(dcg):
    import torch
    small = dcg.Context(0, budget_bytes=1 << 20)
    cfg = synth.DopplerBank()
    x, v, tec = cfg.draw()
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    n_v, n_tec = 4, 2
    out = torch.full((n_v * n_tec * cfg.n,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    before = dcg.dc_launch_count(small)
    with pytest.raises(dcg.DcError) as e:
        dcg.correct_bank(small, xd, v[:n_v], tec[:n_tec], out, cfg.fs, cfg.fc)
    assert e.value.status == 3                       # DC_EBUSY
    assert dcg.dc_launch_count(small) == before
    dcg.dc_check(small)
    assert np.all(out.cpu().numpy() == np.complex64(7 - 7j))
    # a call that fits the budget still runs on the same context
    y = torch.empty(4096, dtype=torch.complex64, device="cuda")
    dcg.iono_correct(small, xd[:4096].contiguous(), y, cfg.fs, cfg.fc, 50.0)
    dcg.dc_check(small)
    ref = oracle.iono_correct(x[:4096].astype(np.complex64).astype(np.complex128), cfg.fs, cfg.fc, 50.0)
    assert rel(y.cpu().numpy(), ref) <= TOL
    small.close()
