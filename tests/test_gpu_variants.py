"""GPU parity of the cheap Doppler variants of Sec. I / Table I against the FP64
oracle: frequency conversion (DC_FREQCONV, the O(N) tone multiply) and the
carrier term of a passband dilation (dc_opts.carrier_shift), through every
entry point that takes them: doppler_resample, correct_batch, correct_bank and
their plans.  Tolerance: rel-L2 <= 1e-5 per pulse (FP32 paths).
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
    return synth.bandlimited_noise(n, synth.rng_for(8, salt=salt)).astype(np.complex64)


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy().astype(np.complex128)


# n, v_r, n_out: the tiled resampler with 8 and 4 outputs per lane, its
# exact-weight warp tiles, the direct kernel, ragged ends, long pulses
@pytest.mark.parametrize("n,v,n_out", [(4096, 7500.0, 4096), (70001, -8000.0, 70001),
                                       (70001, 15000.0, 69000), (5000, 1.4e6, 5000),
                                       (3000, -2e7, 3300), (1 << 20, 8000.0, 1 << 20)])
def test_windowed_with_carrier_term(dcg, ctx, n, v, n_out):
    import torch
    x = noise(n, salt=n % 89)
    xd = dev(x)
    # output one sample into a buffer: an 8-byte-aligned (not 16) output too
    buf = torch.full((n_out + 1,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    for off in (0, 1):
        y = buf[off:off + n_out]
        dcg.doppler_resample(ctx, xd, y, FS, FC, v, n_out=n_out, carrier_shift=True)
        dcg.dc_check(ctx)
        ref = oracle.resample(x.astype(np.complex128), FS, FC, v, n_out=n_out, carrier_shift=True)
        assert rel(host(y), ref) <= TOL, off


@pytest.mark.parametrize("n,n_out", [(4096, 4096), (3000, 3100)])
def test_exact_with_carrier_term(dcg, ctx, n, n_out):
    import torch
    x = noise(n, salt=3)
    y = torch.empty(n_out, dtype=torch.complex64, device="cuda")
    dcg.doppler_resample(ctx, dev(x), y, FS, FC, -7500.0, n_out=n_out, mode=dcg.DC_EXACT_FP32,
                         carrier_shift=True)
    dcg.dc_check(ctx)
    ref = oracle.resample(x.astype(np.complex128), FS, FC, -7500.0, mode="exact", n_out=n_out,
                          carrier_shift=True)
    assert rel(host(y), ref) <= TOL


@pytest.mark.parametrize("n,n_out,f_ref,shift", [(1, 1, 0.0, True), (4096, 4096, 2.5e6, False),
                                                 (70001, 80000, -3e6, True), (1 << 20, 1 << 20, 4e6, True)])
def test_freqconv_single_pulse(dcg, ctx, n, n_out, f_ref, shift):
    import torch
    x = noise(n, salt=5) if n > 1 else np.array([1 + 2j], dtype=np.complex64)
    y = torch.full((n_out,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    dcg.doppler_resample(ctx, dev(x), y, FS, FC, 8000.0, n_out=n_out, mode=dcg.DC_FREQCONV,
                         carrier_shift=shift, freq_ref=f_ref)
    dcg.dc_check(ctx)
    ref = oracle.resample(x.astype(np.complex128), FS, FC, 8000.0, mode="freqconv", n_out=n_out,
                          carrier_shift=shift, freq_ref=f_ref)
    assert rel(host(y), ref) <= TOL


@pytest.mark.parametrize("mode,shift", [("freqconv", False), ("freqconv", True), ("windowed", True),
                                        ("exact", True)])
def test_correct_batch_variants(dcg, ctx, mode, shift):
    import torch
    lens = [700, 4096, 5000, 70000, 3] if mode != "exact" else [700, 4096, 3]
    rng = np.random.default_rng(12)
    items = np.zeros(len(lens), dtype=dcg.ITEM_DTYPE)
    xs, off = [], 0
    for i, n in enumerate(lens):
        xs.append(noise(n, 20 + i))
        items[i] = (off, n, off, n, FS, FC, rng.uniform(-8000, 8000), rng.uniform(5, 150))
        off += n
    xd = dev(np.concatenate(xs))
    od = torch.full_like(xd, complex(7.0, -7.0))
    m = {"freqconv": dcg.DC_FREQCONV, "windowed": dcg.DC_WINDOWED, "exact": dcg.DC_EXACT_FP32}[mode]
    dcg.correct_batch(ctx, xd, od, items, mode=m, carrier_shift=shift, freq_ref=1.5e6)
    dcg.dc_check(ctx)
    out = od.cpu().numpy()
    # the recorded plan replays the same call bitwise
    od2 = torch.zeros_like(xd)
    plan = dcg.dc_plan_batch(ctx, xd, od2, items, mode=m, carrier_shift=shift, freq_ref=1.5e6)
    od2.zero_()
    plan.execute()
    torch.cuda.synchronize()
    assert torch.equal(od2, od)
    plan.close()
    off = 0
    for i, n in enumerate(lens):
        it = items[i]
        ref = oracle.correct(xs[i].astype(np.complex128), FS, FC, it["v_r"], it["tec_tecu"], mode=mode,
                             carrier_shift=shift, freq_ref=1.5e6)
        assert rel(out[off:off + n], ref) <= TOL, (i, n)
        off += n


@pytest.mark.parametrize("mode,shift", [("freqconv", True), ("windowed", True)])
def test_correct_bank_variants(dcg, ctx, mode, shift):
    import torch
    n, v, tec = 65536, np.array([-8000.0, -10.0, 3000.0, 7999.0]), np.array([5.0, 150.0])
    x = noise(n, 31)
    out = torch.empty(len(v) * len(tec) * n, dtype=torch.complex64, device="cuda")
    m = dcg.DC_FREQCONV if mode == "freqconv" else dcg.DC_WINDOWED
    dcg.correct_bank(ctx, dev(x), v, tec, out, FS, FC, mode=m, carrier_shift=shift, freq_ref=-2e6)
    dcg.dc_check(ctx)
    ref = oracle.correct_bank(x.astype(np.complex128), FS, FC, v, tec, mode=mode, carrier_shift=shift,
                              freq_ref=-2e6)
    got = out.view(len(v), len(tec), n).cpu().numpy()
    for i in range(len(v)):
        for t in range(len(tec)):
            assert rel(got[i, t], ref[i, t]) <= TOL, (i, t)


def test_variant_options_validated(dcg, ctx):
    import torch
    x = dev(noise(64, 1))
    y = torch.full((64,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    with pytest.raises(dcg.DcError):
        dcg.doppler_resample(ctx, x, y, FS, FC, 0.0, mode=5)
    with pytest.raises(dcg.DcError):
        dcg.doppler_resample(ctx, x, y, FS, FC, 0.0, mode=dcg.DC_FREQCONV, freq_ref=float("inf"))
    with pytest.raises(dcg.DcError):
        dcg.doppler_resample(ctx, x, y, FS, FC, 0.0, mode=dcg.DC_EXACT_BF16X3)
    dcg.dc_check(ctx)
    assert np.all(y.cpu().numpy() == np.complex64(7 - 7j))
