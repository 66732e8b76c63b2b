"""GPU test: a recorded plan replayed back to back gives, every time, the
result of the direct call.

The single-pulse plan launches its correction kernel programmatically behind
the resampler, so that kernel may be running while the resampler still
writes the pulse it reads; it must wait for the resampler before reading.
Many replays in a row, each result copied aside on the same stream, give
that ordering many chances to go wrong: every copy must equal the direct
call bitwise.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

REPLAYS = 200


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


def replay_all(torch, plan, out, replays):
    """Every replay's output, copied aside on the replay's stream."""
    keep = torch.empty((replays, out.numel()), dtype=out.dtype, device=out.device)
    for k in range(replays):
        plan.execute()
        keep[k].copy_(out)
    torch.cuda.synchronize()
    return keep


@pytest.mark.parametrize("mode_name", ["windowed", "exact"])
def test_single_pulse_plan_replays_equal_direct_call(dcg, ctx, mode_name):
    import torch
    mode = dcg.DC_WINDOWED if mode_name == "windowed" else dcg.DC_EXACT_FP32
    cfg = synth.PlainPulse()
    x = cfg.pulse().astype(np.complex64)
    items = np.zeros(1, dtype=dcg.ITEM_DTYPE)
    items[0] = (0, cfg.n, 0, cfg.n, cfg.fs, cfg.fc, cfg.v_r, cfg.tec)
    xd = torch.from_numpy(x).cuda()
    direct = torch.empty_like(xd)
    dcg.correct_batch(ctx, xd, direct, items, mode=mode)
    torch.cuda.synchronize()
    ref = oracle.correct(x.astype(np.complex128), cfg.fs, cfg.fc, cfg.v_r, cfg.tec, mode=mode_name)
    d = direct.cpu().numpy()
    assert np.linalg.norm(d - ref) / np.linalg.norm(ref) <= 1e-5
    out = torch.zeros_like(xd)
    plan = dcg.dc_plan_batch(ctx, xd, out, items, mode=mode)
    keep = replay_all(torch, plan, out, REPLAYS)
    plan.close()
    dcg.dc_check(ctx)
    same = (keep == direct.unsqueeze(0)).all(dim=1).cpu().numpy()
    assert same.all(), f"replays differing from the direct call: {np.flatnonzero(~same)[:10]}"


def test_fused_class_plan_replays_equal_direct_call(dcg, ctx):
    # one pulse per cluster-fused length class (L = 2^12 .. 2^16): each class
    # kernel follows the kernel before it programmatically
    import torch
    ns = [3000, 6000, 12000, 30000, 60000]
    items = np.zeros(len(ns), dtype=dcg.ITEM_DTYPE)
    xs, off = [], 0
    for i, n in enumerate(ns):
        xs.append(synth.bandlimited_noise(n, synth.rng_for(9, salt=40 + i)).astype(np.complex64))
        items[i] = (off, n, off, n, 20e6, 1e9, 6000.0 - 2500.0 * i, 20.0 + 25.0 * i)
        off += n
    xd = torch.from_numpy(np.concatenate(xs)).cuda()
    direct = torch.empty_like(xd)
    dcg.correct_batch(ctx, xd, direct, items)
    torch.cuda.synchronize()
    out = torch.zeros_like(xd)
    plan = dcg.dc_plan_batch(ctx, xd, out, items)
    keep = replay_all(torch, plan, out, 50)
    plan.close()
    dcg.dc_check(ctx)
    same = (keep == direct.unsqueeze(0)).all(dim=1).cpu().numpy()
    assert same.all(), f"replays differing from the direct call: {np.flatnonzero(~same)[:10]}"
