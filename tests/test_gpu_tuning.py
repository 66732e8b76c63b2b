"""Schedules of correct_batch / correct_bank: every alternative the
autotuner may pick (three-pass transforms for 4096 <= L <= 65536, 4 outputs
per lane in the resampler, small three-pass chunks) against the FP64 oracle,
and the autotuner's own contract."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def dcg():
    import paper_2508_04951_gb300 as m
    m.build.build()
    m.load()
    return m


@pytest.fixture()
def ctx(dcg):
    c = dcg.Context(0)
    yield c
    c.close()


def batch(dcg, lens, seed=7):
    rng = np.random.default_rng(seed)
    xs = [synth.bandlimited_noise(int(n), synth.rng_for(6, salt=int(n))) for n in lens]
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    x = np.concatenate(xs).astype(np.complex64)
    items = np.zeros(len(lens), dtype=dcg.ITEM_DTYPE)
    for i, n in enumerate(lens):
        items[i] = (offs[i], n, offs[i], n, 20e6, 1e9, rng.uniform(-8000, 8000), rng.uniform(5, 150))
    return x, items


def check_batch(dcg, ctx, x, items, run):
    import torch
    xd = torch.from_numpy(x).cuda()
    od = torch.empty_like(xd)
    out = run(xd, od)
    dcg.dc_check(ctx)
    got = od.cpu().numpy().astype(np.complex128)
    for it in items:
        a, n = int(it["in_off"]), int(it["n"])
        ref = oracle.correct(x[a:a + n].astype(np.complex128), it["fs"], it["fc"], it["v_r"],
                             it["tec_tecu"])
        assert rel(got[a:a + n], ref) <= TOL, (n, it["v_r"])
    return out


LENS = [3000, 4096, 10000, 30000, 60000, 100000, 100000, 140000]   # L = 2^12 .. 2^18


@pytest.mark.parametrize("schedule", [
    {"fft": {12: 2, 14: 2, 15: 2, 16: 2}},                  # one row pass / three passes
    {"resample_q": 4},
    {"chunk": {17: 8 << 17, 18: 8 << 18}},                 # one transform per chunk
    {"fft": {16: 2}, "chunk": {16: 8 << 16}, "resample_q": 4},
])
def test_forced_batch_schedules_match_oracle(dcg, ctx, schedule):
    x, items = batch(dcg, LENS)
    dcg.dc_tuning_set(ctx, schedule)
    check_batch(dcg, ctx, x, items, lambda xd, od: dcg.correct_batch(ctx, xd, od, items))


@pytest.mark.parametrize("n,schedule", [(65536, {"fft": {16: 2}}),
                                        (65536, {"fft": {16: 2}, "chunk": {16: 16 << 20}}),
                                        (4096, {"fft": {12: 2}}),
                                        (65536, {"apply_kind": 1}),    # one row per CTA
                                        (65536, {"apply_kind": 2}),    # two rows per CTA
                                        (40000, {"apply_kind": 2}),    # truncated to n_out
                                        (32768, {"apply_kind": 1}),
                                        (20000, {"apply_kind": 2}),
                                        (65536, {"apply_kind": 3}),    # two passes through L2
                                        (40000, {"apply_kind": 3}),
                                        (20000, {"apply_kind": 3}),
                                        (10000, {"apply_kind": 3}),
                                        (5000, {"apply_kind": 3})])
def test_forced_bank_schedules_match_oracle(dcg, ctx, n, schedule):
    import torch
    x = synth.bandlimited_noise(n, synth.rng_for(6, salt=3)).astype(np.complex64)
    v = np.array([-7000.0, 2500.0])
    tec = np.array([20.0, 90.0, 140.0])
    dcg.dc_tuning_set(ctx, schedule)
    od = torch.empty(len(v) * len(tec) * n, dtype=torch.complex64, device="cuda:0")
    dcg.correct_bank(ctx, torch.from_numpy(x).cuda(), v, tec, od, 20e6, 1e9)
    dcg.dc_check(ctx)
    out = od.cpu().numpy().reshape(len(v), len(tec), n)
    ref = oracle.correct_bank(x.astype(np.complex128), 20e6, 1e9, v, tec)
    for i in range(len(v)):
        for t in range(len(tec)):
            assert rel(out[i, t], ref[i, t]) <= TOL


@pytest.mark.parametrize("n,n_v,n_tec", [(65536, 12, 8), (16384, 40, 16)])
def test_two_pass_apply_reuses_its_scratch_slots(dcg, ctx, n, n_v, n_tec):
    # more transforms than the scratch holds (two chunks of 32 at L = 65536,
    # of 128 at L = 16384): slots are reused after their columns are done;
    # every pair agrees with the cluster kernel, sampled pairs with the oracle
    import torch
    x = synth.bandlimited_noise(n, synth.rng_for(6, salt=7)).astype(np.complex64)
    v = np.linspace(-7900.0, 7900.0, n_v)
    tec = np.linspace(5.0, 150.0, n_tec)
    xd = torch.from_numpy(x).cuda()
    outs = {}
    for kind in (1, 3):
        dcg.dc_tuning_set(ctx, {"apply_kind": kind})
        od = torch.full((n_v * n_tec * n,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda:0")
        dcg.correct_bank(ctx, xd, v, tec, od, 20e6, 1e9)
        dcg.dc_check(ctx)
        outs[kind] = od.cpu().numpy().reshape(n_v, n_tec, n)
    dcg.dc_tuning_set(ctx, None)
    for i in range(n_v):
        for t in range(n_tec):
            assert rel(outs[3][i, t], outs[1][i, t]) <= 1e-6, (i, t)
    ref = oracle.correct_bank(x.astype(np.complex128), 20e6, 1e9, v[[0, n_v - 1]], tec[[0, n_tec - 1]])
    for a, i in enumerate((0, n_v - 1)):
        for b, t in enumerate((0, n_tec - 1)):
            assert rel(outs[3][i, t], ref[a, b]) <= TOL


def test_autotune_batch_keeps_the_fastest_and_correct(dcg, ctx):
    x, items = batch(dcg, LENS, seed=11)
    rep = check_batch(dcg, ctx, x, items,
                      lambda xd, od: dcg.dc_autotune_batch(ctx, xd, od, items))
    assert rep["candidates"] >= 3                  # q, the fft classes and the chunk sizes
    assert rep["ms_best"] <= rep["ms_default"]
    held = dcg.dc_tuning_get(ctx)
    assert held["resample_q"] == rep["resample_q"] and held["fft"] == rep["fft"]
    # later calls run the held schedule
    check_batch(dcg, ctx, x, items, lambda xd, od: dcg.correct_batch(ctx, xd, od, items))
    dcg.dc_tuning_set(ctx, None)
    back = dcg.dc_tuning_get(ctx)
    assert back["resample_q"] == 0 and back["fft"] == {} and back["chunk"] == {}


def test_autotune_bank_and_plan_use_the_schedule(dcg, ctx):
    import torch
    n = 65536
    x = synth.bandlimited_noise(n, synth.rng_for(6, salt=5)).astype(np.complex64)
    v = np.linspace(-8000, 8000, 4)
    tec = np.linspace(10, 150, 4)
    xd = torch.from_numpy(x).cuda()
    od = torch.empty(16 * n, dtype=torch.complex64, device="cuda:0")
    rep = dcg.dc_autotune_bank(ctx, xd, v, tec, od, 20e6, 1e9)
    assert rep["candidates"] >= 2 and rep["ms_best"] <= rep["ms_default"]
    plan = dcg.dc_plan_bank(ctx, xd, v, tec, od, 20e6, 1e9)
    od.zero_()
    plan.execute()
    torch.cuda.synchronize()
    dcg.dc_check(ctx)
    out = od.cpu().numpy().reshape(4, 4, n)
    ref = oracle.correct_bank(x.astype(np.complex128), 20e6, 1e9, v, tec)
    for i in range(4):
        for t in range(4):
            assert rel(out[i, t], ref[i, t]) <= TOL
    plan.close()


def test_tuning_set_rejects_bad_schedules(dcg, ctx):
    for bad in ({"resample_q": 6}, {"fft": {17: 1}}, {"fft": {14: 3}}, {"chunk": {18: -2}},
                {"apply_kind": 4}, {"apply_kind": -1}):
        with pytest.raises(dcg.DcError):
            dcg.dc_tuning_set(ctx, bad)
    assert dcg.dc_tuning_get(ctx)["fft"] == {}


def test_schedule_cache_round_trip(dcg, ctx, tmp_path, monkeypatch):
    sched = {"resample_q": 4, "resample_tc": 2, "apply_kind": 1, "fft": {13: 2, 16: 1},
             "chunk": {17: 64 << 20}}
    dcg.dc_tuning_set(ctx, sched)
    path = str(tmp_path / "sched.json")
    dcg.dc_tuning_save(ctx, path)
    text = open(path).read()
    assert '"format": "dc_tuning/1"' in text
    other = dcg.Context(0)
    dcg.dc_tuning_load(other, path)
    got = dcg.dc_tuning_get(other)
    assert (got["resample_q"], got["resample_tc"], got["apply_kind"], got["fft"], got["chunk"]) == \
        (4, 2, 1, {13: 2, 16: 1}, {17: 64 << 20})
    other.close()
    # a context created with DC_TUNING_CACHE set starts from that file
    monkeypatch.setenv("DC_TUNING_CACHE", path)
    third = dcg.Context(0)
    assert dcg.dc_tuning_get(third)["fft"] == {13: 2, 16: 1}
    third.close()
    monkeypatch.delenv("DC_TUNING_CACHE")
    # malformed files and invalid schedules are refused and change nothing
    bad = tmp_path / "bad.json"
    for body in ('{"format": "dc_tuning/1", "fft": {"3": 2}}', "not json", '{"format": "other"}'):
        bad.write_text(body)
        with pytest.raises(dcg.DcError):
            dcg.dc_tuning_load(ctx, str(bad))
    assert dcg.dc_tuning_get(ctx)["resample_q"] == 4
    dcg.dc_tuning_set(ctx, None)
