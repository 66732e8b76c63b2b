"""GPU tests of the batch/bank plans (CUDA graphs) and the serving loop.

Plans must reproduce the direct calls bitwise (same kernels, same order).
The server must return, for every request of a concurrent mixed stream, the
result the FP64 oracle gives (rel-L2 <= 1e-5) and bitwise the result of the
same request corrected alone.
"""

import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


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
    return synth.bandlimited_noise(n, synth.rng_for(5, salt=salt)).astype(np.complex64)


def test_plan_batch_matches_direct_call(dcg, ctx):
    import torch
    lengths = [700, 4096, 5000, 70000, 200000, 3, 65536]
    rng = np.random.default_rng(1)
    items = np.zeros(len(lengths), dtype=dcg.ITEM_DTYPE)
    xs, off = [], 0
    for i, n in enumerate(lengths):
        xs.append(noise(n, i))
        items[i] = (off, n, off, n, 20e6, 1e9, rng.uniform(-8000, 8000), rng.uniform(5, 150))
        off += n
    x = torch.from_numpy(np.concatenate(xs)).cuda()
    direct = torch.zeros_like(x)
    dcg.correct_batch(ctx, x, direct, items)
    out = torch.zeros_like(x)
    plan = dcg.dc_plan_batch(ctx, x, out, items)
    assert plan.launches > 0
    out.zero_()
    plan.execute()
    plan.execute()
    torch.cuda.synchronize()
    assert torch.equal(out, direct)
    plan.close()


def test_plan_bank_matches_direct_call(dcg, ctx):
    import torch
    x = torch.from_numpy(noise(65536, 9)).cuda()
    v = np.linspace(-8000, 8000, 8)
    tec = np.array([5.0, 77.0, 150.0])
    direct = torch.empty(8 * 3 * 65536, dtype=torch.complex64, device="cuda")
    dcg.correct_bank(ctx, x, v, tec, direct, 20e6, 1e9)
    out = torch.zeros_like(direct)
    plan = dcg.dc_plan_bank(ctx, x, v, tec, out, 20e6, 1e9)
    out.zero_()
    plan.execute()
    torch.cuda.synchronize()
    assert torch.equal(out, direct)
    plan.close()


@pytest.mark.parametrize("staged", [False, True])
def test_serve_mixed_stream_matches_alone_and_oracle(dcg, ctx, staged, monkeypatch):
    # direct: copy kernels between the callers' buffers and the pool (where
    # the device reaches pageable host memory); staged: host copies through
    # pinned staging.  Both give every request the same bits as alone.
    import torch
    if staged:
        monkeypatch.setenv("DC_SERVE_STAGED", "1")
    else:
        monkeypatch.delenv("DC_SERVE_STAGED", raising=False)
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(48):
        n = int(np.exp(rng.uniform(np.log(2048), np.log(300000))))
        reqs.append((noise(n, 100 + i), rng.uniform(-8000, 8000), rng.uniform(5, 150)))
    srv = dcg.dc_serve_start(0, 1 << 30, slots=3)
    outs = [np.zeros_like(x) for x, _, _ in reqs]
    ids = [None] * len(reqs)

    def submit(lo, hi):
        for k in range(lo, hi):
            x, v, t = reqs[k]
            ids[k] = srv.submit(x, outs[k], 20e6, 1e9, v, t)

    th = [threading.Thread(target=submit, args=(a, a + 16)) for a in (0, 16, 32)]
    for t_ in th:
        t_.start()
    for t_ in th:
        t_.join()
    lat = [srv.wait(i, 30000) for i in ids]
    st = srv.stats()
    assert st["completed"] == len(reqs) and all(l > 0 for l in lat)
    assert 0 < st["p50_s"] <= st["p99_s"]
    srv.stop()
    for k, (x, v, t) in enumerate(reqs):
        ref = oracle.correct(x.astype(np.complex128), 20e6, 1e9, v, t)
        got = outs[k].astype(np.complex128)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5, k
        # the same request alone through correct_batch
        items = np.zeros(1, dtype=dcg.ITEM_DTYPE)
        items[0] = (0, x.size, 0, x.size, 20e6, 1e9, v, t)
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        dcg.correct_batch(ctx, xd, yd, items)
        assert np.array_equal(yd.cpu().numpy(), outs[k]), k


def test_serve_rejects_cancels_and_times_out(dcg):
    srv = dcg.dc_serve_start(0, 1 << 30, slots=1)
    big = np.zeros((1 << 20) + 1, dtype=np.complex64)
    with pytest.raises(dcg.DcError):
        srv.submit(big, big, 20e6, 1e9, 0.0, 10.0)                 # n > 2^20
    x = noise(1 << 20, 3)
    y = np.zeros_like(x)
    with pytest.raises(dcg.DcError):
        srv.submit(x, y, 20e6, 5e6, 0.0, 10.0)                     # fc <= fs/2
    # fill the single slot, then queue more and cancel the last one
    ids = [srv.submit(x, np.zeros_like(x), 20e6, 1e9, 100.0 * k, 10.0) for k in range(6)]
    try:
        dcg.dc_serve_cancel(srv, ids[-1])
        cancelled = True
    except dcg.DcError:
        cancelled = False                                          # already admitted
    for i in ids[:-1]:
        srv.wait(i, 60000)
    if cancelled:
        with pytest.raises(dcg.DcError) as e:
            srv.wait(ids[-1], 1000)
        assert e.value.status == 6
    srv.stop()


def test_serve_admission_waits_for_the_hbm_budget(dcg):
    # 8 slots but a budget whose pool holds two 700k-sample requests at once
    # (each ~25 MB: input, output, resampled copy, four-step scratch): the
    # third waits for memory although slots are free, and no more than the
    # pool is ever in use
    budget = 8 * (1 << 20) + 60 * (1 << 20)
    srv = dcg.dc_serve_start(0, budget, slots=8)
    reqs = [(noise(700000, 300 + k), -8000.0 + 4000 * k, 20.0 + 30 * k) for k in range(4)]
    outs = [np.zeros_like(x) for x, _, _ in reqs]
    ids = [srv.submit(x, outs[k], 20e6, 1e9, v, t) for k, (x, v, t) in enumerate(reqs)]
    for i in ids:
        srv.wait(i, 60000)
    c = srv.counters()
    srv.stop()
    assert c["completed"] == 4
    assert c["waited_memory"] >= 1
    assert c["pool_bytes"] <= budget and 0 < c["peak_bytes_in_flight"] <= c["pool_bytes"]
    for k, (x, v, t) in enumerate(reqs):
        ref = oracle.correct(x.astype(np.complex128), 20e6, 1e9, v, t)
        assert np.linalg.norm(outs[k] - ref) / np.linalg.norm(ref) <= 1e-5, k


def test_serve_budget_too_small_for_a_full_pulse(dcg):
    with pytest.raises(dcg.DcError) as e:
        dcg.dc_serve_start(0, 16 << 20, slots=2)
    assert e.value.status == 1


def test_serve_budget_beyond_the_device_is_enomem_and_the_device_survives(dcg, ctx):
    # a budget far beyond the GPU's memory: the pool allocation fails cleanly
    # (DC_ENOMEM, nothing launched), and the device keeps working
    import torch
    with pytest.raises(dcg.DcError) as e:
        dcg.dc_serve_start(0, 1 << 50, slots=2)
    assert e.value.status == 2                       # DC_ENOMEM
    x = synth.bandlimited_noise(4096, synth.rng_for(8, salt=1)).astype(np.complex64)
    y = torch.empty(4096, dtype=torch.complex64, device="cuda")
    dcg.iono_correct(ctx, torch.from_numpy(x).cuda(), y, 20e6, 1e9, 40.0)
    dcg.dc_check(ctx)
    ref = oracle.iono_correct(x.astype(np.complex128), 20e6, 1e9, 40.0)
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5
