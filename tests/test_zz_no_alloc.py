"""iono_correct_noalloc: the context-free, allocation-free variant of
iono_correct for callers that may not allocate device memory while running.

Checked through the C ABI against iono_correct (the entry point that uses a
context and its scratch) on two calls in a row -- the second reuses the
static scratch the first one left behind -- within the FP32 tolerance of the
other parity tests.  This file sorts last so that a run stopping at the first
failure has already run every other test; it also passes alone.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def dcg():
    import paper_2508_04951_gb300 as m
    m.build.build()
    m.load()
    return m


def _pulse(n, salt):
    import torch
    x = synth.bandlimited_noise(n, synth.rng_for(1, salt=salt)).astype(np.complex64)
    return torch.from_numpy(x).to("cuda:0")


def test_noalloc_matches_context_path_twice(dcg):
    import torch
    ctx = dcg.Context(0)
    # four-step path (L = 2^17 uses the static scratch), then a single-pass one,
    # then the four-step path again on a different size.
    for n, tec, salt in ((100000, 120.0, 1), (3000, 40.0, 2), (262144, -60.0, 3)):
        x = _pulse(n, salt)
        want = torch.empty_like(x)
        got = torch.full_like(x, complex(5.0, 5.0))
        dcg.iono_correct(ctx, x, want, 20e6, 1e9, tec)
        dcg.iono_correct_noalloc(x, got, 20e6, 1e9, tec)
        torch.cuda.synchronize()
        w = want.cpu().numpy().astype(np.complex128)
        g = got.cpu().numpy().astype(np.complex128)
        assert rel(g, w) <= TOL, n
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(dcg):
    import torch
    x = torch.zeros((1 << 18) + 1, dtype=torch.complex64, device="cuda:0")
    with pytest.raises(dcg.DcError) as e:
        dcg.iono_correct_noalloc(x, x, 20e6, 1e9, 10.0)
    assert "exceeds" in str(e.value)
    # the C entry point itself refuses too (no launch)
    L = dcg.load()
    assert L.iono_correct_noalloc(x.data_ptr(), x.numel(), x.data_ptr(), 20e6, 1e9, 10.0,
                                  torch.cuda.current_stream().cuda_stream) == 1
