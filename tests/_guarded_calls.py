"""Representative calls of every hot-path family with guard words around
their device outputs, checked against the FP64 oracle.

Used in-process with the normal library (guard words only) and in a
subprocess with the checked library (DC_CHECKED=1: the kernels' bounds checks
raise the context's error flag, which dc_check turns into an error).  Each
output buffer is allocated with GUARD elements of a canary value before and
after the region a call may write; any write outside it changes a canary.
"""

import numpy as np

import oracle
import synth

GUARD = 4096
CANARY = complex(1234.5, -4321.25)
TOL = 1e-5
FS, FC = 20e6, 1e9


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


class Guarded:
    """A device buffer of n complex64 values between two guard zones."""

    def __init__(self, n):
        import torch
        self.n = n
        self.buf = torch.full((GUARD + n + GUARD,), CANARY, dtype=torch.complex64, device="cuda")
        self.inner = self.buf[GUARD:GUARD + n]

    def check(self, what):
        b = self.buf.cpu().numpy()
        lo, hi = b[:GUARD], b[GUARD + self.n:]
        assert np.all(lo == np.complex64(CANARY)) and np.all(hi == np.complex64(CANARY)), \
            f"{what}: a guard word changed"
        return b[GUARD:GUARD + self.n]


def run_all(dcg):
    """Runs the calls; returns (name, rel-L2 error, tolerance) triples."""
    import torch
    ctx = dcg.Context(0)
    done = []
    noise = lambda n, salt: synth.bandlimited_noise(n, synth.rng_for(31, salt=salt)).astype(np.complex64)

    # single pulse: windowed resample, then the correction (cluster-fused FULL at L = 32768)
    x = noise(20000, 1)
    xd = torch.from_numpy(x).cuda()
    y = Guarded(20000)
    dcg.doppler_resample(ctx, xd, y.inner, FS, FC, 6500.0)
    z = Guarded(20000)
    dcg.iono_correct(ctx, y.inner, z.inner, FS, FC, 80.0)
    dcg.dc_check(ctx)
    y.check("doppler_resample")
    got = z.check("iono_correct")
    ref = oracle.correct(x.astype(np.complex128), FS, FC, 6500.0, 80.0)
    done.append(("single pulse", _rel(got, ref), TOL))

    # ragged batch: tiled resampler, one-row FFT, cluster FULL, three passes (L = 2^17)
    lens = [900, 4096, 9000, 33000, 70000]
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    xb = np.concatenate([noise(n, 10 + i) for i, n in enumerate(lens)])
    v = [-7000.0, 3000.0, 7900.0, -100.0, 5000.0]
    tec = [5.0, 60.0, 150.0, 20.0, 90.0]
    items = np.zeros(len(lens), dtype=dcg.ITEM_DTYPE)
    for i, n in enumerate(lens):
        items[i] = (offs[i], n, offs[i], n, FS, FC, v[i], tec[i])
    ob = Guarded(int(sum(lens)))
    dcg.correct_batch(ctx, torch.from_numpy(xb).cuda(), ob.inner, items)
    dcg.dc_check(ctx)
    got = ob.check("correct_batch")
    for i, n in enumerate(lens):
        ref = oracle.correct(xb[offs[i]:offs[i] + n].astype(np.complex128), FS, FC, v[i], tec[i])
        done.append((f"batch item n={n}", _rel(got[offs[i]:offs[i] + n], ref), TOL))

    # the bank on every spectrum-apply form: tensor-core resampling, spectra,
    # factor tables, two-pass apply (more transforms than its scratch holds),
    # cluster apply with one and with two rows per CTA
    n = 65536
    xk = noise(n, 40)
    vb = np.linspace(-7900.0, 7900.0, 10)
    tb = np.linspace(5.0, 150.0, 8)
    ref = oracle.correct_bank(xk.astype(np.complex128), FS, FC, vb[[0, -1]], tb[[0, -1]])
    for kind in (3, 1, 2):
        dcg.dc_tuning_set(ctx, {"apply_kind": kind})
        ok = Guarded(len(vb) * len(tb) * n)
        dcg.correct_bank(ctx, torch.from_numpy(xk).cuda(), vb, tb, ok.inner, FS, FC)
        dcg.dc_check(ctx)
        got = ok.check(f"correct_bank apply_kind {kind}").reshape(len(vb), len(tb), n)
        for a_, i in enumerate((0, len(vb) - 1)):
            for b_, t in enumerate((0, len(tb) - 1)):
                done.append((f"bank kind {kind} ({i},{t})", _rel(got[i, t], ref[a_, b_]), TOL))
    dcg.dc_tuning_set(ctx, None)

    # exact sinc on tensor cores (bf16 hi/lo), a few pulses per range rate
    P, ne = 64, 2048
    xe = np.stack([noise(ne, 60 + p) for p in range(P)])
    ve = [-6000.0, 7000.0]
    oe = Guarded(len(ve) * P * ne)
    dcg.resample_exact_batch(ctx, torch.from_numpy(xe.reshape(-1)).cuda(), ne, P, ve, oe.inner,
                             mode=dcg.DC_EXACT_BF16X3)
    dcg.dc_check(ctx)
    got = oe.check("resample_exact_batch").reshape(len(ve), P, ne)
    for i in range(len(ve)):
        for p in (0, P - 1):
            r = oracle.resample_exact(xe[p].astype(np.complex128), oracle.alpha(ve[i]), ne)
            done.append((f"exact tc v={ve[i]} p={p}", _rel(got[i, p], r), 1e-3))   # bf16x3 bar
    ctx.close()
    return done


def main():
    import paper_2508_04951_gb300 as dcg
    dcg.build.build(checked=True)
    dcg.load()
    assert dcg.lib_path().endswith("_build_checked/libdc.so"), dcg.lib_path()
    res = run_all(dcg)
    for name, e, tol in res:
        assert e <= tol, (name, e, tol)
    print(f"CHECKED OK {len(res)} results")


if __name__ == "__main__":
    main()
