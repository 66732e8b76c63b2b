"""GB300 Doppler resampling and FFT ionospheric correction (arXiv 2508.04951).

Thin ctypes binding over the C ABI of ``libdc.so`` (``include/dc.h``): the
functions here carry the C entry points' names and only marshal arguments
(torch tensors -> device pointers, the current torch stream -> cudaStream_t,
host lists -> C arrays).  Every step of the computation runs in the library's
CUDA kernels; there is no CPU path.  If the library has not been built the
import of a function that needs it raises immediately.

PyTorch is used for device memory and streams only.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "DcError", "Context", "load", "lib_path",
    "DC_WINDOWED", "DC_EXACT_FP32", "DC_EXACT_BF16X3", "DC_EXACT_FP16X3", "DC_FREQCONV",
    "ITEM_DTYPE", "dc_opts_default", "dc_check", "dc_launch_count", "dc_profile_enable",
    "dc_profile_read", "doppler_resample", "iono_correct", "iono_correct_noalloc",
    "correct_batch", "correct_bank", "correct_compress", "correct_compress_bank",
    "predistort_lfm", "DC_LFM_PLAIN", "DC_LFM_CUBIC", "DC_LFM_POLY", "DC_LFM_POLY_ORIGINAL",
    "resample_exact_batch", "exported_symbols",
    "Plan", "dc_plan_batch", "dc_plan_bank", "dc_plan_execute", "dc_plan_launches",
    "dc_plan_destroy", "Server", "dc_serve_start", "dc_serve_submit", "dc_serve_wait",
    "dc_serve_cancel", "dc_serve_stats", "dc_serve_stop", "dc_serve_counters",
]

DC_WINDOWED, DC_EXACT_FP32, DC_EXACT_BF16X3, DC_EXACT_FP16X3, DC_FREQCONV = 0, 1, 2, 3, 4
DC_LFM_PLAIN, DC_LFM_CUBIC, DC_LFM_POLY, DC_LFM_POLY_ORIGINAL = 0, 1, 2, 3
STATUS = {0: "DC_OK", 1: "DC_EINVAL", 2: "DC_ENOMEM", 3: "DC_EBUSY", 4: "DC_ECUDA",
          5: "DC_ETIMEOUT", 6: "DC_ECANCELLED"}

# dc_item: 4 x int64 then 4 x double (64 bytes)
ITEM_DTYPE = np.dtype([("in_off", "<i8"), ("n", "<i8"), ("out_off", "<i8"), ("n_out", "<i8"),
                       ("fs", "<f8"), ("fc", "<f8"), ("v_r", "<f8"), ("tec_tecu", "<f8")])


class DcOpts(ctypes.Structure):
    _fields_ = [("taps", ctypes.c_int), ("kaiser_beta", ctypes.c_double),
                ("mode", ctypes.c_int), ("n_out", ctypes.c_longlong),
                ("carrier_shift", ctypes.c_int), ("freq_ref", ctypes.c_double)]


class DcTuning(ctypes.Structure):
    _fields_ = [("resample_q", ctypes.c_int), ("fft", ctypes.c_int * 21),
                ("chunk", ctypes.c_longlong * 21), ("ms_default", ctypes.c_double),
                ("ms_best", ctypes.c_double), ("candidates", ctypes.c_int),
                ("resample_tc", ctypes.c_int), ("apply_kind", ctypes.c_int)]


class DcServeInfo(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("waited_memory", ctypes.c_longlong), ("waited_slot", ctypes.c_longlong),
                ("pool_bytes", ctypes.c_size_t), ("peak_bytes_in_flight", ctypes.c_size_t),
                ("batch_capacity", ctypes.c_longlong)]


class DcPhaseTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong),
                ("samples", ctypes.c_longlong), ("ms", ctypes.c_double)]


class DcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


def lib_path() -> str:
    """libdc.so, or its checked build when the environment sets DC_CHECKED=1."""
    return _build.LIB_CHECKED if os.environ.get("DC_CHECKED") == "1" else _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libdc.so (building it first when asked).  Raises when absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(
                f"CUDA library {path} is not built; run paper_2508_04951_gb300.build.build() "
                "(or __graft_entry__.build()) first")
        _build.build(checked=path == _build.LIB_CHECKED)
    lib = ctypes.CDLL(path)
    vp, ll, d, i = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double, ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "dc_opts_default": (None, [ctypes.POINTER(DcOpts)]),
        "dc_status_str": (ctypes.c_char_p, [i]),
        "dc_create": (i, [ctypes.POINTER(vp), i, ctypes.c_size_t]),
        "dc_destroy": (i, [vp]),
        "dc_last_error": (ctypes.c_char_p, [vp]),
        "dc_check": (i, [vp, vp]),
        "dc_selftest_wait_timeout": (i, [vp, vp]),
        "dc_launch_count": (ll, [vp]),
        "dc_profile_enable": (i, [vp, i]),
        "dc_profile_read": (i, [vp, ctypes.POINTER(DcPhaseTime), i]),
        "doppler_resample": (i, [vp, vp, ll, vp, d, d, d, ctypes.POINTER(DcOpts), vp]),
        "iono_correct": (i, [vp, vp, ll, vp, d, d, d, vp]),
        "iono_correct_noalloc": (i, [vp, ll, vp, d, d, d, vp]),
        "correct_batch": (i, [vp, vp, vp, vp, i, ctypes.POINTER(DcOpts), vp]),
        "correct_bank": (i, [vp, vp, ll, dp, i, dp, i, vp, d, d, ctypes.POINTER(DcOpts), vp]),
        "predistort_lfm": (i, [vp, vp, ll, d, d, d, d, d, d, i, vp]),
        "correct_compress": (i, [vp, vp, ll, vp, ll, vp, d, d, d, d, ctypes.POINTER(DcOpts), vp]),
        "correct_compress_bank": (i, [vp, vp, ll, vp, ll, dp, i, dp, i, vp, d, d,
                                      ctypes.POINTER(DcOpts), vp]),
        "resample_exact_batch": (i, [vp, vp, ll, i, ll, dp, i, vp, ll, i, vp]),
        "dc_plan_batch": (i, [vp, vp, vp, vp, i, ctypes.POINTER(DcOpts), ctypes.POINTER(vp)]),
        "dc_plan_bank": (i, [vp, vp, ll, dp, i, dp, i, vp, d, d, ctypes.POINTER(DcOpts),
                             ctypes.POINTER(vp)]),
        "dc_plan_execute": (i, [vp, vp]),
        "dc_plan_launches": (ll, [vp]),
        "dc_plan_destroy": (i, [vp]),
        "dc_serve_start": (i, [i, ctypes.c_size_t, i, ctypes.POINTER(DcOpts), ctypes.POINTER(vp)]),
        "dc_serve_submit": (i, [vp, vp, ll, d, d, d, d, vp, ctypes.POINTER(ll)]),
        "dc_serve_wait": (i, [vp, ll, i, ctypes.POINTER(d)]),
        "dc_serve_cancel": (i, [vp, ll]),
        "dc_serve_stats": (i, [vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d),
                               ctypes.POINTER(ll)]),
        "dc_serve_stop": (i, [vp]),
        "dc_serve_counters": (i, [vp, ctypes.POINTER(DcServeInfo)]),
        "dc_autotune_batch": (i, [vp, vp, vp, vp, i, ctypes.POINTER(DcOpts), vp,
                                  ctypes.POINTER(DcTuning)]),
        "dc_autotune_bank": (i, [vp, vp, ll, dp, i, dp, i, vp, d, d, ctypes.POINTER(DcOpts), vp,
                                 ctypes.POINTER(DcTuning)]),
        "dc_tuning_get": (i, [vp, ctypes.POINTER(DcTuning)]),
        "dc_tuning_set": (i, [vp, ctypes.POINTER(DcTuning)]),
        "dc_tuning_save": (i, [vp, ctypes.c_char_p]),
        "dc_tuning_load": (i, [vp, ctypes.c_char_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    """Names of the C entry points this binding binds (all declared in dc.h)."""
    return ["dc_opts_default", "dc_status_str", "dc_create", "dc_destroy", "dc_last_error",
            "dc_check", "dc_launch_count", "dc_profile_enable", "dc_profile_read", "doppler_resample", "iono_correct", "iono_correct_noalloc", "correct_batch", "correct_bank",
            "correct_compress", "correct_compress_bank", "predistort_lfm",
            "resample_exact_batch", "dc_plan_batch", "dc_plan_bank", "dc_plan_execute",
            "dc_plan_launches", "dc_plan_destroy", "dc_serve_start", "dc_serve_submit",
            "dc_serve_wait", "dc_serve_cancel", "dc_serve_stats", "dc_serve_stop",
            "dc_serve_counters"]


# ---------------------------------------------------------------- helpers

def _ptr(t, pinned_ok: bool = False) -> int:
    """Device address of a contiguous complex64 tensor: a CUDA tensor, or
    (pinned_ok) a page-locked host tensor, which the GPU addresses directly."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda and not (pinned_ok and t.is_pinned()):
        raise ValueError("expected a CUDA tensor" + (" or a pinned host tensor" if pinned_ok else ""))
    if t.dtype != torch.complex64:
        raise TypeError(f"expected complex64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _opts(taps=32, beta=8.0, mode=DC_WINDOWED, n_out=0, carrier_shift=False,
          freq_ref=0.0) -> DcOpts:
    return DcOpts(int(taps), float(beta), int(mode), int(n_out), int(bool(carrier_shift)),
                  float(freq_ref))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """Owns a dc_ctx (twiddle tables and scratch) on one device."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.dc_create(ctypes.byref(h), int(device), int(budget_bytes))
        if st:
            raise DcError(st, f"dc_create(device={device}) failed")
        self.handle = h

    def check(self, st: int):
        if st:
            msg = self.lib.dc_last_error(self.handle).decode()
            raise DcError(st, msg)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.dc_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dc_opts_default() -> DcOpts:
    o = DcOpts()
    load().dc_opts_default(ctypes.byref(o))
    return o


def dc_check(ctx: Context, stream=None) -> None:
    ctx.check(ctx.lib.dc_check(ctx.handle, _stream(stream)))


def dc_selftest_wait_timeout(ctx: Context, stream=None) -> None:
    """Queue a kernel whose bounded wait runs out; the next dc_check raises
    DcError with status DC_ETIMEOUT and the context stays usable."""
    ctx.check(ctx.lib.dc_selftest_wait_timeout(ctx.handle, _stream(stream)))


def dc_launch_count(ctx: Context) -> int:
    return int(ctx.lib.dc_launch_count(ctx.handle))


def dc_profile_enable(ctx: Context, on: bool = True) -> None:
    ctx.check(ctx.lib.dc_profile_enable(ctx.handle, int(bool(on))))


def dc_profile_read(ctx: Context) -> dict:
    """{phase name: (launches, samples, total ms)} of the profiled calls."""
    buf = (DcPhaseTime * 32)()
    n = ctx.lib.dc_profile_read(ctx.handle, buf, 32)
    if n < 0:
        raise DcError(1, "dc_profile_read failed")
    return {buf[i].name.decode(): (buf[i].launches, buf[i].samples, buf[i].ms) for i in range(min(n, 32))}


def doppler_resample(ctx: Context, x, y, fs: float, fc: float, v_r: float, *, taps=32,
                     beta=8.0, mode=DC_WINDOWED, n_out=0, carrier_shift=False, freq_ref=0.0,
                     stream=None) -> None:
    o = _opts(taps, beta, mode, n_out, carrier_shift, freq_ref)
    ctx.check(ctx.lib.doppler_resample(ctx.handle, _ptr(x), x.numel(), _ptr(y), fs, fc, v_r,
                                       ctypes.byref(o), _stream(stream)))


def iono_correct(ctx: Context, x, y, fs: float, fc: float, tec_tecu: float, *, stream=None) -> None:
    ctx.check(ctx.lib.iono_correct(ctx.handle, _ptr(x), x.numel(), _ptr(y), fs, fc, tec_tecu,
                                   _stream(stream)))


NOALLOC_MAX = 1 << 18


def iono_correct_noalloc(x, y, fs: float, fc: float, tec_tecu: float, *, stream=None) -> None:
    """iono_correct without a context and without any device allocation, for
    callers that may not allocate device memory at run time (fixed-size
    scratch inside the library; n <= 2^18).  Calls that overlap on the GPU
    share that scratch, so keep them on one stream."""
    import torch
    lib = load()
    n = x.numel()
    if n > NOALLOC_MAX:
        raise DcError(1, f"n = {n} exceeds the {NOALLOC_MAX}-sample static scratch of "
                         "iono_correct_noalloc; use iono_correct with a Context")
    xp, yp = _ptr(x), _ptr(y)
    if y.numel() < n:
        raise DcError(1, f"output holds {y.numel()} samples, the input {n}")
    if x.device != y.device:
        raise DcError(1, f"input on {x.device}, output on {y.device}")
    # the C entry point runs on the current device: make it the tensors' one
    with torch.cuda.device(x.device):
        st = lib.iono_correct_noalloc(xp, n, yp, fs, fc, tec_tecu, _stream(stream))
    if st:
        raise DcError(st, "iono_correct_noalloc rejected its arguments or failed")


def correct_batch(ctx: Context, inp, out, items, *, taps=32, beta=8.0, mode=DC_WINDOWED,
                  carrier_shift=False, freq_ref=0.0, stream=None) -> None:
    """items: numpy array of ITEM_DTYPE (or anything convertible to it)."""
    it = np.ascontiguousarray(np.asarray(items, dtype=ITEM_DTYPE))
    o = _opts(taps, beta, mode, 0, carrier_shift, freq_ref)
    ctx.check(ctx.lib.correct_batch(ctx.handle, _ptr(inp), _ptr(out), it.ctypes.data, len(it),
                                    ctypes.byref(o), _stream(stream)))


def correct_bank(ctx: Context, x, v_r, tec_tecu, out, fs: float, fc: float, *, taps=32,
                 beta=8.0, n_out=0, mode=DC_WINDOWED, carrier_shift=False, freq_ref=0.0,
                 stream=None) -> None:
    v = np.ascontiguousarray(np.asarray(v_r, dtype=np.float64))
    t = np.ascontiguousarray(np.asarray(tec_tecu, dtype=np.float64))
    o = _opts(taps, beta, mode, n_out, carrier_shift, freq_ref)
    ctx.check(ctx.lib.correct_bank(ctx.handle, _ptr(x), x.numel(), _dptr(v), len(v), _dptr(t),
                                   len(t), _ptr(out, pinned_ok=True), fs, fc, ctypes.byref(o),
                                   _stream(stream)))


def correct_compress(ctx: Context, x, replica, y, fs: float, fc: float, v_r: float, tec_tecu: float, *,
                     taps=32, beta=8.0, mode=DC_WINDOWED, n_out=0, carrier_shift=False, freq_ref=0.0,
                     stream=None) -> None:
    """Resample, correct and compress one pulse against `replica` (matched
    filter in the same frequency-domain pass); y receives the n_out lags."""
    o = _opts(taps, beta, mode, n_out, carrier_shift, freq_ref)
    ctx.check(ctx.lib.correct_compress(ctx.handle, _ptr(x), x.numel(), _ptr(replica), replica.numel(),
                                       _ptr(y), fs, fc, v_r, tec_tecu, ctypes.byref(o), _stream(stream)))


def correct_compress_bank(ctx: Context, x, replica, v_r, tec_tecu, out, fs: float, fc: float, *,
                          taps=32, beta=8.0, n_out=0, mode=DC_WINDOWED, carrier_shift=False,
                          freq_ref=0.0, stream=None) -> None:
    v = np.ascontiguousarray(np.asarray(v_r, dtype=np.float64))
    t = np.ascontiguousarray(np.asarray(tec_tecu, dtype=np.float64))
    o = _opts(taps, beta, mode, n_out, carrier_shift, freq_ref)
    ctx.check(ctx.lib.correct_compress_bank(ctx.handle, _ptr(x), x.numel(), _ptr(replica),
                                            replica.numel(), _dptr(v), len(v), _dptr(t), len(t),
                                            _ptr(out, pinned_ok=True), fs, fc, ctypes.byref(o),
                                            _stream(stream)))


def predistort_lfm(ctx: Context, y, fs: float, f0: float, bandwidth: float, T: float, tec_tecu: float,
                   *, f_mix: float = 0.0, kind=DC_LFM_CUBIC, stream=None) -> None:
    """Fill y (complex64, its length = samples) with a predistorted LFM
    transmit waveform (kind: DC_LFM_PLAIN / _CUBIC / _POLY / _POLY_ORIGINAL)."""
    ctx.check(ctx.lib.predistort_lfm(ctx.handle, _ptr(y), y.numel(), fs, f0, bandwidth, T, tec_tecu,
                                     f_mix, int(kind), _stream(stream)))


def resample_exact_batch(ctx: Context, x, n: int, n_pulses: int, v_r, y, *, n_out=0,
                         x_alpha_stride=0, mode=DC_EXACT_FP32, stream=None) -> None:
    v = np.ascontiguousarray(np.asarray(v_r, dtype=np.float64))
    ctx.check(ctx.lib.resample_exact_batch(ctx.handle, _ptr(x), int(n), int(n_pulses),
                                           int(x_alpha_stride), _dptr(v), len(v), _ptr(y),
                                           int(n_out), int(mode), _stream(stream)))


# ------------------------------------------------------------------- plans

class Plan:
    """A correct_batch / correct_bank call recorded into a CUDA graph.  Keeps
    references to the tensors and host lists it was built from."""

    def __init__(self, ctx: Context, handle, keep):
        self.ctx, self.handle, self._keep = ctx, handle, keep

    def execute(self, stream=None) -> None:
        dc_plan_execute(self, stream=stream)

    @property
    def launches(self) -> int:
        return dc_plan_launches(self)

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.dc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dc_plan_batch(ctx: Context, inp, out, items, *, taps=32, beta=8.0, mode=DC_WINDOWED,
                  carrier_shift=False, freq_ref=0.0) -> Plan:
    it = np.ascontiguousarray(np.asarray(items, dtype=ITEM_DTYPE))
    o = _opts(taps, beta, mode, 0, carrier_shift, freq_ref)
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.dc_plan_batch(ctx.handle, _ptr(inp), _ptr(out), it.ctypes.data, len(it),
                                    ctypes.byref(o), ctypes.byref(h)))
    return Plan(ctx, h, (inp, out, it))


def dc_plan_bank(ctx: Context, x, v_r, tec_tecu, out, fs: float, fc: float, *, taps=32, beta=8.0,
                 n_out=0, mode=DC_WINDOWED, carrier_shift=False, freq_ref=0.0) -> Plan:
    v = np.ascontiguousarray(np.asarray(v_r, dtype=np.float64))
    t = np.ascontiguousarray(np.asarray(tec_tecu, dtype=np.float64))
    o = _opts(taps, beta, mode, n_out, carrier_shift, freq_ref)
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.dc_plan_bank(ctx.handle, _ptr(x), x.numel(), _dptr(v), len(v), _dptr(t), len(t),
                                   _ptr(out, pinned_ok=True), fs, fc, ctypes.byref(o), ctypes.byref(h)))
    return Plan(ctx, h, (x, out, v, t))


def dc_plan_execute(plan: Plan, stream=None) -> None:
    plan.ctx.check(plan.ctx.lib.dc_plan_execute(plan.handle, _stream(stream)))


def dc_plan_launches(plan: Plan) -> int:
    return int(plan.ctx.lib.dc_plan_launches(plan.handle))


def dc_plan_destroy(plan: Plan) -> None:
    plan.close()


# ------------------------------------------------------------------ serving

class Server:
    """A dc_server: continuous-batching request loop on one device.  Host
    buffers of submitted requests are kept referenced until waited for."""

    def __init__(self, handle, lib):
        self.handle, self.lib = handle, lib
        self._keep = {}

    def submit(self, x, y, fs, fc, v_r, tec_tecu) -> int:
        return dc_serve_submit(self, x, y, fs, fc, v_r, tec_tecu)

    def wait(self, req_id, timeout_ms=-1) -> float:
        return dc_serve_wait(self, req_id, timeout_ms)

    def stats(self) -> dict:
        return dc_serve_stats(self)

    def stop(self):
        dc_serve_stop(self)

    def counters(self) -> dict:
        return dc_serve_counters(self)

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def _host_c64(a, name):
    if not isinstance(a, np.ndarray) or a.dtype != np.complex64 or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a contiguous complex64 numpy array")
    return a.ctypes.data


def dc_serve_start(device: int = 0, budget_bytes: int = 0, slots: int = 3, *, taps=32, beta=8.0,
                   mode=DC_WINDOWED, carrier_shift=False, freq_ref=0.0) -> Server:
    lib = load()
    o = _opts(taps, beta, mode, 0, carrier_shift, freq_ref)
    h = ctypes.c_void_p()
    st = lib.dc_serve_start(int(device), int(budget_bytes), int(slots), ctypes.byref(o), ctypes.byref(h))
    if st:
        raise DcError(st, "dc_serve_start failed")
    return Server(h, lib)


def dc_serve_submit(srv: Server, x, y, fs, fc, v_r, tec_tecu) -> int:
    rid = ctypes.c_longlong()
    st = srv.lib.dc_serve_submit(srv.handle, _host_c64(x, "x"), x.size, float(fs), float(fc), float(v_r),
                                 float(tec_tecu), _host_c64(y, "y"), ctypes.byref(rid))
    if st:
        raise DcError(st, "dc_serve_submit rejected the request")
    srv._keep[rid.value] = (x, y)
    return rid.value


def dc_serve_wait(srv: Server, req_id: int, timeout_ms: int = -1) -> float:
    lat = ctypes.c_double()
    st = srv.lib.dc_serve_wait(srv.handle, int(req_id), int(timeout_ms), ctypes.byref(lat))
    if st == 5:
        raise DcError(st, f"request {req_id} still running")
    srv._keep.pop(req_id, None)
    if st:
        raise DcError(st, f"request {req_id} failed")
    return lat.value


def dc_serve_cancel(srv: Server, req_id: int) -> None:
    st = srv.lib.dc_serve_cancel(srv.handle, int(req_id))
    if st:
        raise DcError(st, f"request {req_id} could not be cancelled")


def dc_serve_stats(srv: Server) -> dict:
    p50, p99, msps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_longlong()
    st = srv.lib.dc_serve_stats(srv.handle, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(msps),
                                ctypes.byref(n))
    if st:
        raise DcError(st, "dc_serve_stats failed")
    return {"p50_s": p50.value, "p99_s": p99.value, "msamples_per_s": msps.value, "completed": n.value}


def dc_serve_counters(srv: Server) -> dict:
    """Admission counters: batches, completed, waited_memory (requests held
    back by the HBM budget), waited_slot, pool_bytes, peak_bytes_in_flight,
    batch_capacity."""
    info = DcServeInfo()
    st = srv.lib.dc_serve_counters(srv.handle, ctypes.byref(info))
    if st:
        raise DcError(st, "dc_serve_counters failed")
    return {f: getattr(info, f) for f, _ in DcServeInfo._fields_}


def dc_serve_stop(srv: Server) -> None:
    if getattr(srv, "handle", None):
        srv.lib.dc_serve_stop(srv.handle)
        srv.handle = None
        srv._keep.clear()


# ----------------------------------------------------------- autotuning

def _tuning_dict(t: DcTuning) -> dict:
    return {"resample_q": t.resample_q, "resample_tc": t.resample_tc, "apply_kind": t.apply_kind,
            "fft": {m: t.fft[m] for m in range(21) if t.fft[m]},
            "chunk": {m: t.chunk[m] for m in range(21) if t.chunk[m]},
            "ms_default": t.ms_default, "ms_best": t.ms_best, "candidates": t.candidates}


def dc_autotune_batch(ctx: Context, inp, out, items, *, taps=32, beta=8.0, mode=DC_WINDOWED,
                      stream=None) -> dict:
    """Time the schedule choices of this correct_batch call on its data and keep
    the fastest in the context (outputs written); returns the schedule."""
    it = np.ascontiguousarray(np.asarray(items, dtype=ITEM_DTYPE))
    o = _opts(taps, beta, mode, 0)
    t = DcTuning()
    ctx.check(ctx.lib.dc_autotune_batch(ctx.handle, _ptr(inp), _ptr(out), it.ctypes.data, len(it),
                                        ctypes.byref(o), _stream(stream), ctypes.byref(t)))
    return _tuning_dict(t)


def dc_autotune_bank(ctx: Context, x, v_r, tec_tecu, out, fs: float, fc: float, *, taps=32,
                     beta=8.0, n_out=0, stream=None) -> dict:
    """As dc_autotune_batch for a correct_bank call."""
    v = np.ascontiguousarray(v_r, dtype=np.float64)
    tt = np.ascontiguousarray(tec_tecu, dtype=np.float64)
    o = _opts(taps, beta, DC_WINDOWED, n_out)
    t = DcTuning()
    ctx.check(ctx.lib.dc_autotune_bank(ctx.handle, _ptr(x), x.numel(), _dptr(v), len(v), _dptr(tt),
                                       len(tt), _ptr(out, pinned_ok=True), fs, fc, ctypes.byref(o),
                                       _stream(stream), ctypes.byref(t)))
    return _tuning_dict(t)


def dc_tuning_get(ctx: Context) -> dict:
    t = DcTuning()
    ctx.check(ctx.lib.dc_tuning_get(ctx.handle, ctypes.byref(t)))
    return _tuning_dict(t)


def dc_tuning_set(ctx: Context, schedule: dict | None) -> None:
    """Replace the context's schedule ({"resample_q", "resample_tc", "apply_kind",
    "fft": {m: v}, "chunk": {m: bytes}});
    None restores the built-in rules."""
    if schedule is None:
        ctx.check(ctx.lib.dc_tuning_set(ctx.handle, None))
        return
    t = DcTuning()
    t.resample_q = int(schedule.get("resample_q", 0))
    t.resample_tc = int(schedule.get("resample_tc", 0))
    t.apply_kind = int(schedule.get("apply_kind", 0))
    for m, v in schedule.get("fft", {}).items():
        t.fft[int(m)] = int(v)
    for m, v in schedule.get("chunk", {}).items():
        t.chunk[int(m)] = int(v)
    ctx.check(ctx.lib.dc_tuning_set(ctx.handle, ctypes.byref(t)))



def dc_tuning_save(ctx: Context, path: str) -> None:
    """Write the context's schedule to a JSON file (dc_tuning/1)."""
    st = ctx.lib.dc_tuning_save(ctx.handle, os.fsencode(path))
    if st:
        raise DcError(st, f"could not write {path}")


def dc_tuning_load(ctx: Context, path: str) -> None:
    """Apply a schedule written by dc_tuning_save."""
    ctx.check(ctx.lib.dc_tuning_load(ctx.handle, os.fsencode(path)))
