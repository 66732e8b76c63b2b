// iono_correct_noalloc: the ionospheric correction of iono_correct for
// callers that must not allocate device memory at run time.
//
// Everything this entry point touches on the device, apart from the caller's
// input and output, lives in file-scope __device__ arrays of fixed size: the
// four-step scratch (kNoAllocMax samples, 2 MiB), the twiddle tables (80 KiB)
// and the launch descriptors.  Each GPU that loads the library holds one copy of
// them until the process exits; nothing is allocated or freed per call.
//
// Host code cannot use these arrays' names as device addresses (in host code
// the name refers to a host-side shadow).  The first call on a device looks
// up their device addresses with cudaGetSymbolAddress while that device is
// current, fills the twiddle tables with a synchronous copy, and caches the
// addresses per device; later calls reuse them.  A call's launch descriptors
// travel as kernel parameters (by value) into a one-thread kernel that writes
// them into the descriptor array, so no host memory is read after the call
// returns.
#include <cmath>
#include <mutex>

#include "../../include/dc.h"
#include "fft.cuh"
#include "phase.cuh"
#include "twiddle_host.h"

namespace {

constexpr int kLog2NoAllocMax = 18;
constexpr long long kNoAllocMax = 1LL << kLog2NoAllocMax;   // samples
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_scratch[kNoAllocMax];
static __device__ __align__(256) float2 g_twiddle[dc::kTwSize];
static __device__ __align__(256) dc::FftItem g_items[3];

struct DeviceSlots {
  bool ready = false;
  float2* scratch = nullptr;
  float2* twiddle = nullptr;
  dc::FftItem* items = nullptr;
};

std::mutex g_mu;
DeviceSlots g_dev[kMaxDevices];

constexpr double kPi = 3.14159265358979323846;
constexpr double kC = 299792458.0;

// First use on the current device: resolve the arrays' device addresses and
// write the twiddle tables (same layout and values as a dc_ctx's tables).
dc_status prepare(int device, DeviceSlots** out) {
  std::lock_guard<std::mutex> g(g_mu);
  DeviceSlots& d = g_dev[device];
  if (!d.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return DC_ECUDA;
    d.scratch = static_cast<float2*>(p);
    if (cudaGetSymbolAddress(&p, g_twiddle) != cudaSuccess) return DC_ECUDA;
    d.twiddle = static_cast<float2*>(p);
    if (cudaGetSymbolAddress(&p, g_items) != cudaSuccess) return DC_ECUDA;
    d.items = static_cast<dc::FftItem*>(p);
    static float2 tw[dc::kTwSize];
    dc::fill_twiddles(tw);
    if (cudaMemcpy(d.twiddle, tw, sizeof tw, cudaMemcpyHostToDevice) != cudaSuccess)
      return DC_ECUDA;
    d.ready = true;
  }
  *out = &d;
  return DC_OK;
}

// Writes this call's descriptors into the static descriptor array, which
// device code of this file may name directly.
__global__ void set_items_kernel(dc::FftItem a, dc::FftItem b, dc::FftItem c, int count) {
  g_items[0] = a;
  if (count > 1) {
    g_items[1] = b;
    g_items[2] = c;
  }
}

void split(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

}  // namespace

extern "C" dc_status iono_correct_noalloc(const dc_c64* x, long long n, dc_c64* y, double fs,
                                          double fc, double tec_tecu, void* stream) {
  if (!x || !y) return DC_EINVAL;
  if (n < 1 || n > kNoAllocMax) return DC_EINVAL;      // beyond the static scratch
  if (!(fs > 0.0) || !std::isfinite(fs) || !(fc >= 0.0) || !std::isfinite(fc) ||
      (fc != 0.0 && !(fc > fs / 2.0)) || !std::isfinite(tec_tecu))
    return DC_EINVAL;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
    return DC_ECUDA;
  DeviceSlots* d = nullptr;
  dc_status st = prepare(device, &d);
  if (st) return st;

  int log2L = 0;
  while ((1LL << log2L) < n) ++log2L;
  const double kappa = [] {
    const double e = 1.602176634e-19, me = 9.1093837015e-31, eps0 = 8.8541878128e-12;
    return e * e / (8.0 * kPi * kPi * me * eps0);
  }();
  dc::FftItem it{};
  it.src = reinterpret_cast<const float2*>(x);
  it.dst = reinterpret_cast<float2*>(y);
  it.ptab = nullptr;
  split(4.0 * kPi * kappa * tec_tecu * 1e16 / kC, it.ph.a_hi, it.ph.a_lo);
  split(fc, it.ph.fc_hi, it.ph.fc_lo);
  split(fs / (double)(1LL << log2L), it.ph.d_hi, it.ph.d_lo);
  it.ph.log2L = log2L;
  it.ph.enabled = tec_tecu != 0.0;
  it.ph.run = 1;                               // every bin evaluated in full
  it.n_valid = (int)n;
  it.n_out = (int)n;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  dc::FftItem host_items[3] = {it, it, it};
  int count = 1;
  if (log2L > 12) {
    host_items[0].dst = d->scratch;              // F1: x -> scratch
    host_items[1].src = d->scratch;              // F2 + phase + A in place
    host_items[1].dst = d->scratch;
    host_items[2].src = d->scratch;              // B: scratch -> y
    count = 3;
  }
  set_items_kernel<<<1, 1, 0, s>>>(host_items[0], host_items[1], host_items[2], count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return DC_ECUDA;
  if (log2L <= 12) {
    dc::RowArgs a{d->items, 1, log2L, 0, d->twiddle};
    e = dc::launch_row(dc::ROW_FULL, a, s);
  } else {
    const int log2L1 = log2L - 12;
    dc::ColArgs a1{d->items + 0, 1, log2L, log2L1, d->twiddle};
    if ((e = dc::launch_col(dc::COL_F1, a1, s)) != cudaSuccess) return DC_ECUDA;
    dc::RowArgs a2{d->items + 1, 1, log2L, log2L1, d->twiddle};
    if ((e = dc::launch_row(dc::ROW_MID, a2, s)) != cudaSuccess) return DC_ECUDA;
    dc::ColArgs a3{d->items + 2, 1, log2L, log2L1, d->twiddle};
    e = dc::launch_col(dc::COL_B, a3, s);
  }
  return e == cudaSuccess ? DC_OK : DC_ECUDA;
}
