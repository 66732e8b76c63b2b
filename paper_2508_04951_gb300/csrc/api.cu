// C ABI of libdc.so (declared in include/dc.h): context, validation, host
// parameter arithmetic in FP64 (alpha, delta, K2, phase constants) and the
// launch sequences of each entry point.
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dc.h"
#include "exact_tc.cuh"
#include "fft.cuh"
#include "fused.cuh"
#include "internal.h"
#include "phase.cuh"
#include "predist.cuh"
#include "resample.cuh"
#include "tma.cuh"
#include "twiddle_host.h"

using namespace dc;

namespace {

constexpr double kC = 299792458.0;
// kappa = e^2 / (8 pi^2 m_e eps0), CODATA 2018 (Eq. 3)
const double kKappa = [] {
  const double e = 1.602176634e-19, me = 9.1093837015e-31, eps0 = 8.8541878128e-12;
  const double pi = 3.14159265358979323846;
  return e * e / (8.0 * pi * pi * me * eps0);
}();
constexpr double kPi = 3.14159265358979323846;
constexpr long long kMaxN = 1LL << 20;

}  // namespace

struct dc_ctx {
  int device = 0;
  size_t budget = 0;
  std::string last_error;
  float2* tw = nullptr;       // twiddle tables (kTwSize)
  float2* t4 = nullptr;       // four-step twiddles of the spectrum-apply kernel (kT4Size)
  int* err = nullptr;         // device error flag
  char* ws = nullptr;         // scratch
  size_t ws_bytes = 0;
  std::vector<void*> retired; // outgrown scratch, freed at destroy
  char* items = nullptr;      // device item arrays
  size_t items_bytes = 0;
  long long launches = 0;     // kernels launched by this context
  // While a plan is being recorded: item uploads go to this host staging
  // buffer (copied to the plan's device item buffer once the capture ends).
  std::vector<char>* rec = nullptr;
  // per-phase CUDA-event timing (dc_profile_enable / dc_profile_read)
  bool profiling = false;
  struct Rec { int phase; cudaEvent_t a, b; long long samples; };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> pending;
  static constexpr int kMaxPhases = 24;
  double acc_ms[kMaxPhases] = {};
  long long acc_launches[kMaxPhases] = {};
  long long acc_samples[kMaxPhases] = {};
  // Schedule decisions, 0 = the built-in rule; dc_opts.autotune measures
  // them on a call's own data (see autotune below).
  struct Tune {
    int rs_q = 0;              // outputs per lane of the tiled resampler: 8 or 4
    long long chunk[21] = {};  // three-pass intermediate bytes per chunk (-1: whole class)
    int fft[21] = {};          // 4096 <= L <= 65536: 1 cluster-fused, 2 three passes
    int rs_tc = 0;             // bank resampling: 1 tensor cores (where eligible), 2 CUDA cores
    int apply_kind = 0;        // spectrum apply: 1 cluster, one row per CTA; 2 cluster, two rows
                               // per CTA (L >= 32768); 3 two passes through L2 (L >= 8192)
  } tune;
  std::recursive_mutex mu;
};

namespace {

dc_status fail(dc_ctx* c, dc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->last_error = buf;
  return s;
}

dc_status cuda_fail(dc_ctx* c, cudaError_t e, const char* what) {
  return fail(c, DC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Kernel phases, named in dc_profile_read().
enum Ph { PH_RS_TILED, PH_RS_DIRECT, PH_EXACT, PH_ROW_FULL, PH_COL_F1, PH_ROW_MID, PH_COL_B,
          PH_ROW_SPEC, PH_ROW_APPLY, PH_PHASE_TABLE, PH_FUSED_FULL, PH_FUSED_SPEC, PH_FUSED_APPLY,
          PH_EXACT_TC, PH_FREQCONV, PH_PREDIST, PH_RS_TC, PH_COUNT };
const char* kPhaseName[PH_COUNT] = {"resample_tiled", "resample_direct", "exact_fp32", "row_full",
                                    "col_f1", "row_mid", "col_b", "row_spec", "row_apply",
                                    "phase_table", "fused_full", "fused_spec", "fused_apply",
                                    "exact_tc", "freqconv", "predistort_lfm", "resample_tc"};
// Transform lengths handled by the cluster-fused kernels.
bool fused_L(int log2L) { return log2L >= 12 && log2L <= 16; }

// The transform schedule of a length class: cluster-fused (4096 <= L <=
// 65536 unless tuned otherwise), else one row pass (L <= 4096) or three
// passes over an intermediate processed in chunks.
bool use_fused(const dc_ctx* c, int log2L) { return fused_L(log2L) && c->tune.fft[log2L] != 2; }
// Two rows per CTA in the spectrum-apply kernel (L >= 32768 only).  The
// built-in rule keeps one: on the 256 x 16 bank at L = 65536 two rows (8-CTA
// clusters, 2 CTAs per SM) ran 1.46 ms against 1.36 ms.
bool apply_rows2(const dc_ctx* c, int log2L) { return log2L >= 15 && c->tune.apply_kind == 2; }
// The spectrum apply in two passes through an L2-resident scratch (no
// clusters), for 8192 <= L <= 65536.  The built-in rule takes it at
// L = 65536, where the 16-CTA clusters' exchange costs more than the second
// pass through L2 (256 x 16 bank: 1.19 vs 1.36 ms); below, the smaller
// clusters win (L = 32768: 0.60 vs 0.57 ms; 16384: 0.30 vs 0.27 ms).
bool apply_l2(const dc_ctx* c, int log2L) {
  return log2L >= 13 && (c->tune.apply_kind == 3 || (c->tune.apply_kind == 0 && log2L == 16));
}
// Transforms per chunk of the two-pass apply: 8 MiB of them (256 row tasks),
// so that the scratch (kApplyL2Slots chunks, 32 MiB) stays in L2 beside the
// spectra and factor tables.
int apply_l2_chunk(int log2L, size_t n_pairs) {
  const size_t per = (size_t)8 << 20 >> (log2L + 3);
  return (int)std::max<size_t>(1, std::min(per, n_pairs));
}

// Transforms per chunk of a three-pass class.  The tuned intermediate size
// wins; else `dflt` bytes (0: the whole class at once -- the batch, whose
// passes lose more to small launches than they gain from L2; the bank uses
// 64 MiB, which also bounds its scratch).
size_t chunk_items(const dc_ctx* c, int log2L, size_t count, size_t dflt) {
  const long long cb = c->tune.chunk[log2L] ? c->tune.chunk[log2L] : (long long)dflt;
  if (cb <= 0) return std::max<size_t>(count, 1);
  const size_t per = ((size_t)1 << log2L) * sizeof(float2);
  return std::max<size_t>(1, std::min(count, (size_t)cb / per));
}

cudaEvent_t take_event(dc_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Counts one kernel launch; with profiling on, brackets it with events on
// the launching stream.
struct Phase {
  dc_ctx* c;
  int id;
  cudaStream_t s;
  long long samples;
  cudaEvent_t a = nullptr;
  Phase(dc_ctx* c_, int id_, cudaStream_t s_, long long samples_)
      : c(c_), id(id_), s(s_), samples(samples_) {
    ++c->launches;
    nvtxRangePushA(kPhaseName[id]);   // host-side range per phase (profilers; no cost without one)
    if (c->profiling && !c->rec) {
      a = take_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~Phase() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, s);
      c->pending.push_back({id, a, b, samples});
    }
    nvtxRangePop();
  }
};

void split(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// Rotation rate (cycles per output sample) multiplied into a resampled pulse:
// frequency conversion's tone (freq_ref, plus fc with carrier_shift) or, for
// the interpolating modes with carrier_shift, the carrier term of a passband
// dilation, fc (alpha - 1) / fs.  0 when neither applies.
double rotation_rate(const dc_opts& o, double delta, double fs, double fc) {
  double f = 0.0;
  if (o.mode == DC_FREQCONV) f = o.freq_ref + (o.carrier_shift ? fc : 0.0);
  else if (o.carrier_shift) f = fc;
  return f * delta / fs;
}

int log2_ceil(long long n) {
  int m = 0;
  while ((1LL << m) < n) ++m;
  return m;
}

double alpha_minus_one(double v_r) {
  const double b = v_r / kC;
  return (2.0 * b) / (1.0 - b);
}

// Per-pulse ionospheric constants (Eq. 16): A = 4 pi kappa E / c.
PhaseParams phase_params(double fs, double fc, double tec_tecu, int log2L) {
  PhaseParams p{};
  const double A = 4.0 * kPi * kKappa * tec_tecu * 1e16 / kC;
  split(A, p.a_hi, p.a_lo);
  split(fc, p.fc_hi, p.fc_lo);
  split(fs / (double)(1LL << log2L), p.d_hi, p.d_lo);
  p.log2L = log2L;
  p.enabled = tec_tecu != 0.0;
  // Stepped phase runs (16 bins, s d = fs / 4096): the largest step over the
  // band is |A| (fs / 4096) / f_min^2; 15 steps of relative error ~3.3e-7
  // stay within 1e-7 rad while it is <= 0.02 rad.  RF sampling (a bin at
  // f = 0) always evaluates every bin.
  p.run = 1;
  if (fc > 0.0) {
    const double fmin = fc - 0.5 * fs;
    if (fmin > 0.0 && std::fabs(A) * (fs / 4096.0) / (fmin * fmin) <= 0.02) p.run = 16;
  }
  return p;
}

// Make sure the context has `bytes` of scratch (stream-ordered: the old
// block stays allocated until destroy, since queued work may still use it).
dc_status ensure_ws(dc_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return DC_OK;
  if (c->rec) return fail(c, DC_ENOMEM, "plan scratch too small");
  if (c->budget && bytes > c->budget)
    return fail(c, DC_EBUSY, "scratch of %zu bytes exceeds the context budget of %zu", bytes,
                c->budget);
  size_t want = std::max(bytes, c->ws_bytes + c->ws_bytes / 2);
  if (c->budget) want = std::min(want, c->budget);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DC_ENOMEM, "cudaMalloc(%zu) for scratch failed: %s", want, cudaGetErrorString(e));
  }
  if (c->ws) c->retired.push_back(c->ws);
  c->ws = (char*)p;
  c->ws_bytes = want;
  return DC_OK;
}

dc_status ensure_items(dc_ctx* c, size_t bytes) {
  if (bytes <= c->items_bytes) return DC_OK;
  if (c->rec) return fail(c, DC_ENOMEM, "plan item buffer too small");
  size_t want = std::max(bytes, (size_t)1 << 16);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DC_ENOMEM, "cudaMalloc(%zu) for item lists failed", want);
  }
  if (c->items) c->retired.push_back(c->items);
  c->items = (char*)p;
  c->items_bytes = want;
  return DC_OK;
}

// Byte layout helper for one call's scratch.
struct Arena {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  }
};

// Kaiser window w(u) = I0(beta sqrt(1 - (u/R)^2)) / I0(beta), |u| <= R.
double kaiser_fp64(double u, double R, double beta) {
  const double r = u / R;
  if (std::fabs(r) > 1.0) return 0.0;
  auto i0 = [](double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 200; ++k) {
      term *= q / ((double)k * (double)k);
      sum += term;
      if (term < 1e-17 * sum) break;
    }
    return sum;
  };
  return i0(beta * std::sqrt(std::max(0.0, 1.0 - r * r))) / i0(beta);
}

// Per-tap polynomial of the window in the fractional delay e in [0, 1]:
// w(e - k) = sum_d c[d] e^d, degree kWCoef-1, interpolating at Chebyshev
// nodes of [0, 1] (solved in FP64).  Layout [tap t = k + R - 1][kWCoef].
std::vector<double> window_poly_fit(int taps, double beta) {
  const int R = taps / 2, D = kWCoef;
  std::vector<double> out((size_t)taps * D);
  const double pi = 3.14159265358979323846;
  double nodes[kWCoef];
  for (int i = 0; i < D; ++i) nodes[i] = 0.5 + 0.5 * std::cos(pi * (i + 0.5) / D);
  for (int t = 0; t < taps; ++t) {
    const int k = t - R + 1;
    double A[kWCoef][kWCoef + 1];
    for (int i = 0; i < D; ++i) {
      double p = 1.0;
      for (int d = 0; d < D; ++d, p *= nodes[i]) A[i][d] = p;
      A[i][D] = kaiser_fp64(nodes[i] - k, (double)R, beta);
    }
    for (int c = 0; c < D; ++c) {             // Gaussian elimination, partial pivoting
      int piv = c;
      for (int i = c + 1; i < D; ++i)
        if (std::fabs(A[i][c]) > std::fabs(A[piv][c])) piv = i;
      for (int d = 0; d <= D; ++d) std::swap(A[c][d], A[piv][d]);
      for (int i = c + 1; i < D; ++i) {
        const double f = A[i][c] / A[c][c];
        for (int d = c; d <= D; ++d) A[i][d] -= f * A[c][d];
      }
    }
    double coef[kWCoef];
    for (int c = D - 1; c >= 0; --c) {
      double v = A[c][D];
      for (int d = c + 1; d < D; ++d) v -= A[c][d] * coef[d];
      coef[c] = v / A[c][c];
    }
    for (int d = 0; d < D; ++d) out[(size_t)t * D + d] = coef[d];
  }
  return out;
}

std::vector<float> window_poly(int taps, double beta) {
  const std::vector<double> c = window_poly_fit(taps, beta);
  return std::vector<float>(c.begin(), c.end());
}

// The same polynomials and their first two derivatives in e, per tap
// [w (8 coefficients) | w' (7, then 0) | w'' (6, then 0, 0)].
std::vector<float> window_poly_d012(int taps, double beta) {
  const std::vector<double> c = window_poly_fit(taps, beta);
  const int D = kWCoef;
  std::vector<float> out((size_t)taps * 3 * D, 0.f);
  for (int t = 0; t < taps; ++t) {
    const double* ct = &c[(size_t)t * D];
    float* o = &out[(size_t)t * 3 * D];
    for (int d = 0; d < D; ++d) o[d] = (float)ct[d];
    for (int d = 0; d + 1 < D; ++d) o[D + d] = (float)((d + 1) * ct[d + 1]);
    for (int d = 0; d + 2 < D; ++d) o[2 * D + d] = (float)((d + 2) * (d + 1) * ct[d + 2]);
  }
  return out;
}

dc_status check_opts(dc_ctx* c, const dc_opts* o) {
  if (o->taps < 2 || o->taps > 2 * kMaxHalf || (o->taps & 1))
    return fail(c, DC_EINVAL, "taps must be even and in [2, %d], got %d", 2 * kMaxHalf, o->taps);
  if (!(o->kaiser_beta >= 0.0 && o->kaiser_beta <= 20.0))
    return fail(c, DC_EINVAL, "kaiser_beta must be in [0, 20], got %g", o->kaiser_beta);
  if (o->mode < DC_WINDOWED || o->mode > DC_FREQCONV)
    return fail(c, DC_EINVAL, "unknown mode %d", o->mode);
  if (o->carrier_shift != 0 && o->carrier_shift != 1)
    return fail(c, DC_EINVAL, "carrier_shift must be 0 or 1, got %d", o->carrier_shift);
  if (!std::isfinite(o->freq_ref)) return fail(c, DC_EINVAL, "freq_ref must be finite");
  if (o->n_out < 0 || o->n_out > kMaxN)
    return fail(c, DC_EINVAL, "n_out must be in [0, 2^20], got %lld", o->n_out);
  return DC_OK;
}

dc_status check_pulse(dc_ctx* c, long long n, long long n_out, double fs, double fc, double v_r,
                      double tec) {
  if (n < 1 || n > kMaxN) return fail(c, DC_EINVAL, "n must be in [1, 2^20], got %lld", n);
  if (n_out < 1 || n_out > kMaxN)
    return fail(c, DC_EINVAL, "n_out must be in [1, 2^20], got %lld", n_out);
  if (!(fs > 0.0) || !std::isfinite(fs)) return fail(c, DC_EINVAL, "fs must be > 0, got %g", fs);
  if (!(fc >= 0.0) || !std::isfinite(fc)) return fail(c, DC_EINVAL, "fc must be >= 0, got %g", fc);
  if (fc != 0.0 && !(fc > fs / 2.0))
    return fail(c, DC_EINVAL, "baseband needs fc > fs/2 (fc=%g, fs=%g); fc = 0 means RF samples", fc,
                fs);
  if (!(std::fabs(v_r) < kC)) return fail(c, DC_EINVAL, "|v_r| must be < c, got %g", v_r);
  if (!std::isfinite(tec)) return fail(c, DC_EINVAL, "tec must be finite");
  return DC_OK;
}

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Upload an item array to the context's device item buffer (stream-ordered;
// the pageable source may be reused as soon as this returns).
template <class T>
dc_status upload(dc_ctx* c, const std::vector<T>& v, size_t at, cudaStream_t s, const T** dev) {
  const size_t bytes = v.size() * sizeof(T);
  if (at + bytes > c->items_bytes) return fail(c, DC_ENOMEM, "item list overflow");
  if (c->rec) {
    memcpy(c->rec->data() + at, v.data(), bytes);
  } else {
    cudaError_t e = cudaMemcpyAsync(c->items + at, v.data(), bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "item upload");
  }
  *dev = reinterpret_cast<const T*>(c->items + at);
  return DC_OK;
}

// ------------------------------------------------------------ resampling
// Windowed resample of `items` (host list, tile_begin filled here).
dc_status run_windowed(dc_ctx* c, std::vector<RsItem>& items, const dc_opts& o, size_t item_at,
                       cudaStream_t s) {
  if (items.empty()) return DC_OK;
  if (o.mode == DC_FREQCONV) {
    int tiles = 0;
    long long outs = 0;
    for (auto& it : items) {
      it.tile_begin = tiles;
      tiles += (int)((it.n_out + kRsTile - 1) / kRsTile);
      outs += it.n_out;
    }
    const RsItem* dev = nullptr;
    dc_status st = upload(c, items, item_at, s, &dev);
    if (st) return st;
    RsArgs a{};
    a.items = dev;
    a.n_items = (int)items.size();
    a.n_tiles = tiles;
    a.err = c->err;
    Phase ph(c, PH_FREQCONV, s, outs);
    cudaError_t e = launch_freqconv(a, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "frequency conversion launch");
    return DC_OK;
  }
  const std::vector<float> wp = window_poly(o.taps, o.kaiser_beta);
  const float* dwp = nullptr;
  dc_status st = upload(c, wp, item_at, s, &dwp);
  if (st) return st;
  size_t at = item_at + ((wp.size() * sizeof(float) + 255) & ~(size_t)255);
  // Split into the tiled launches (32 taps, |delta| <= 0.01; 8 outputs per
  // lane while the quadratic weights hold over 256 outputs, else 4) and the
  // direct one.
  std::vector<RsItem> tiled8, tiled4, direct;
  for (auto& it : items) {
    const double dl = std::fabs((double)it.dl_hi + (double)it.dl_lo);
    if (o.taps != 32 || dl > kRsTiledMaxDelta) direct.push_back(it);
    else (resample_q(dl) == 8 && c->tune.rs_q != 4 ? tiled8 : tiled4).push_back(it);
  }
  for (int pass = 0; pass < 3; ++pass) {
    auto& v = pass == 0 ? tiled8 : pass == 1 ? tiled4 : direct;
    if (v.empty()) continue;
    int tiles = 0;
    for (auto& it : v) {
      it.tile_begin = tiles;
      tiles += (int)((it.n_out + kRsTile - 1) / kRsTile);
    }
    const RsItem* dev = nullptr;
    if ((st = upload(c, v, at, s, &dev))) return st;
    at += (v.size() * sizeof(RsItem) + 255) & ~(size_t)255;
    RsArgs a{};
    a.items = dev;
    a.n_items = (int)v.size();
    a.n_tiles = tiles;
    a.half = o.taps / 2;
    a.wpoly = dwp;
    a.err = c->err;
    long long outs = 0;
    for (auto& it : v) outs += it.n_out;
    Phase ph(c, pass < 2 ? PH_RS_TILED : PH_RS_DIRECT, s, outs);
    cudaError_t e = pass < 2 ? launch_resample_tiled32(a, pass == 0 ? 8 : 4, s)
                             : launch_resample_direct(a, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "resample launch");
  }
  return DC_OK;
}

// The bank's resampling on tensor cores (rs_tc.cu): the range rates ordered
// by delta in groups of 32, each group's integer offsets over a 128-output
// tile spanning at most rs_tc_max_span() samples.  Returns DC_EINVAL, having
// launched and uploaded nothing, when the range rates are too far apart for
// that (the caller then takes the CUDA-core kernel); other failures as usual.
dc_status run_resample_tc(dc_ctx* c, const float2* x, int n_in, int n_out, const double* v_r,
                          int n_v, const dc_opts& o, float2* Y, size_t item_at, cudaStream_t s) {
  std::vector<int> order(n_v);
  std::vector<double> dl(n_v);
  for (int i = 0; i < n_v; ++i) {
    order[i] = i;
    dl[i] = alpha_minus_one(v_r[i]);
  }
  std::sort(order.begin(), order.end(), [&](int p, int q) { return dl[p] < dl[q]; });
  for (int g = 0; g < n_v; g += 32) {
    const int last = std::min(n_v, g + 32) - 1;
    const double spread = (dl[order[last]] - dl[order[g]]) * ((double)n_out + 64.0) + 2.0;
    if (spread > (double)rs_tc_max_span()) return DC_EINVAL;
  }
  const std::vector<float> wp = window_poly_d012(o.taps, o.kaiser_beta);
  std::vector<float> dls(2 * (size_t)n_v);
  std::vector<int> vidx(n_v);
  for (int i = 0; i < n_v; ++i) {
    split(dl[order[i]], dls[2 * i], dls[2 * i + 1]);
    vidx[i] = order[i];
  }
  const float* dwp = nullptr;
  const float* ddl = nullptr;
  const int* dvi = nullptr;
  dc_status st = upload(c, wp, item_at, s, &dwp);
  if (st) return st;
  item_at += (wp.size() * sizeof(float) + 255) & ~(size_t)255;
  if ((st = upload(c, dls, item_at, s, &ddl))) return st;
  item_at += (dls.size() * sizeof(float) + 255) & ~(size_t)255;
  if ((st = upload(c, vidx, item_at, s, &dvi))) return st;
  RsTcArgs a{x, n_in, n_out, Y, ddl, dvi, n_v, dwp, c->err};
  Phase ph(c, PH_RS_TC, s, (long long)n_v * n_out);
  cudaError_t e = launch_resample_tc(a, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core resample launch");
  return DC_OK;
}

size_t items_bytes_for(size_t n) { return ((n * 128 + 255) & ~(size_t)255) + 16384; }

// Scratch layout of one correct_batch call: the resampled pulse of each item,
// then per length class 2^13..2^20 on the three-pass schedule the four-step
// intermediate of `class_chunk` transforms.  Items grouped by L.
struct BatchLayout {
  std::vector<size_t> yoff;
  std::vector<std::vector<int>> by_L;
  std::vector<size_t> class_T, class_chunk;
  size_t bytes = 0;
};
BatchLayout batch_layout(const dc_ctx* c, const dc_item* items, int n_items) {
  BatchLayout b;
  Arena ar;
  b.yoff.resize(n_items);
  b.by_L.resize(21);
  for (int i = 0; i < n_items; ++i) {
    const long long no = items[i].n_out ? items[i].n_out : items[i].n;
    b.yoff[i] = ar.take((size_t)no * sizeof(float2));
    b.by_L[log2_ceil(no)].push_back(i);
  }
  b.class_T.assign(21, 0);
  b.class_chunk.assign(21, 1);
  for (int m = 13; m <= 20; ++m)
    if (!b.by_L[m].empty() && !use_fused(c, m)) {
      b.class_chunk[m] = chunk_items(c, m, b.by_L[m].size(), 0);
      b.class_T[m] = ar.take(b.class_chunk[m] * ((size_t)1 << m) * sizeof(float2));
    }
  b.bytes = ar.off;
  return b;
}

// ------------------------------------------------------ correction pipeline
// One L class of pulses already resampled into y; writes corrected outputs.
// Four-step classes use T (L samples per item) from the scratch.
dc_status run_iono_class(dc_ctx* c, std::vector<FftItem>& it, int log2L, float2* T,
                         size_t chunk, size_t& item_at, cudaStream_t s) {
  if (it.empty()) return DC_OK;
  const FftItem* dev = nullptr;
  cudaError_t e;
  if (use_fused(c, log2L)) {
    dc_status st = upload(c, it, item_at, s, &dev);
    if (st) return st;
    item_at += (it.size() * sizeof(FftItem) + 255) & ~(size_t)255;
    FusedArgs a{dev, (int)it.size(), log2L, c->tw, c->err, c->t4};
    a.pdl = std::none_of(it.begin(), it.end(), [](const FftItem& f) { return f.ptab != nullptr; });
    long long outs = 0;
    for (auto& f : it) outs += f.n_out;
    Phase ph(c, PH_FUSED_FULL, s, outs);
    e = launch_fused(FUSED_FULL, a, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "fused launch");
    return DC_OK;
  }
  if (log2L <= 12) {
    dc_status st = upload(c, it, item_at, s, &dev);
    if (st) return st;
    item_at += (it.size() * sizeof(FftItem) + 255) & ~(size_t)255;
    RowArgs a{dev, (int)it.size(), log2L, 0, c->tw};
    long long outs = 0;
    for (auto& f : it) outs += f.n_out;
    Phase ph(c, PH_ROW_FULL, s, outs);
    e = launch_row(ROW_FULL, a, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "row launch");
    return DC_OK;
  }
  const int log2L1 = log2L - 12;
  const size_t L = (size_t)1 << log2L;
  // pass 1: y -> T ; pass 2: T in place ; pass 3: T -> out, chunk by chunk
  // (T holds `chunk` transforms)
  std::vector<FftItem> p1 = it, p2 = it, p3 = it;
  for (size_t i = 0; i < it.size(); ++i) {
    float2* Ti = T + (i % chunk) * L;
    p1[i].dst = Ti;
    p2[i].src = Ti;
    p2[i].dst = Ti;
    p3[i].src = Ti;
  }
  const FftItem *d1, *d2, *d3;
  dc_status st;
  if ((st = upload(c, p1, item_at, s, &d1))) return st;
  item_at += (it.size() * sizeof(FftItem) + 255) & ~(size_t)255;
  if ((st = upload(c, p2, item_at, s, &d2))) return st;
  item_at += (it.size() * sizeof(FftItem) + 255) & ~(size_t)255;
  if ((st = upload(c, p3, item_at, s, &d3))) return st;
  item_at += (it.size() * sizeof(FftItem) + 255) & ~(size_t)255;
  for (size_t j0 = 0; j0 < it.size(); j0 += chunk) {
    const int cnt = (int)std::min(chunk, it.size() - j0);
    long long outs = 0;
    for (size_t i = j0; i < j0 + cnt; ++i) outs += it[i].n_out;
    ColArgs a1{d1 + j0, cnt, log2L, log2L1, c->tw};
    {
      Phase ph(c, PH_COL_F1, s, outs);
      if ((e = launch_col(COL_F1, a1, s)) != cudaSuccess) return cuda_fail(c, e, "col F1 launch");
    }
    RowArgs a2{d2 + j0, cnt, log2L, log2L1, c->tw};
    {
      Phase ph(c, PH_ROW_MID, s, outs);
      e = log2L >= 17 ? launch_row_mid_4096(a2, s) : launch_row(ROW_MID, a2, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "row launch");
    }
    ColArgs a3{d3 + j0, cnt, log2L, log2L1, c->tw};
    {
      Phase ph(c, PH_COL_B, s, outs);
      if ((e = launch_col(COL_B, a3, s)) != cudaSuccess) return cuda_fail(c, e, "col B launch");
    }
  }
  return DC_OK;
}

}  // namespace

namespace dc {
__global__ void stuck_wait_kernel(int* err, int polls);   // failure-detection self-test
}

// ==================================================================== ABI
extern "C" {

void dc_opts_default(dc_opts* o) {
  if (!o) return;
  o->taps = 32;
  o->kaiser_beta = 8.0;
  o->mode = DC_WINDOWED;
  o->n_out = 0;
  o->carrier_shift = 0;
  o->freq_ref = 0.0;
}

const char* dc_status_str(int s) {
  switch (s) {
    case DC_OK: return "DC_OK";
    case DC_EINVAL: return "DC_EINVAL";
    case DC_ENOMEM: return "DC_ENOMEM";
    case DC_EBUSY: return "DC_EBUSY";
    case DC_ECUDA: return "DC_ECUDA";
    case DC_ETIMEOUT: return "DC_ETIMEOUT";
    case DC_ECANCELLED: return "DC_ECANCELLED";
    default: return "DC_UNKNOWN";
  }
}

dc_status dc_create(dc_ctx** out, int device, size_t budget) {
  if (!out) return DC_EINVAL;
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DC_ECUDA;
  }
  if (device < 0 || device >= count) return DC_EINVAL;
  if ((e = cudaSetDevice(device)) != cudaSuccess) return DC_ECUDA;
  dc_ctx* c = new (std::nothrow) dc_ctx();
  if (!c) return DC_ENOMEM;
  c->device = device;
  c->budget = budget;
  // Twiddle tables in FP64, rounded to float (layout in common.cuh).
  std::vector<float2> tw(kTwSize), t4(kT4Size);
  fill_twiddles(tw.data());
  fill_four_step(t4.data());
  if ((e = cudaMalloc(&c->tw, sizeof(float2) * kTwSize)) != cudaSuccess ||
      (e = cudaMemcpy(c->tw, tw.data(), sizeof(float2) * kTwSize, cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMalloc(&c->t4, sizeof(float2) * kT4Size)) != cudaSuccess ||
      (e = cudaMemcpy(c->t4, t4.data(), sizeof(float2) * kT4Size, cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMalloc(&c->err, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(c->err, 0, sizeof(int))) != cudaSuccess) {
    cudaGetLastError();
    if (c->tw) cudaFree(c->tw);
    if (c->t4) cudaFree(c->t4);
    if (c->err) cudaFree(c->err);
    delete c;
    return DC_ENOMEM;
  }
  // a schedule cache named by DC_TUNING_CACHE is loaded when it exists (a
  // missing or unreadable file leaves the built-in rules)
  if (const char* path = getenv("DC_TUNING_CACHE")) {
    if (FILE* f = fopen(path, "r")) {
      fclose(f);
      if (dc_tuning_load(c, path) != DC_OK) c->tune = dc_ctx::Tune{};
    }
  }
  *out = c;
  return DC_OK;
}

dc_status dc_destroy(dc_ctx* c) {
  if (!c) return DC_EINVAL;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (auto& r : c->pending) c->pool.push_back(r.a), c->pool.push_back(r.b);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  for (void* p : c->retired) cudaFree(p);
  if (c->ws) cudaFree(c->ws);
  if (c->items) cudaFree(c->items);
  if (c->tw) cudaFree(c->tw);
  if (c->t4) cudaFree(c->t4);
  if (c->err) cudaFree(c->err);
  delete c;
  return DC_OK;
}

const char* dc_last_error(const dc_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

long long dc_launch_count(const dc_ctx* c) { return c ? c->launches : -1; }

dc_status dc_profile_enable(dc_ctx* c, int on) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  for (auto& r : c->pending) {
    cudaEventSynchronize(r.b);
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->pending.clear();
  for (int i = 0; i < dc_ctx::kMaxPhases; ++i)
    c->acc_ms[i] = 0, c->acc_launches[i] = 0, c->acc_samples[i] = 0;
  c->profiling = on != 0;
  return DC_OK;
}

int dc_profile_read(dc_ctx* c, dc_phase_time* out, int max) {
  if (!c) return -1;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  for (auto& r : c->pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    c->acc_ms[r.phase] += ms;
    c->acc_launches[r.phase] += 1;
    c->acc_samples[r.phase] += r.samples;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->pending.clear();
  int n = 0;
  for (int i = 0; i < PH_COUNT; ++i) {
    if (!c->acc_launches[i]) continue;
    if (out && n < max) {
      memset(out[n].name, 0, sizeof out[n].name);
      strncpy(out[n].name, kPhaseName[i], sizeof out[n].name - 1);
      out[n].launches = c->acc_launches[i];
      out[n].samples = c->acc_samples[i];
      out[n].ms = c->acc_ms[i];
    }
    ++n;
  }
  return n;
}

dc_status dc_selftest_wait_timeout(dc_ctx* c, void* stream) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  cudaSetDevice(c->device);
  stuck_wait_kernel<<<1, 32, 0, S(stream)>>>(c->err, 1 << 16);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "self-test launch");
  ++c->launches;
  return DC_OK;
}

dc_status dc_check(dc_ctx* c, void* stream) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  cudaError_t e = cudaStreamSynchronize(S(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  int flag = 0;
  if ((e = cudaMemcpy(&flag, c->err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(c, e, "error flag read");
  if (flag) {
    cudaMemset(c->err, 0, sizeof(int));
    if (flag == 1) return fail(c, DC_ETIMEOUT, "a kernel's bounded wait ran out");
    if (flag == 3) return fail(c, DC_ECUDA, "a bounds check of the checked build failed");
    return fail(c, DC_EINVAL, "a kernel met parameters outside its range (code %d)", flag);
  }
  return DC_OK;
}

dc_status doppler_resample(dc_ctx* c, const dc_c64* x, long long n, dc_c64* y, double fs,
                           double fc, double v_r, const dc_opts* opts, void* stream) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dc_opts o;
  dc_opts_default(&o);
  if (opts) o = *opts;
  dc_status st = check_opts(c, &o);
  if (st) return st;
  const long long n_out = o.n_out ? o.n_out : n;
  if ((st = check_pulse(c, n, n_out, fs, fc, v_r, 0.0))) return st;
  if (!x || !y) return fail(c, DC_EINVAL, "null buffer");
  cudaSetDevice(c->device);
  const double dl = alpha_minus_one(v_r);
  cudaStream_t s = S(stream);
  if ((st = ensure_items(c, items_bytes_for(4)))) return st;
  if (o.mode == DC_WINDOWED || o.mode == DC_FREQCONV) {
    std::vector<RsItem> items(1);
    items[0] = RsItem{};
    items[0].x = reinterpret_cast<const float2*>(x);
    items[0].y = reinterpret_cast<float2*>(y);
    items[0].n_in = (int)n;
    items[0].n_out = (int)n_out;
    split(dl, items[0].dl_hi, items[0].dl_lo);
    split(rotation_rate(o, dl, fs, fc), items[0].rot_hi, items[0].rot_lo);
    return run_windowed(c, items, o, 0, s);
  }
  if (o.mode != DC_EXACT_FP32) return fail(c, DC_EINVAL, "single-pulse exact resampling uses FP32");
  std::vector<ExItem> ex(1);
  ex[0] = ExItem{};
  ex[0].x = reinterpret_cast<const float2*>(x);
  ex[0].y = reinterpret_cast<float2*>(y);
  split(dl, ex[0].dl_hi, ex[0].dl_lo);
  split(rotation_rate(o, dl, fs, fc), ex[0].rot_hi, ex[0].rot_lo);
  const ExItem* dev = nullptr;
  if ((st = upload(c, ex, 0, s, &dev))) return st;
  ExArgs a{dev, (int)n, (int)n_out, 1};
  Phase ph(c, PH_EXACT, s, n_out);
  cudaError_t e = launch_exact_fp32(a, 1, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "exact launch");
  return DC_OK;
}

dc_status iono_correct(dc_ctx* c, const dc_c64* x, long long n, dc_c64* y, double fs, double fc,
                       double tec, void* stream) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dc_status st = check_pulse(c, n, n, fs, fc, 0.0, tec);
  if (st) return st;
  if (!x || !y) return fail(c, DC_EINVAL, "null buffer");
  cudaSetDevice(c->device);
  const int log2L = log2_ceil(n);
  const size_t L = (size_t)1 << log2L;
  if ((st = ensure_ws(c, log2L > 12 ? L * sizeof(float2) : 256))) return st;
  if ((st = ensure_items(c, items_bytes_for(8)))) return st;
  std::vector<FftItem> it(1);
  it[0].src = reinterpret_cast<const float2*>(x);
  it[0].dst = reinterpret_cast<float2*>(y);
  it[0].ptab = nullptr;
  it[0].ph = phase_params(fs, fc, tec, log2L);
  it[0].n_valid = (int)n;
  it[0].n_out = (int)n;
  size_t at = 0;
  return run_iono_class(c, it, log2L, reinterpret_cast<float2*>(c->ws), 1, at, S(stream));
}

dc_status correct_batch(dc_ctx* c, const dc_c64* in, dc_c64* out, const dc_item* items,
                        int n_items, const dc_opts* opts, void* stream) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dc_opts o;
  dc_opts_default(&o);
  if (opts) o = *opts;
  dc_status st = check_opts(c, &o);
  if (st) return st;
  if (n_items < 0 || (n_items > 0 && (!items || !in || !out)))
    return fail(c, DC_EINVAL, "bad item list");
  if (n_items == 0) return DC_OK;
  if (o.mode != DC_WINDOWED && o.mode != DC_EXACT_FP32 && o.mode != DC_FREQCONV)
    return fail(c, DC_EINVAL, "correct_batch supports DC_WINDOWED, DC_EXACT_FP32 and DC_FREQCONV");
  for (int i = 0; i < n_items; ++i) {
    const dc_item& it = items[i];
    const long long no = it.n_out ? it.n_out : it.n;
    if ((st = check_pulse(c, it.n, no, it.fs, it.fc, it.v_r, it.tec_tecu)))
      return fail(c, st, "item %d: %s", i, c->last_error.c_str());
    if (it.in_off < 0 || it.out_off < 0) return fail(c, DC_EINVAL, "item %d: negative offset", i);
  }
  cudaSetDevice(c->device);
  cudaStream_t s = S(stream);
  const float2* X = reinterpret_cast<const float2*>(in);
  float2* Y = reinterpret_cast<float2*>(out);

  const BatchLayout lay = batch_layout(c, items, n_items);
  const std::vector<size_t>& yoff = lay.yoff;
  const std::vector<std::vector<int>>& by_L = lay.by_L;
  const std::vector<size_t>& class_T = lay.class_T;
  const std::vector<size_t>& class_chunk = lay.class_chunk;
  if ((st = ensure_ws(c, lay.bytes))) return st;
  if ((st = ensure_items(c, items_bytes_for((size_t)n_items * 4)))) return st;
  char* ws = c->ws;
  size_t item_at = 0;

  // 1. resampling
  if (o.mode == DC_WINDOWED || o.mode == DC_FREQCONV) {
    std::vector<RsItem> rs(n_items);
    for (int i = 0; i < n_items; ++i) {
      const dc_item& it = items[i];
      const double dl = alpha_minus_one(it.v_r);
      rs[i] = RsItem{};
      rs[i].x = X + it.in_off;
      rs[i].y = reinterpret_cast<float2*>(ws + yoff[i]);
      rs[i].n_in = (int)it.n;
      rs[i].n_out = (int)(it.n_out ? it.n_out : it.n);
      split(dl, rs[i].dl_hi, rs[i].dl_lo);
      split(rotation_rate(o, dl, it.fs, it.fc), rs[i].rot_hi, rs[i].rot_lo);
    }
    if ((st = run_windowed(c, rs, o, item_at, s))) return st;
    item_at += 2 * ((n_items * sizeof(RsItem) + 255) & ~(size_t)255) + 4096;
  } else {
    for (int i = 0; i < n_items; ++i) {
      const dc_item& it = items[i];
      std::vector<ExItem> ex(1);
      const double dl = alpha_minus_one(it.v_r);
      ex[0] = ExItem{};
      ex[0].x = X + it.in_off;
      ex[0].y = reinterpret_cast<float2*>(ws + yoff[i]);
      split(dl, ex[0].dl_hi, ex[0].dl_lo);
      split(rotation_rate(o, dl, it.fs, it.fc), ex[0].rot_hi, ex[0].rot_lo);
      const ExItem* dev = nullptr;
      if ((st = upload(c, ex, item_at, s, &dev))) return st;
      item_at += 256;
      ExArgs a{dev, (int)it.n, (int)(it.n_out ? it.n_out : it.n), 1};
      Phase ph(c, PH_EXACT, s, a.n_out);
      cudaError_t e = launch_exact_fp32(a, 1, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "exact launch");
    }
  }
  // 2. ionospheric correction per L class
  for (int m = 0; m <= 20; ++m) {
    if (by_L[m].empty()) continue;
    std::vector<FftItem> fi(by_L[m].size());
    for (size_t j = 0; j < by_L[m].size(); ++j) {
      const int i = by_L[m][j];
      const dc_item& it = items[i];
      const int no = (int)(it.n_out ? it.n_out : it.n);
      fi[j].src = reinterpret_cast<const float2*>(ws + yoff[i]);
      fi[j].dst = Y + it.out_off;
      fi[j].ptab = nullptr;
      fi[j].ph = phase_params(it.fs, it.fc, it.tec_tecu, m);
      fi[j].n_valid = no;
      fi[j].n_out = no;
    }
    float2* T = reinterpret_cast<float2*>(ws + class_T[m]);
    if ((st = run_iono_class(c, fi, m, T, class_chunk[m], item_at, s))) return st;
  }
  return DC_OK;
}

}  // extern "C"

// Phase table for the bank: P[t][k] = exp(-i phi_k(TEC_t)).
namespace dc {
// Failure-detection self-test: one thread polls, with the same try-wait and
// flag the library's bounded waits use, an mbarrier that nothing arrives
// on; the poll runs out, the flag is raised and the kernel returns.
__global__ void stuck_wait_kernel(int* err, int polls) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  for (int i = 0; i < polls; ++i)
    if (mbar_try_wait(&bar, 0)) return;
  atomicMax(err, 1);
}

// Factor tables P[t][.] in the spectrum layout (element k1*4096 + k2 holds
// bin k1 + L1 k2, L1 = L/4096, for L > 4096; natural order for L <= 4096 --
// the same formula with L1 = 1): exp(-i phi_k(TEC_t)) times `scale` (1/L
// for the spectrum-apply kernel, which folds in the inverse transform's
// factor; else 1).  H (optional): a replica's spectrum in the same layout;
// each factor is then multiplied by conj(H_k), the matched filter of pulse
// compression (Sec. II-B).
__global__ void phase_table_kernel(const PhaseParams* ph, int n_tec, int log2L, float scale,
                                   const float2* H, float2* P) {
  const size_t L = (size_t)1 << log2L;
  const size_t total = L * (size_t)n_tec;
  const int log2L1 = log2L > 12 ? log2L - 12 : 0;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(g >> log2L), idx = (int)(g & (L - 1));
    const int k = (idx >> 12) + ((idx & 4095) << log2L1);
    float2 w = ph[t].enabled ? iono_factor(ph[t], k) : make_float2(1.f, 0.f);
    if (H) {
      const float2 h = __ldg(H + idx);
      w = cmul(w, make_float2(h.x, -h.y));
    }
    P[g] = cscale(w, scale);
  }
}
}  // namespace dc

namespace {

// Forward spectra of the items' sources (zero-padded past n_valid) into their
// dst, length L = 2^log2L, in the spectrum layout (bin k1 + L1 k2 at
// k1*4096 + k2 for L > 4096, natural order below): cluster-fused, one row
// pass, or the first two passes of the four-step split (T: L samples per
// item of scratch).
dc_status run_spectra(dc_ctx* c, std::vector<FftItem>& sp, int log2L, float2* T, size_t& item_at,
                      cudaStream_t s) {
  const int n_sp = (int)sp.size();
  const bool four = log2L > 12;
  const size_t L = (size_t)1 << log2L;
  long long samples = 0;
  for (auto& f : sp) samples += f.n_valid;
  const FftItem* dev = nullptr;
  dc_status st;
  cudaError_t e;
  if (use_fused(c, log2L)) {
    if ((st = upload(c, sp, item_at, s, &dev))) return st;
    item_at += (n_sp * sizeof(FftItem) + 255) & ~(size_t)255;
    FusedArgs a{dev, n_sp, log2L, c->tw, c->err, c->t4};
    Phase ph(c, PH_FUSED_SPEC, s, samples);
    if ((e = launch_fused(FUSED_SPEC, a, s)) != cudaSuccess) return cuda_fail(c, e, "spec launch");
  } else if (!four) {
    if ((st = upload(c, sp, item_at, s, &dev))) return st;
    item_at += (n_sp * sizeof(FftItem) + 255) & ~(size_t)255;
    RowArgs a{dev, n_sp, log2L, 0, c->tw};
    Phase ph(c, PH_ROW_SPEC, s, samples);
    if ((e = launch_row(ROW_SPEC, a, s)) != cudaSuccess) return cuda_fail(c, e, "spec launch");
  } else {
    std::vector<FftItem> f1 = sp, f2 = sp;
    for (int i = 0; i < n_sp; ++i) {
      f1[i].dst = T + (size_t)i * L;
      f2[i].src = T + (size_t)i * L;
    }
    if ((st = upload(c, f1, item_at, s, &dev))) return st;
    item_at += (n_sp * sizeof(FftItem) + 255) & ~(size_t)255;
    ColArgs a1{dev, n_sp, log2L, log2L - 12, c->tw};
    {
      Phase ph(c, PH_COL_F1, s, samples);
      if ((e = launch_col(COL_F1, a1, s)) != cudaSuccess) return cuda_fail(c, e, "F1 launch");
    }
    if ((st = upload(c, f2, item_at, s, &dev))) return st;
    item_at += (n_sp * sizeof(FftItem) + 255) & ~(size_t)255;
    RowArgs a2{dev, n_sp, log2L, log2L - 12, c->tw};
    Phase ph(c, PH_ROW_SPEC, s, samples);
    if ((e = launch_row(ROW_SPEC, a2, s)) != cudaSuccess) return cuda_fail(c, e, "F2 launch");
  }
  return DC_OK;
}

// The Doppler bank (correct_bank), and with a replica (rep, n_rep samples)
// the bank compressed against it (correct_compress_bank): the replica's
// spectrum is computed with the range rates' spectra and its conjugate
// folded into every TEC's factor table, so the phase-and-inverse pass is
// unchanged (Sec. II-B's bundling of the correction with pulse compression).
dc_status bank_impl(dc_ctx* c, const dc_c64* x, long long n, const dc_c64* rep, long long n_rep,
                    const double* v_r, int n_v, const double* tec, int n_tec, dc_c64* out,
                    double fs, double fc, const dc_opts* opts, void* stream) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dc_opts o;
  dc_opts_default(&o);
  if (opts) o = *opts;
  dc_status st = check_opts(c, &o);
  if (st) return st;
  if (o.mode != DC_WINDOWED && o.mode != DC_FREQCONV)
    return fail(c, DC_EINVAL, "the bank supports DC_WINDOWED and DC_FREQCONV");
  if (n_v < 1 || n_tec < 1 || !v_r || !tec || !x || !out)
    return fail(c, DC_EINVAL, "bad bank lists");
  const long long n_out = o.n_out ? o.n_out : n;
  for (int i = 0; i < n_v; ++i)
    if ((st = check_pulse(c, n, n_out, fs, fc, v_r[i], 0.0))) return st;
  for (int t = 0; t < n_tec; ++t)
    if (!std::isfinite(tec[t])) return fail(c, DC_EINVAL, "tec[%d] not finite", t);
  const int log2L = log2_ceil(n_out);
  const size_t L = (size_t)1 << log2L;
  const bool compress = rep != nullptr;
  if (compress && (n_rep < 1 || (size_t)n_rep > L))
    return fail(c, DC_EINVAL, "replica length %lld outside [1, L = %zu]", n_rep, L);
  cudaSetDevice(c->device);
  cudaStream_t s = S(stream);
  const bool four = log2L > 12;
  const bool fused = use_fused(c, log2L);
  // Transforms per chunk of the inverse (four-step T kept small enough to
  // stay in L2 between its two passes).
  const int chunk =
      four ? (int)chunk_items(c, log2L, (size_t)n_v * n_tec, (size_t)64 << 20) : n_v * n_tec;
  const int n_sp = n_v + (compress ? 1 : 0);     // spectra: one per v_r, then the replica's
  Arena ar;
  const size_t y_at = ar.take((size_t)n_v * n_out * sizeof(float2));
  const size_t p_at = ar.take((size_t)n_tec * L * sizeof(float2));
  const size_t s_at = ar.take((size_t)n_sp * L * sizeof(float2));
  const size_t t_at =
      ar.take(fused ? 0 : (size_t)std::max(chunk, four ? n_sp : 0) * L * sizeof(float2));
  const size_t n_pairs = (size_t)n_v * n_tec;
  const bool l2 = fused && apply_l2(c, log2L);
  const int l2_chunk = l2 ? apply_l2_chunk(log2L, n_pairs) : 0;
  const size_t q_at = ar.take(l2 ? (size_t)kApplyL2Slots * l2_chunk * L * sizeof(float2) : 0);
  const size_t k_at = ar.take(l2 ? (1 + 2 * n_pairs) * sizeof(int) : 0);
  if ((st = ensure_ws(c, ar.off))) return st;
  if ((st = ensure_items(c, items_bytes_for(n_pairs * 2 + n_sp * 6 + n_tec)))) return st;
  char* ws = c->ws;
  float2* Yr = reinterpret_cast<float2*>(ws + y_at);
  float2* P = reinterpret_cast<float2*>(ws + p_at);
  float2* Sp = reinterpret_cast<float2*>(ws + s_at);
  float2* T = reinterpret_cast<float2*>(ws + t_at);
  size_t item_at = 0;
  cudaError_t e;

  // 1. resample per v_r
  std::vector<RsItem> rs(n_v);
  for (int i = 0; i < n_v; ++i) {
    const double dl = alpha_minus_one(v_r[i]);
    rs[i] = RsItem{};
    rs[i].x = reinterpret_cast<const float2*>(x);
    rs[i].y = Yr + (size_t)i * n_out;
    rs[i].n_in = (int)n;
    rs[i].n_out = (int)n_out;
    split(dl, rs[i].dl_hi, rs[i].dl_lo);
    split(rotation_rate(o, dl, fs, fc), rs[i].rot_hi, rs[i].rot_lo);
  }
  const bool tc_ok = o.mode == DC_WINDOWED && o.taps == 32 && !o.carrier_shift && c->tune.rs_tc != 2;
  st = tc_ok ? run_resample_tc(c, reinterpret_cast<const float2*>(x), (int)n, (int)n_out, v_r, n_v, o,
                               Yr, item_at, s)
             : DC_EINVAL;
  if (st == DC_EINVAL) st = run_windowed(c, rs, o, item_at, s);   // not eligible: CUDA cores
  if (st) return st;
  item_at += 2 * ((n_v * sizeof(RsItem) + 255) & ~(size_t)255) + 4096 +
             ((n_v * 3 * sizeof(float) + 32 * 8 * sizeof(float) + 3 * 255) & ~(size_t)255);
  // 2. spectra per v_r (and of the zero-padded replica): four-step layout
  // for L > 4096, natural order below
  std::vector<FftItem> sp(n_sp);
  for (int i = 0; i < n_sp; ++i) {
    const bool is_rep = i == n_v;
    sp[i] = FftItem{};
    sp[i].src = is_rep ? reinterpret_cast<const float2*>(rep) : Yr + (size_t)i * n_out;
    sp[i].dst = Sp + (size_t)i * L;
    sp[i].n_valid = (int)(is_rep ? n_rep : n_out);
    sp[i].n_out = sp[i].n_valid;
  }
  if ((st = run_spectra(c, sp, log2L, T, item_at, s))) return st;
  // 3. factor table per TEC: exp(-i phi_k) (times conj of the replica's
  // spectrum when compressing), in the layout the inverse pass reads
  std::vector<PhaseParams> ph(n_tec);
  for (int t = 0; t < n_tec; ++t) ph[t] = phase_params(fs, fc, tec[t], log2L);
  const PhaseParams* dph = nullptr;
  if ((st = upload(c, ph, item_at, s, &dph))) return st;
  item_at += (n_tec * sizeof(PhaseParams) + 255) & ~(size_t)255;
  {
    const size_t total = L * n_tec;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    Phase phs(c, PH_PHASE_TABLE, s, (long long)total);
    phase_table_kernel<<<grid, 256, 0, s>>>(dph, n_tec, log2L, fused ? 1.0f / (float)L : 1.0f,
                                            compress ? Sp + (size_t)n_v * L : nullptr, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "phase table launch");
  }
  // 4. factors + inverse per (v_r, TEC), in chunks
  if (fused) {
    // the transforms form a grid (spectrum i x factor table t): the kernels
    // form each one from its index, no item list is uploaded
    FusedArgs a{nullptr, (int)n_pairs, log2L, c->tw, c->err, c->t4};
    a.grid_src = Sp;
    a.grid_ptab = P;
    a.grid_dst = reinterpret_cast<float2*>(out);
    a.grid_n_tec = n_tec;
    a.grid_n_out = (int)n_out;
    a.apply_rows2 = apply_rows2(c, log2L);
    if (l2) {
      a.scratch = reinterpret_cast<float2*>(ws + q_at);
      a.ctr = reinterpret_cast<int*>(ws + k_at);
      a.chunk = l2_chunk;
      if ((e = cudaMemsetAsync(a.ctr, 0, (1 + 2 * n_pairs) * sizeof(int), s)) != cudaSuccess)
        return cuda_fail(c, e, "apply counters");
    }
    Phase ph(c, PH_FUSED_APPLY, s, (long long)n_pairs * n_out);
    if ((e = launch_fused(FUSED_APPLY, a, s)) != cudaSuccess) return cuda_fail(c, e, "apply launch");
    return DC_OK;
  }
  const FftItem* dev = nullptr;
  std::vector<FftItem> ap(n_pairs);
  for (int i = 0; i < n_v; ++i)
    for (int t = 0; t < n_tec; ++t) {
      FftItem& f = ap[(size_t)i * n_tec + t];
      f = FftItem{};
      f.src = Sp + (size_t)i * L;
      f.ptab = P + (size_t)t * L;
      f.dst = reinterpret_cast<float2*>(out) + ((size_t)i * n_tec + t) * n_out;
      f.n_valid = (int)n_out;
      f.n_out = (int)n_out;
    }
  if (!four) {
    if ((st = upload(c, ap, item_at, s, &dev))) return st;
    RowArgs a{dev, (int)n_pairs, log2L, 0, c->tw};
    Phase ph(c, PH_ROW_APPLY, s, (long long)n_pairs * n_out);
    if ((e = launch_row(ROW_APPLY, a, s)) != cudaSuccess) return cuda_fail(c, e, "apply launch");
    return DC_OK;
  }
  std::vector<FftItem> ra = ap, cb = ap;
  for (size_t j = 0; j < n_pairs; ++j) {
    float2* Tj = T + (j % (size_t)chunk) * L;
    ra[j].dst = Tj;
    cb[j].src = Tj;
  }
  const FftItem *dra = nullptr, *dcb = nullptr;
  if ((st = upload(c, ra, item_at, s, &dra))) return st;
  item_at += (n_pairs * sizeof(FftItem) + 255) & ~(size_t)255;
  if ((st = upload(c, cb, item_at, s, &dcb))) return st;
  for (size_t j0 = 0; j0 < n_pairs; j0 += chunk) {
    const int cnt = (int)std::min<size_t>(chunk, n_pairs - j0);
    RowArgs a{dra + j0, cnt, log2L, log2L - 12, c->tw};
    {
      Phase ph(c, PH_ROW_APPLY, s, (long long)cnt * n_out);
      if ((e = launch_row(ROW_APPLY, a, s)) != cudaSuccess) return cuda_fail(c, e, "apply launch");
    }
    ColArgs b{dcb + j0, cnt, log2L, log2L - 12, c->tw};
    {
      Phase ph(c, PH_COL_B, s, (long long)cnt * n_out);
      if ((e = launch_col(COL_B, b, s)) != cudaSuccess) return cuda_fail(c, e, "B launch");
    }
  }
  return DC_OK;
}

}  // namespace

extern "C" dc_status correct_bank(dc_ctx* c, const dc_c64* x, long long n, const double* v_r,
                                  int n_v, const double* tec, int n_tec, dc_c64* out, double fs,
                                  double fc, const dc_opts* opts, void* stream) {
  return bank_impl(c, x, n, nullptr, 0, v_r, n_v, tec, n_tec, out, fs, fc, opts, stream);
}

extern "C" dc_status correct_compress_bank(dc_ctx* c, const dc_c64* x, long long n,
                                           const dc_c64* replica, long long n_rep,
                                           const double* v_r, int n_v, const double* tec,
                                           int n_tec, dc_c64* out, double fs, double fc,
                                           const dc_opts* opts, void* stream) {
  if (!replica) return fail(c, DC_EINVAL, "null replica");
  return bank_impl(c, x, n, replica, n_rep, v_r, n_v, tec, n_tec, out, fs, fc, opts, stream);
}

extern "C" dc_status correct_compress(dc_ctx* c, const dc_c64* x, long long n,
                                      const dc_c64* replica, long long n_rep, dc_c64* y, double fs,
                                      double fc, double v_r, double tec, const dc_opts* opts,
                                      void* stream) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  dc_opts o;
  dc_opts_default(&o);
  if (opts) o = *opts;
  dc_status st = check_opts(c, &o);
  if (st) return st;
  if (o.mode != DC_WINDOWED && o.mode != DC_EXACT_FP32 && o.mode != DC_FREQCONV)
    return fail(c, DC_EINVAL, "correct_compress supports DC_WINDOWED, DC_EXACT_FP32 and DC_FREQCONV");
  const long long n_out = o.n_out ? o.n_out : n;
  if ((st = check_pulse(c, n, n_out, fs, fc, v_r, tec))) return st;
  if (!x || !y || !replica) return fail(c, DC_EINVAL, "null buffer");
  const int log2L = log2_ceil(n_out);
  const size_t L = (size_t)1 << log2L;
  if (n_rep < 1 || (size_t)n_rep > L)
    return fail(c, DC_EINVAL, "replica length %lld outside [1, L = %zu]", n_rep, L);
  cudaSetDevice(c->device);
  cudaStream_t s = S(stream);
  // scratch: resampled pulse, replica spectrum, factor table, four-step T
  Arena ar;
  const size_t y_at = ar.take((size_t)n_out * sizeof(float2));
  const size_t h_at = ar.take(L * sizeof(float2));
  const size_t p_at = ar.take(L * sizeof(float2));
  const size_t t_at = ar.take(log2L > 12 ? L * sizeof(float2) : 0);
  if ((st = ensure_ws(c, ar.off))) return st;
  if ((st = ensure_items(c, items_bytes_for(16)))) return st;
  char* ws = c->ws;
  float2* Yr = reinterpret_cast<float2*>(ws + y_at);
  float2* H = reinterpret_cast<float2*>(ws + h_at);
  float2* P = reinterpret_cast<float2*>(ws + p_at);
  float2* T = reinterpret_cast<float2*>(ws + t_at);
  size_t item_at = 0;
  cudaError_t e;
  const double dl = alpha_minus_one(v_r);
  // 1. resampling
  if (o.mode == DC_EXACT_FP32) {
    std::vector<ExItem> ex(1);
    ex[0] = ExItem{};
    ex[0].x = reinterpret_cast<const float2*>(x);
    ex[0].y = Yr;
    split(dl, ex[0].dl_hi, ex[0].dl_lo);
    split(rotation_rate(o, dl, fs, fc), ex[0].rot_hi, ex[0].rot_lo);
    const ExItem* dev = nullptr;
    if ((st = upload(c, ex, item_at, s, &dev))) return st;
    item_at += 256;
    ExArgs a{dev, (int)n, (int)n_out, 1};
    Phase ph(c, PH_EXACT, s, n_out);
    if ((e = launch_exact_fp32(a, 1, s)) != cudaSuccess) return cuda_fail(c, e, "exact launch");
  } else {
    std::vector<RsItem> rs(1);
    rs[0] = RsItem{};
    rs[0].x = reinterpret_cast<const float2*>(x);
    rs[0].y = Yr;
    rs[0].n_in = (int)n;
    rs[0].n_out = (int)n_out;
    split(dl, rs[0].dl_hi, rs[0].dl_lo);
    split(rotation_rate(o, dl, fs, fc), rs[0].rot_hi, rs[0].rot_lo);
    if ((st = run_windowed(c, rs, o, item_at, s))) return st;
    item_at += 2 * 256 + 4096;
  }
  // 2. the replica's spectrum (zero-padded to L)
  std::vector<FftItem> sp(1);
  sp[0] = FftItem{};
  sp[0].src = reinterpret_cast<const float2*>(replica);
  sp[0].dst = H;
  sp[0].n_valid = (int)n_rep;
  sp[0].n_out = (int)n_rep;
  if ((st = run_spectra(c, sp, log2L, T, item_at, s))) return st;
  // 3. factors exp(-i phi_k) conj(H_k) in the spectrum layout
  std::vector<PhaseParams> ph(1, phase_params(fs, fc, tec, log2L));
  const PhaseParams* dph = nullptr;
  if ((st = upload(c, ph, item_at, s, &dph))) return st;
  item_at += 256;
  {
    const int grid = (int)std::min<size_t>((L + 255) / 256, 152 * 16);
    Phase phs(c, PH_PHASE_TABLE, s, (long long)L);
    phase_table_kernel<<<grid, 256, 0, s>>>(dph, 1, log2L, 1.0f, H, P);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "factor table launch");
  }
  // 4. forward transform, factors, inverse transform, first n_out lags
  std::vector<FftItem> it(1);
  it[0] = FftItem{};
  it[0].src = Yr;
  it[0].dst = reinterpret_cast<float2*>(y);
  it[0].ptab = P;
  it[0].ph = ph[0];
  it[0].n_valid = (int)n_out;
  it[0].n_out = (int)n_out;
  return run_iono_class(c, it, log2L, T, 1, item_at, s);
}

extern "C" dc_status predistort_lfm(dc_ctx* c, dc_c64* y, long long n, double fs, double f0,
                                    double bandwidth, double T, double tec, double f_mix, int kind,
                                    void* stream) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  if (!y) return fail(c, DC_EINVAL, "null buffer");
  if (n < 1 || n > (1LL << 22)) return fail(c, DC_EINVAL, "n must be in [1, 2^22], got %lld", n);
  if (kind < DC_LFM_PLAIN || kind > DC_LFM_POLY_ORIGINAL)
    return fail(c, DC_EINVAL, "unknown waveform kind %d", kind);
  if (!(fs > 0.0) || !(f0 > 0.0) || !(bandwidth > 0.0) || !(T > 0.0) || !std::isfinite(fs) ||
      !std::isfinite(f0) || !std::isfinite(bandwidth) || !std::isfinite(T) || !std::isfinite(f_mix))
    return fail(c, DC_EINVAL, "fs, f0, bandwidth and T must be finite and > 0");
  if (!(tec >= 0.0) || !std::isfinite(tec)) return fail(c, DC_EINVAL, "tec must be finite and >= 0");
  cudaSetDevice(c->device);
  cudaStream_t s = S(stream);
  dc_status st;
  if (kind == DC_LFM_CUBIC && (st = ensure_ws(c, predist_scratch_bytes(n)))) return st;
  const PredistParams p =
      predist_params(kind, fs, f0, bandwidth, T, kKappa * tec * 1e16, kC, f_mix);
  Phase ph(c, PH_PREDIST, s, n);
  cudaError_t e = launch_predist(p, reinterpret_cast<float2*>(y), n, c->ws, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "predistortion launch");
  return DC_OK;
}

extern "C" dc_status resample_exact_batch(dc_ctx* c, const dc_c64* x, long long n, int n_pulses,
                                          long long stride, const double* v_r, int n_alpha,
                                          dc_c64* y, long long n_out, int mode, void* stream) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  if (!x || !y || !v_r || n_alpha < 1 || n_pulses < 1)
    return fail(c, DC_EINVAL, "bad exact-batch arguments");
  if (n_alpha > 65535) return fail(c, DC_EINVAL, "n_alpha %d above 65535", n_alpha);
  if (n_out == 0) n_out = n;
  dc_status st;
  for (int i = 0; i < n_alpha; ++i)
    if ((st = check_pulse(c, n, n_out, 1.0, 0.0, v_r[i], 0.0))) return st;
  if (stride < 0) return fail(c, DC_EINVAL, "negative alpha stride");
  if (mode != DC_EXACT_FP32 && mode != DC_EXACT_BF16X3 && mode != DC_EXACT_FP16X3)
    return fail(c, DC_EINVAL, "unknown exact mode %d", mode);
  cudaSetDevice(c->device);
  cudaStream_t s = S(stream);
  if (mode != DC_EXACT_FP32) {
    // Tensor-core path: pulses of all alphas contiguous, or shared (stride 0).
    if (stride != 0 && stride != (long long)n_pulses * n)
      return fail(c, DC_EINVAL, "tensor-core exact mode needs x_alpha_stride 0 or n_pulses*n");
    const long long rows_c = stride ? (long long)n_pulses * n_alpha : n_pulses;
    Arena ar;
    const size_t plane = exact_tc_plane_bytes(2 * rows_c, (int)n);
    const size_t hi_at = ar.take(plane), lo_at = ar.take(plane);
    if ((st = ensure_ws(c, ar.off))) return st;
    if ((st = ensure_items(c, items_bytes_for(n_alpha)))) return st;
    std::vector<float> dl(2 * (size_t)n_alpha);
    for (int i = 0; i < n_alpha; ++i) split(alpha_minus_one(v_r[i]), dl[2 * i], dl[2 * i + 1]);
    const float* ddl = nullptr;
    if ((st = upload(c, dl, 0, s, &ddl))) return st;
    ExTcArgs a{(int)n, (int)n_out, n_pulses, stride ? 2 * n_pulses : 0,
               reinterpret_cast<float2*>(y), ddl, c->err};
    Phase ph(c, PH_EXACT_TC, s, (long long)n_alpha * n_pulses * n_out);
    cudaError_t e = launch_exact_tc(mode == DC_EXACT_FP16X3, reinterpret_cast<const float2*>(x), rows_c,
                                    (int)n, c->ws + hi_at, c->ws + lo_at, a, n_alpha, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core exact launch");
    return DC_OK;
  }
  if ((st = ensure_items(c, items_bytes_for(n_alpha)))) return st;
  std::vector<ExItem> ex(n_alpha);
  for (int i = 0; i < n_alpha; ++i) {
    ex[i] = ExItem{};
    ex[i].x = reinterpret_cast<const float2*>(x) + (size_t)i * stride;
    ex[i].y = reinterpret_cast<float2*>(y) + (size_t)i * n_pulses * n_out;
    split(alpha_minus_one(v_r[i]), ex[i].dl_hi, ex[i].dl_lo);
  }
  const ExItem* dev = nullptr;
  if ((st = upload(c, ex, 0, s, &dev))) return st;
  ExArgs a{dev, (int)n, (int)n_out, n_pulses};
  Phase ph(c, PH_EXACT, s, (long long)n_alpha * n_pulses * n_out);
  cudaError_t e = launch_exact_fp32(a, n_alpha, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "exact launch");
  return DC_OK;
}

// ================================================================ plans
// A plan is one of the calls above recorded once into a CUDA graph: the call
// runs once on a private stream (sizing the context's scratch and warming
// up), then again with the plan's own scratch and item buffers swapped in,
// item uploads staged on the host and every kernel launch captured.  The
// staged items are copied to the plan's device buffer and the graph is
// instantiated; dc_plan_execute replays it with one cudaGraphLaunch.
struct dc_plan {
  dc_ctx* c = nullptr;
  char* ws = nullptr;
  char* items = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
};

namespace {

template <class F>
dc_status make_plan(dc_ctx* c, F&& call, dc_plan** out) {
  std::lock_guard<std::recursive_mutex> g(c->mu);
  *out = nullptr;
  cudaSetDevice(c->device);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(c, e, "plan stream");
  dc_status st = call(cs);
  if (!st && (e = cudaStreamSynchronize(cs)) != cudaSuccess) st = cuda_fail(c, e, "plan warm-up");
  dc_plan* p = nullptr;
  if (!st) {
    p = new dc_plan();
    p->c = c;
    if (cudaMalloc(&p->ws, std::max<size_t>(c->ws_bytes, 256)) != cudaSuccess ||
        cudaMalloc(&p->items, c->items_bytes) != cudaSuccess) {
      cudaGetLastError();
      st = fail(c, DC_ENOMEM, "plan buffers");
    }
  }
  if (!st) {
    char* ws0 = c->ws;
    char* it0 = c->items;
    std::vector<char> staging(c->items_bytes, 0);
    c->ws = p->ws;
    c->items = p->items;
    c->rec = &staging;
    const long long l0 = c->launches;
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      st = cuda_fail(c, e, "begin capture");
    } else {
      dc_status st2 = call(cs);
      e = cudaStreamEndCapture(cs, &graph);
      if (st2) st = st2;
      else if (e != cudaSuccess) st = cuda_fail(c, e, "end capture");
    }
    c->rec = nullptr;
    c->ws = ws0;
    c->items = it0;
    p->launches = c->launches - l0;
    c->launches = l0;
    if (!st && (e = cudaMemcpy(p->items, staging.data(), staging.size(), cudaMemcpyHostToDevice)) !=
                   cudaSuccess)
      st = cuda_fail(c, e, "plan item upload");
    if (!st && (e = cudaGraphInstantiate(&p->exec, graph, 0)) != cudaSuccess)
      st = cuda_fail(c, e, "graph instantiate");
    if (graph) cudaGraphDestroy(graph);
  }
  cudaStreamDestroy(cs);
  if (st) {
    if (p) {
      if (p->exec) cudaGraphExecDestroy(p->exec);
      if (p->ws) cudaFree(p->ws);
      if (p->items) cudaFree(p->items);
      delete p;
    }
    return st;
  }
  *out = p;
  return DC_OK;
}

}  // namespace

extern "C" dc_status dc_plan_batch(dc_ctx* c, const dc_c64* in, dc_c64* out, const dc_item* items,
                                   int n_items, const dc_opts* opts, dc_plan** plan) {
  if (!c || !plan) return DC_EINVAL;
  std::vector<dc_item> copy(items, items + (items ? n_items : 0));
  dc_opts o;
  dc_opts_default(&o);
  if (opts) o = *opts;
  return make_plan(
      c, [&](cudaStream_t s) { return correct_batch(c, in, out, copy.data(), n_items, &o, s); }, plan);
}

extern "C" dc_status dc_plan_bank(dc_ctx* c, const dc_c64* x, long long n, const double* v_r, int n_v,
                                  const double* tec, int n_tec, dc_c64* out, double fs, double fc,
                                  const dc_opts* opts, dc_plan** plan) {
  if (!c || !plan || !v_r || !tec || n_v < 1 || n_tec < 1) return DC_EINVAL;
  std::vector<double> v(v_r, v_r + n_v), t(tec, tec + n_tec);
  dc_opts o;
  dc_opts_default(&o);
  if (opts) o = *opts;
  return make_plan(
      c,
      [&](cudaStream_t s) {
        return correct_bank(c, x, n, v.data(), n_v, t.data(), n_tec, out, fs, fc, &o, s);
      },
      plan);
}

extern "C" dc_status dc_plan_execute(dc_plan* p, void* stream) {
  if (!p || !p->exec) return DC_EINVAL;
  cudaError_t e = cudaGraphLaunch(p->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(p->c, e, "graph launch");
  p->c->launches += p->launches;
  return DC_OK;
}

extern "C" long long dc_plan_launches(const dc_plan* p) { return p ? p->launches : -1; }

extern "C" dc_status dc_plan_destroy(dc_plan* p) {
  if (!p) return DC_EINVAL;
  cudaSetDevice(p->c->device);
  cudaDeviceSynchronize();
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->ws) cudaFree(p->ws);
  if (p->items) cudaFree(p->items);
  delete p;
  return DC_OK;
}

// ============================================================ autotuning
// A call's schedule choices measured on its own data: one choice at a time
// (resampler outputs per lane, then per length class the transform
// schedule, then the three-pass chunk size), each candidate run once to
// settle the scratch and then timed (best of three) with CUDA events, kept
// if it beats the best so far by more than 2 %.
namespace {

struct Choice {
  int kind;   // 0 resample_q, 1 fft[m], 2 chunk[m], 3 bank resampling engine, 4 spectrum-apply kind
  int m;
  std::vector<long long> values;
};

long long tune_get(const dc_ctx* c, const Choice& d) {
  if (d.kind == 4) return c->tune.apply_kind;
  if (d.kind == 3) return c->tune.rs_tc;
  if (d.kind == 0) return c->tune.rs_q;
  if (d.kind == 1) return c->tune.fft[d.m];
  return c->tune.chunk[d.m];
}
void tune_set(dc_ctx* c, const Choice& d, long long v) {
  if (d.kind == 4) c->tune.apply_kind = (int)v;
  else if (d.kind == 3) c->tune.rs_tc = (int)v;
  else if (d.kind == 0) c->tune.rs_q = (int)v;
  else if (d.kind == 1) c->tune.fft[d.m] = (int)v;
  else c->tune.chunk[d.m] = v;
}

template <class F>
dc_status time_call(dc_ctx* c, F& call, cudaStream_t s, double& ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return cuda_fail(c, e, "tuning events");
  }
  ms = 1e30;
  dc_status st = DC_OK;
  for (int r = 0; r < 3 && !st; ++r) {
    cudaEventRecord(a, s);
    st = call();
    cudaEventRecord(b, s);
    if (!st && (e = cudaEventSynchronize(b)) != cudaSuccess) st = cuda_fail(c, e, "tuning run");
    float t = 0.f;
    if (!st && cudaEventElapsedTime(&t, a, b) == cudaSuccess) ms = std::min(ms, (double)t);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}

void tuning_out(const dc_ctx* c, dc_tuning* t) {
  *t = dc_tuning{};
  t->resample_q = c->tune.rs_q;
  t->resample_tc = c->tune.rs_tc;
  t->apply_kind = c->tune.apply_kind;
  for (int m = 0; m <= 20; ++m) {
    t->fft[m] = c->tune.fft[m];
    t->chunk[m] = c->tune.chunk[m];
  }
}

template <class F>
dc_status autotune(dc_ctx* c, F&& call, std::vector<Choice> choices, cudaStream_t s,
                   dc_tuning* report) {
  if (c->rec) return fail(c, DC_EINVAL, "autotuning while a plan is being recorded");
  dc_status st = call();
  cudaError_t e;
  if (!st && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(c, e, "tuning warm-up");
  double ms_default = 0, best = 0;
  if (!st) st = time_call(c, call, s, ms_default);
  best = ms_default;
  int candidates = 1;
  for (const Choice& d : choices) {
    if (st) break;
    // the three-pass chunk matters only while the class runs three passes
    if (d.kind == 2 && d.m <= 16 && c->tune.fft[d.m] != 2) continue;
    const long long keep = tune_get(c, d);
    long long best_v = keep;
    for (long long v : d.values) {
      if (v == keep) continue;
      tune_set(c, d, v);
      st = call();                             // settle scratch for this schedule
      if (!st && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(c, e, "tuning run");
      double ms = 0;
      if (!st) st = time_call(c, call, s, ms);
      if (st) break;
      ++candidates;
      if (ms < 0.98 * best) {
        best = ms;
        best_v = v;
      }
    }
    tune_set(c, d, best_v);
  }
  if (!st) st = call();                        // outputs from the chosen schedule
  if (!st && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(c, e, "tuned run");
  if (st) return st;
  if (const char* path = getenv("DC_TUNING_CACHE")) dc_tuning_save(c, path);
  if (report) {
    tuning_out(c, report);
    report->ms_default = ms_default;
    report->ms_best = best;
    report->candidates = candidates;
  }
  return DC_OK;
}

// Choices a correct_batch / correct_bank call meets: per length class m.
void class_choices(std::vector<Choice>& ch, int m, size_t transforms) {
  if (m >= 12 && m <= 16) ch.push_back({1, m, {1, 2}});
  if (m >= 13) {
    const long long whole = (long long)transforms << (m + 3);
    std::vector<long long> v{-1};
    for (long long b : {256ll << 20, 64ll << 20, 16ll << 20})
      if (b < whole && b >= (8ll << m)) v.push_back(b);
    if (v.size() > 1) ch.push_back({2, m, v});
  }
}

}  // namespace

extern "C" dc_status dc_autotune_batch(dc_ctx* c, const dc_c64* in, dc_c64* out,
                                       const dc_item* items, int n_items, const dc_opts* opts,
                                       void* stream, dc_tuning* report) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  if (n_items < 0 || (n_items > 0 && !items)) return fail(c, DC_EINVAL, "bad item list");
  dc_opts o;
  dc_opts_default(&o);
  if (opts) o = *opts;
  std::vector<Choice> ch;
  std::vector<size_t> count(21, 0);
  bool q8 = false;
  for (int i = 0; i < n_items; ++i) {
    const long long no = items[i].n_out ? items[i].n_out : items[i].n;
    if (no < 1 || no > kMaxN) return fail(c, DC_EINVAL, "item %d: bad length", i);
    ++count[log2_ceil(no)];
    if (std::fabs(items[i].v_r) < kC) q8 |= resample_q(std::fabs(alpha_minus_one(items[i].v_r))) == 8;
  }
  if (o.mode == DC_WINDOWED && o.taps == 32 && q8) ch.push_back({0, 0, {8, 4}});
  for (int m = 0; m <= 20; ++m)
    if (count[m]) class_choices(ch, m, count[m]);
  cudaSetDevice(c->device);
  cudaStream_t s = S(stream);
  return autotune(
      c, [&]() { return correct_batch(c, in, out, items, n_items, &o, s); }, ch, s, report);
}

extern "C" dc_status dc_autotune_bank(dc_ctx* c, const dc_c64* x, long long n, const double* v_r,
                                      int n_v, const double* tec, int n_tec, dc_c64* out,
                                      double fs, double fc, const dc_opts* opts, void* stream,
                                      dc_tuning* report) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  if (n_v < 1 || n_tec < 1 || !v_r || !tec) return fail(c, DC_EINVAL, "bad bank lists");
  dc_opts o;
  dc_opts_default(&o);
  if (opts) o = *opts;
  const long long n_out = o.n_out ? o.n_out : n;
  if (n_out < 1 || n_out > kMaxN) return fail(c, DC_EINVAL, "bad length");
  std::vector<Choice> ch;
  bool q8 = false;
  for (int i = 0; i < n_v; ++i)
    if (std::fabs(v_r[i]) < kC) q8 |= resample_q(std::fabs(alpha_minus_one(v_r[i]))) == 8;
  if (o.mode == DC_WINDOWED && o.taps == 32 && !o.carrier_shift) ch.push_back({3, 0, {1, 2}});
  if (o.mode == DC_WINDOWED && o.taps == 32 && q8) ch.push_back({0, 0, {8, 4}});
  class_choices(ch, log2_ceil(n_out), (size_t)n_v * n_tec);
  if (log2_ceil(n_out) >= 13 && log2_ceil(n_out) <= 16)
    ch.push_back({4, 0, log2_ceil(n_out) >= 15 ? std::vector<long long>{1, 2, 3} : std::vector<long long>{1, 3}});
  cudaSetDevice(c->device);
  cudaStream_t s = S(stream);
  return autotune(
      c, [&]() { return correct_bank(c, x, n, v_r, n_v, tec, n_tec, out, fs, fc, &o, s); }, ch, s,
      report);
}

extern "C" dc_status dc_tuning_get(const dc_ctx* c, dc_tuning* out) {
  if (!c || !out) return DC_EINVAL;
  tuning_out(c, out);
  return DC_OK;
}

extern "C" dc_status dc_tuning_set(dc_ctx* c, const dc_tuning* t) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  if (!t) {
    c->tune = dc_ctx::Tune{};
    return DC_OK;
  }
  if (t->resample_q != 0 && t->resample_q != 4 && t->resample_q != 8)
    return fail(c, DC_EINVAL, "resample_q must be 0, 4 or 8");
  if (t->resample_tc < 0 || t->resample_tc > 2)
    return fail(c, DC_EINVAL, "resample_tc must be 0, 1 or 2");
  if (t->apply_kind < 0 || t->apply_kind > 3)
    return fail(c, DC_EINVAL, "apply_kind must be 0, 1, 2 or 3");
  for (int m = 0; m <= 20; ++m) {
    if (t->fft[m] < 0 || t->fft[m] > 2 || (t->fft[m] && (m < 12 || m > 16)))
      return fail(c, DC_EINVAL, "fft[%d] must be 0, 1 or 2 (and 0 outside 4096 <= L <= 65536)", m);
    if (t->chunk[m] < -1) return fail(c, DC_EINVAL, "chunk[%d] must be >= -1", m);
  }
  c->tune.rs_q = t->resample_q;
  c->tune.rs_tc = t->resample_tc;
  c->tune.apply_kind = t->apply_kind;
  for (int m = 0; m <= 20; ++m) {
    c->tune.fft[m] = t->fft[m];
    c->tune.chunk[m] = t->chunk[m];
  }
  return DC_OK;
}

// ------------------------------------------------- internal (serve loop)
// Scratch bytes a correct_batch call with these items needs on this context,
// and the call run with caller-provided scratch (the serving loop carves both
// from its HBM pool, so admission can account for every byte a batch uses).
size_t dc_internal_batch_scratch(dc_ctx* c, const dc_item* items, int n_items) {
  std::lock_guard<std::recursive_mutex> g(c->mu);
  return batch_layout(c, items, n_items).bytes;
}

dc_status dc_internal_correct_batch_ws(dc_ctx* c, const dc_c64* in, dc_c64* out,
                                       const dc_item* items, int n_items, const dc_opts* opts,
                                       void* stream, void* ws, size_t ws_bytes) {
  if (!c) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  char* ws0 = c->ws;
  const size_t b0 = c->ws_bytes;
  c->ws = static_cast<char*>(ws);
  c->ws_bytes = ws_bytes;
  const dc_status st = correct_batch(c, in, out, items, n_items, opts, stream);
  c->ws = ws0;
  c->ws_bytes = b0;
  return st;
}

// ------------------------------------------------------ schedule cache
// The context's schedule as a small JSON object, e.g.
//   {"format": "dc_tuning/1", "resample_q": 0, "resample_tc": 1,
//    "apply_kind": 0, "fft": {"16": 1}, "chunk": {"17": 67108864}}
// (only non-zero entries of fft / chunk are written).
namespace {

std::string tuning_json(const dc_ctx* c) {
  std::string s = "{\"format\": \"dc_tuning/1\", \"resample_q\": " + std::to_string(c->tune.rs_q) +
                  ", \"resample_tc\": " + std::to_string(c->tune.rs_tc) +
                  ", \"apply_kind\": " + std::to_string(c->tune.apply_kind) + ", \"fft\": {";
  bool first = true;
  for (int m = 0; m <= 20; ++m)
    if (c->tune.fft[m]) {
      s += (first ? "\"" : ", \"") + std::to_string(m) + "\": " + std::to_string(c->tune.fft[m]);
      first = false;
    }
  s += "}, \"chunk\": {";
  first = true;
  for (int m = 0; m <= 20; ++m)
    if (c->tune.chunk[m]) {
      s += (first ? "\"" : ", \"") + std::to_string(m) + "\": " + std::to_string(c->tune.chunk[m]);
      first = false;
    }
  return s + "}}\n";
}

// Minimal reader for the object tuning_json writes: a flat key -> integer map
// and two nested maps of decimal keys.  Returns false on anything else.
struct JsonIn {
  const char* p;
  void ws() { while (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t') ++p; }
  bool lit(char ch) { ws(); if (*p != ch) return false; ++p; return true; }
  bool str(std::string& out) {
    ws();
    if (*p != '"') return false;
    const char* e = strchr(p + 1, '"');
    if (!e) return false;
    out.assign(p + 1, e);
    p = e + 1;
    return true;
  }
  bool num(long long& v) {
    ws();
    char* e = nullptr;
    v = strtoll(p, &e, 10);
    if (e == p) return false;
    p = e;
    return true;
  }
};

bool parse_map(JsonIn& in, long long (&out)[21]) {
  if (!in.lit('{')) return false;
  in.ws();
  if (*in.p == '}') { ++in.p; return true; }
  while (true) {
    std::string k;
    long long v;
    if (!in.str(k) || !in.lit(':') || !in.num(v)) return false;
    char* e = nullptr;
    const long m = strtol(k.c_str(), &e, 10);
    if (!e || *e || m < 0 || m > 20) return false;
    out[m] = v;
    if (in.lit(',')) continue;
    return in.lit('}');
  }
}

bool parse_tuning(const std::string& text, dc_tuning& t) {
  t = dc_tuning{};
  long long fft[21] = {}, chunk[21] = {};
  JsonIn in{text.c_str()};
  if (!in.lit('{')) return false;
  bool format_ok = false;
  while (true) {
    std::string k;
    if (!in.str(k) || !in.lit(':')) return false;
    if (k == "format") {
      std::string f;
      if (!in.str(f)) return false;
      format_ok = f == "dc_tuning/1";
    } else if (k == "resample_q" || k == "resample_tc" || k == "apply_kind") {
      long long v;
      if (!in.num(v)) return false;
      (k == "resample_q" ? t.resample_q : k == "resample_tc" ? t.resample_tc : t.apply_kind) = (int)v;
    } else if (k == "fft" || k == "chunk") {
      if (!parse_map(in, k == "fft" ? fft : chunk)) return false;
    } else {
      return false;
    }
    if (in.lit(',')) continue;
    if (!in.lit('}')) return false;
    break;
  }
  for (int m = 0; m <= 20; ++m) {
    t.fft[m] = (int)fft[m];
    t.chunk[m] = chunk[m];
  }
  return format_ok;
}

}  // namespace

extern "C" dc_status dc_tuning_save(const dc_ctx* c, const char* path) {
  if (!c || !path) return DC_EINVAL;
  const std::string s = tuning_json(c);
  FILE* f = fopen(path, "w");
  if (!f) return DC_EINVAL;
  const bool ok = fwrite(s.data(), 1, s.size(), f) == s.size();
  return (fclose(f) == 0 && ok) ? DC_OK : DC_EINVAL;
}

extern "C" dc_status dc_tuning_load(dc_ctx* c, const char* path) {
  if (!c || !path) return DC_EINVAL;
  std::lock_guard<std::recursive_mutex> g(c->mu);
  FILE* f = fopen(path, "r");
  if (!f) return fail(c, DC_EINVAL, "cannot open schedule file %s", path);
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0 && text.size() < (1u << 20)) text.append(buf, k);
  fclose(f);
  dc_tuning t;
  if (!parse_tuning(text, t)) return fail(c, DC_EINVAL, "%s is not a dc_tuning/1 schedule", path);
  return dc_tuning_set(c, &t);
}
