// Doppler resampling y[n] = x(alpha n Ts) (Eq. 2) by windowed and exact
// Whittaker-Shannon interpolation (Eq. 17; Sec. III-B; Table I).
#pragma once

#include "common.cuh"

namespace dc {

constexpr int kMaxHalf = 32;      // taps <= 64
constexpr int kWCoef = 8;         // window polynomial coefficients per tap (degree 7)

// One pulse of a windowed-resample launch.
struct RsItem {
  const float2* x;     // input samples [n_in]
  float2* y;           // output samples [n_out]
  int n_in, n_out;
  float dl_hi, dl_lo;  // delta = alpha - 1 as a double-float
  int tile_begin;      // first kRsTile-output tile of this item in the launch
  // Output n is multiplied by exp(2 pi i g n), g = rot_hi + rot_lo cycles per
  // sample (0: no rotation): the carrier term fc (alpha - 1) / fs of a
  // passband dilation, or the tone of frequency conversion.
  float rot_hi, rot_lo;
};

struct RsArgs {
  const RsItem* items;
  int n_items;
  int n_tiles;         // total tiles of the launch
  int half;            // R = taps / 2
  // Kaiser window of tap k at fractional delay e in [0, 1]:
  //   w(e - k) = sum_d wpoly[t * kWCoef + d] e^d,  t = k + R - 1
  // (fitted per tap in FP64 on the host; |error| <= 6e-8 for beta <= 20).
  const float* wpoly;
  int* err;            // device error flag (bounded waits)
};

// One alpha of an exact-sinc launch (config: n_pulses pulses share alpha).
struct ExItem {
  const float2* x;     // [n_pulses][n_in]
  float2* y;           // [n_pulses][n_out]
  float dl_hi, dl_lo;
  float rot_hi, rot_lo;  // carrier term, as in RsItem (0: none)
};
struct ExArgs {
  const ExItem* items; // one per alpha (grid.z)
  int n_in, n_out, n_pulses;
};

// delta * fi = fl + e with fl integer and e in [0, 1), fi a float holding an
// integer or half-integer output position (exact), delta a double-float.
DC_DEV void rs_delay(float dl_hi, float dl_lo, float fi, int& fl, float& e) {
  df p = two_prod(dl_hi, fi);
  const float lo = fmaf(dl_lo, fi, p.lo);
  float f = floorf(p.hi);
  float r = __fadd_rn(__fsub_rn(p.hi, f), lo);      // p.hi - f is exact
  if (r < 0.f) {
    r = __fadd_rn(r, 1.f);
    f -= 1.f;
    if (r >= 1.f) { r = 0.f; f += 1.f; }
  } else if (r >= 1.f) {
    r = __fsub_rn(r, 1.f);
    f += 1.f;
  }
  fl = (int)f;
  e = r;
}

// One launch of the tensor-core bank resampler (rs_tc.cu): one pulse x[n_in]
// for n_slots range rates, slot s holding delta = dl[2s] + dl[2s+1] and
// writing y + vidx[s] * n_out (vidx < 0: an empty slot).  Slots are grouped
// 32 per CTA; within a group the range rates' integer offsets
// floor(delta n) over any 128-output tile must span at most
// rs_tc_max_span() samples (the host orders the slots by delta and checks).
struct RsTcArgs {
  const float2* x;
  int n_in, n_out;
  float2* y;
  const float* dl;
  const int* vidx;
  int n_slots;
  const float* wpoly;  // 32-tap window polynomials and their first two
                       // derivatives: [tap][3][kWCoef] (w, w', w'' in e)
  int* err;
};
int rs_tc_max_span();
cudaError_t launch_resample_tc(const RsTcArgs& a, cudaStream_t s);

constexpr int kRsTile = 1024;     // outputs per CTA of the resampling kernels
constexpr float kRsTiledMaxDelta = 0.01f;
// The tiled kernel's warp tile is 32 q outputs (q = 8 or 4 per lane); its
// per-tap quadratic weights need e to move at most kRsQuadSpan across it,
// else the tile falls back to exact weights: q = 8 while
// |delta| (256 - 1) <= kRsQuadSpan, q = 4 above.
constexpr float kRsQuadSpan = 0.015f;
inline int resample_q(double delta_abs) { return delta_abs * 255.0 <= 0.98 * kRsQuadSpan ? 8 : 4; }

cudaError_t launch_resample_tiled32(const RsArgs& a, int q, cudaStream_t s);
// Frequency conversion (Sec. I, Table I): y[n] = x[n] exp(2 pi i g n) for
// n < n_out, x = 0 beyond n_in; g from the items' rotation fields.
cudaError_t launch_freqconv(const RsArgs& a, cudaStream_t s);
cudaError_t launch_resample_direct(const RsArgs& a, cudaStream_t s);
cudaError_t launch_exact_fp32(const ExArgs& a, int n_alpha, cudaStream_t s);

}  // namespace dc
