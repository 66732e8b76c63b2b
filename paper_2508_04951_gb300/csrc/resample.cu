// Windowed and exact Whittaker-Shannon resampling kernels (Eq. 17, Sec. III-B).
//
// Windowed: y[n] = sum_i x[i] h(alpha n - i), h(u) = sinc(u) w(u), w a Kaiser
// window of half width R, support |u| < R, x zero outside [0, N).  With
// alpha n = n + delta n = m + e (e in [0,1)) the sum runs over i = m + k,
// k = -R+1..R, and sinc(e - k) = (-1)^k sin(pi e) / (pi (e - k)).
//
// Two kernels:
//  * direct (any alpha): one output per thread, every weight evaluated.  This
//    is the paper's Algorithm 1 shape and the library's general path.
//  * tiled (|alpha - 1| <= 0.01, 32 taps): a CTA owns 1024 consecutive outputs;
//    its input window is staged in shared memory by one TMA bulk copy; each
//    lane owns Q = 8 consecutive outputs (a warp 256) while e moves by at most
//    0.015 of a sample across a warp tile (|alpha - 1| <= 5.8e-5, |v_r| <=
//    8.7 km/s), else Q = 4 (|alpha - 1| <= 1.1e-4, |v_r| <= 17 km/s); each tap
//    weight is then the quadratic through its exact values at the warp tile's
//    first, middle and last output (error <= 2e-7).  Other warp tiles, and
//    tiles where floor(delta n) steps, use exact per-output weights read
//    against the same staged window.
#include "resample.cuh"

namespace dc {

constexpr float kInvPi = 0.318309886183790672f;
constexpr int kRsThreads = 256;

// w(e - k) from the per-tap polynomial, t = k + R - 1.
DC_DEV float window_at(const float* __restrict__ wp, int t, float e) {
  const float4 lo = __ldg(reinterpret_cast<const float4*>(wp + t * kWCoef));
  const float4 hi = __ldg(reinterpret_cast<const float4*>(wp + t * kWCoef + 4));
  float w = fmaf(hi.w, e, hi.z);
  w = fmaf(w, e, hi.y);
  w = fmaf(w, e, hi.x);
  w = fmaf(w, e, lo.w);
  w = fmaf(w, e, lo.z);
  w = fmaf(w, e, lo.y);
  return fmaf(w, e, lo.x);
}

// h(e - k) for tap k; s_e = sin(pi e)/pi.
DC_DEV float tap_weight(const RsArgs& a, float e, float s_e, int k) {
  const float u = e - (float)k;
  if (u == 0.f) return 1.f;
  const float sc = __fdividef((k & 1) ? -s_e : s_e, u);
  return sc * window_at(a.wpoly, k + a.half - 1, e);
}

// v exp(2 pi i g n) (the item's carrier rotation), or v when g = 0.
DC_DEV float2 rotate(float2 v, float g_hi, float g_lo, int n) {
  if (g_hi == 0.f && g_lo == 0.f) return v;
  return cmul(v, cycles_rot(g_hi, g_lo, n));
}

// The item owning a tile: the last item with tile_begin <= tile (tile_begin
// strictly increases).  One warp probes 32 evenly spaced items per round, so
// the search takes ceil(log32 n_items) dependent loads instead of log2.
// Every lane of the warp calls it and gets the answer.
DC_DEV int find_item(const RsArgs& a, int tile) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = a.n_items;                  // items[lo].tile_begin <= tile < items[hi]
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) >> 5;
    const int idx = lo + lane * step;
    const bool ok = idx < hi && a.items[idx].tile_begin <= tile;
    const unsigned m = __ballot_sync(0xffffffffu, ok);   // lane 0 always set
    lo += (31 - __clz((int)m)) * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

// ------------------------------------------------------------- direct
__global__ void __launch_bounds__(kRsThreads) resample_direct_kernel(RsArgs a) {
  pdl_release();                        // the transform that follows may start its set-up
  __shared__ int s_item;
  const int tile = blockIdx.x;
  if (threadIdx.x < 32) {
    const int it = find_item(a, tile);
    if (threadIdx.x == 0) s_item = it;
  }
  __syncthreads();
  const RsItem& I = a.items[s_item];
  const int o0 = (tile - I.tile_begin) * kRsTile;
  for (int q = 0; q < kRsTile / kRsThreads; ++q) {
    const int i = o0 + q * kRsThreads + threadIdx.x;
    if (i >= I.n_out) break;
    int fl;
    float e;
    rs_delay(I.dl_hi, I.dl_lo, (float)i, fl, e);
    const int m = i + fl;
    float2 acc = make_float2(0.f, 0.f);
    if (e == 0.f) {
      if (m >= 0 && m < I.n_in) acc = __ldg(I.x + m);
    } else {
      const float s_e = sinpif(e) * kInvPi;
      for (int k = -a.half + 1; k <= a.half; ++k) {
        const int idx = m + k;
        if ((unsigned)idx >= (unsigned)I.n_in) continue;
        const float h = tap_weight(a, e, s_e, k);
        const float2 v = __ldg(I.x + idx);
        acc.x = fmaf(v.x, h, acc.x);
        acc.y = fmaf(v.y, h, acc.y);
      }
    }
    I.y[i] = rotate(acc, I.rot_hi, I.rot_lo, i);
  }
}

// ---------------------------------------------------- frequency conversion
__global__ void __launch_bounds__(kRsThreads) freqconv_kernel(RsArgs a) {
  pdl_release();                        // the transform that follows may start its set-up
  __shared__ int s_item;
  const int tile = blockIdx.x;
  if (threadIdx.x < 32) {
    const int it = find_item(a, tile);
    if (threadIdx.x == 0) s_item = it;
  }
  __syncthreads();
  const RsItem& I = a.items[s_item];
  const int o0 = (tile - I.tile_begin) * kRsTile;
#pragma unroll
  for (int q = 0; q < kRsTile / kRsThreads; ++q) {
    const int i = o0 + q * kRsThreads + threadIdx.x;
    if (i >= I.n_out) break;
    const float2 v = i < I.n_in ? __ldg(I.x + i) : make_float2(0.f, 0.f);
    __stcs(I.y + i, rotate(v, I.rot_hi, I.rot_lo, i));
  }
}

// ------------------------------------------------------------- tiled
DC_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Q consecutive outputs per lane (4 or 8): a warp tile is 32 Q outputs and
// kRsTile / Q threads cover the 1024-output CTA tile.
constexpr int kWaitLimit = 1 << 22;      // bounded mbarrier polls
// Largest move of e across a warp tile for the quadratic weights: the
// interpolation error is about 0.064 |h'''| (span/2)^3 <= 2e-7 per weight.
constexpr float kQuadSpan = kRsQuadSpan;

// Bank-spread window layout: element i at i + i / Q, so that lane l's
// first tap input (Q l + const) lands on bank pair (Q + 1) l + const.
template <int LQ> DC_DEV int wpad(int i) { return i + (i >> LQ); }

// Inner product loop of one lane over all taps: outputs ow + Q lane + q,
// inputs at padded slice positions m + (m >> log2 Q) from the lane's base
// (the slice starts at the warp tile's first input, so every offset is a
// compile-time constant).  The Q inputs of a tap slide by one per tap, so
// each tap loads one new input and one weight quadruple.  The tile's
// quadratic weight h(s) = w.x + w.y s + w.z s^2 (w.w = 2 w.z) is evaluated
// once per lane at its centre sl, value and slope, and the Q outputs
// sl + u, |u| <= (Q - 1) / 2, take the tangent: the term w.z u^2 left out
// is about |h''| / 2 (u de/ds)^2 <= 7.1e-8 per weight (|h''| <= 3.32 for
// the 32-tap Kaiser(8) sinc; |de/ds| <= kRsQuadSpan / (32 Q - 1), so
// |u de/ds| <= 2.06e-4 at Q = 8 and 1.77e-4 at Q = 4).
template <int TAPS, int LQ>
DC_DEV void tap_loop(const float2* __restrict__ w0, const float4* __restrict__ wts,
                     float sl, float2 (&acc)[1 << LQ]) {
  constexpr int Q = 1 << LQ;
  float2 xw[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) xw[q] = w0[q + (q >> LQ)];
#pragma unroll
  for (int t = 0; t < TAPS; ++t) {
    const float4 w = wts[t];
    const float hl = fmaf(fmaf(w.z, sl, w.y), sl, w.x);
    const float dl = fmaf(w.w, sl, w.y);
    // packed two-lane FMAs, each lane rounding as fmaf does: the weight h
    // in both lanes, then both parts of the output at once
    const float2 hl2 = make_float2(hl, hl), dl2 = make_float2(dl, dl);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float u = (float)q - 0.5f * (float)(Q - 1);
      const float2 h2 = __ffma2_rn(dl2, make_float2(u, u), hl2);
      acc[q] = __ffma2_rn(xw[q], h2, acc[q]);
    }
#pragma unroll
    for (int q = 0; q + 1 < Q; ++q) xw[q] = xw[q + 1];
    if (t + 1 < TAPS) {
      const int m = Q + t;
      xw[Q - 1] = w0[m + (m >> LQ)];
    }
  }
}

template <int HALF, int LQ>
__global__ void __launch_bounds__(kRsTile >> LQ) resample_tiled_kernel(RsArgs a) {
  pdl_release();                        // the transform that follows may start its set-up
  constexpr int Q = 1 << LQ;
  constexpr int NT = kRsTile / Q;          // threads
  constexpr int W = 32 * Q;                // outputs per warp tile
  constexpr int TAPS = 2 * HALF;
  constexpr int NW = NT / 32;
  constexpr int WINMAX = kRsTile + 2 * HALF + 40;
  constexpr int WWIN = W + TAPS + 3;                   // a warp's slice (|f2 - f0| <= 4)
  constexpr int WSTRIDE = ((WWIN + (WWIN >> LQ) + 1) | 1) + 1;   // even: 16-byte aligned slices
  static_assert(WSTRIDE >= W, "a slice stages the warp's outputs");
  __shared__ __align__(16) float2 stage[WINMAX + 2];   // the CTA's window, by TMA
  __shared__ __align__(16) float2 win[NW * WSTRIDE];
  __shared__ float4 wts[NW][TAPS];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ int s_geo[6];                     // item, wlo, t0, t1, sh, window too long
  __shared__ int s_done;

  // Warp 0 finds the tile's item; its lane 0 sets out the CTA's input window
  // and starts the TMA copy, alone (nothing in this is needed twice).
  const int tile = blockIdx.x;
  if (threadIdx.x < 32) {
    const int it = find_item(a, tile);
    if (threadIdx.x == 0) {
      const RsItem& J = a.items[it];
      const int p0 = (tile - J.tile_begin) * kRsTile;
      int flA, flB;
      float eA, eB;
      rs_delay(J.dl_hi, J.dl_lo, (float)p0, flA, eA);
      rs_delay(J.dl_hi, J.dl_lo, (float)(p0 + kRsTile - 1), flB, eB);
      const int flmin = min(flA, flB) - 2, flmax = max(flA, flB) + 2;
      const int lo = p0 + flmin - HALF + 1;
      const int hi = p0 + kRsTile - 1 + flmax + HALF;
      const bool too_long = hi - lo + 1 > WINMAX;   // |delta| outside the tiled range
      // the 16-byte-aligned interior of the valid part, by one bulk copy
      const int vlo = max(lo, 0), vhi = min(hi, J.n_in - 1);
      int u0 = vlo, u1 = vhi + 1;
      if (u1 > u0 && (reinterpret_cast<uintptr_t>(J.x + u0) & 15)) ++u0;
      if (u1 > u0 && ((u1 - u0) & 1)) --u1;
      if (u1 < u0) u1 = u0;
      const int shift = (u0 - lo) & 1;
      s_geo[0] = it;
      s_geo[1] = lo;
      s_geo[2] = u0;
      s_geo[3] = u1;
      s_geo[4] = shift;
      s_geo[5] = too_long;
      const uint32_t bytes = (uint32_t)(u1 - u0) * 8u;
      if (!too_long && bytes) {
        const uint32_t mb = smem_u32(&mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(stage + (u0 - lo + shift))),
            "l"(J.x + u0), "r"(bytes), "r"(mb)
            : "memory");
      }
    }
  }
  __syncthreads();
  const RsItem& I = a.items[s_geo[0]];
  const int o0 = (tile - I.tile_begin) * kRsTile;
  const int wlo = s_geo[1], t0 = s_geo[2], t1 = s_geo[3], sh = s_geo[4];
  if (s_geo[5]) {
    if (threadIdx.x == 0) atomicMax(a.err, 2);
    return;
  }
  if (t1 > t0) {
    // thread 0 waits for the copy (bounded); the others wait at the barrier
    if (threadIdx.x == 0) {
      const uint32_t mb = smem_u32(&mbar);
      uint32_t done = 0;
      for (int it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mb)
            : "memory");
      }
      if (!done) {
        atomicMax(a.err, 1);
        for (int it = 0; it < kWaitLimit && !done; ++it) {   // the copy must land before the exit
          asm volatile(
              "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
              : "=r"(done)
              : "r"(mb)
              : "memory");
        }
      }
      s_done = done;
    }
    __syncthreads();
    if (!s_done) return;
  }
  // Each warp repacks its own slice of the window -- global positions
  // G .. G + WWIN - 1, G = ow + min(f0, f2) - HALF + 1 -- into a private,
  // bank-spread region, so tap offsets are compile-time constants and no CTA
  // barrier follows; the region then stages the warp's outputs.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ow = o0 + warp * W;
  if (ow >= I.n_out) return;                   // warp-uniform: nothing to write
  constexpr float H = 0.5f * (W - 1);
  // the warp tile's first, centre and last positions: one per lane 0..2
  int fl_l;
  float e_l;
  rs_delay(I.dl_hi, I.dl_lo, lane == 0 ? (float)ow : lane == 1 ? (float)ow + H : (float)(ow + W - 1),
           fl_l, e_l);
  const float s_l = sinpif(e_l) * kInvPi;
  const int f0 = __shfl_sync(0xffffffffu, fl_l, 0), f1 = __shfl_sync(0xffffffffu, fl_l, 1),
            f2 = __shfl_sync(0xffffffffu, fl_l, 2);
  const float e0 = __shfl_sync(0xffffffffu, e_l, 0), e1 = __shfl_sync(0xffffffffu, e_l, 1),
              e2 = __shfl_sync(0xffffffffu, e_l, 2);
  if (abs(f2 - f0) > 4) {                      // |delta| too large for the slice
    if (lane == 0) atomicMax(a.err, 2);
    return;
  }
  const int fmin = min(f0, f2);
  const int G = ow + fmin - HALF + 1;
  float2* ww = win + warp * WSTRIDE;
  for (int i = lane; i < WWIN; i += 32) {
    const int gi = G + i;
    float2 v = make_float2(0.f, 0.f);
    if (gi >= t0 && gi < t1) {
      if (DC_IN_BOUNDS(gi - wlo + sh >= 0 && gi - wlo + sh < WINMAX + 2, a.err)) v = stage[gi - wlo + sh];
    } else if (gi >= 0 && gi < I.n_in) {
      v = __ldg(I.x + gi);
    }
    if (DC_IN_BOUNDS(wpad<LQ>(i) < WSTRIDE, a.err)) ww[wpad<LQ>(i)] = v;
  }
  __syncwarp();

  float2 acc[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) acc[q] = make_float2(0.f, 0.f);
  if (f0 == f2 && f0 == f1 && fabsf(e2 - e0) <= kQuadSpan) {
    // Quadratic weights per tap through the three nodes s = -H, 0, +H.
    const float s0 = __shfl_sync(0xffffffffu, s_l, 0), s1 = __shfl_sync(0xffffffffu, s_l, 1),
                s2 = __shfl_sync(0xffffffffu, s_l, 2);
    for (int t = lane; t < TAPS; t += 32) {
      const int k = t - HALF + 1;
      const float hA = tap_weight(a, e0, s0, k);
      const float hB = tap_weight(a, e1, s1, k);
      const float hC = tap_weight(a, e2, s2, k);
      const float q1 = (hC - hA) * (0.5f / H);
      const float q2 = (hC - 2.f * hB + hA) * (0.5f / (H * H));
      wts[warp][t] = make_float4(hB, q1, q2, 2.f * q2);
    }
    __syncwarp();
    // Output ow + Q lane + q at tap t reads slice position Q lane + q + t,
    // padded (Q + 1) lane + m + (m >> log2 Q) with m = q + t.
    const float sl = (float)(lane * Q) + 0.5f * (float)(Q - 1) - H;   // the lane's centre
    tap_loop<TAPS, LQ>(ww + (Q + 1) * lane, wts[warp], sl, acc);
  } else {
    // floor(delta n) steps inside this warp tile, or e moves too far:
    // exact weights per output.
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int i = ow + lane * Q + q;
      int fl;
      float e;
      rs_delay(I.dl_hi, I.dl_lo, (float)i, fl, e);
      const int base = (i - ow) + (fl - fmin) + HALF - 1;   // slice position of tap k = 0
      if (e == 0.f) {
        acc[q] = ww[wpad<LQ>(base)];
      } else {
        const float s_e = sinpif(e) * kInvPi;
        for (int k = -HALF + 1; k <= HALF; ++k) {
          const float h = tap_weight(a, e, s_e, k);
          const float2 v = ww[wpad<LQ>(base + k)];
          acc[q].x = fmaf(v.x, h, acc[q].x);
          acc[q].y = fmaf(v.y, h, acc[q].y);
        }
      }
    }
  }
  // Stage the warp's W outputs in its slice (16-byte slots, XOR-swizzled so
  // lanes 4 slots apart use distinct banks), then store them coalesced.
  __syncwarp();
  float4* s4 = reinterpret_cast<float4*>(ww);
#pragma unroll
  for (int q = 0; q < Q / 2; ++q) {
    const int f = lane * (Q / 2) + q;
    s4[f ^ ((f >> 3) & 7)] = make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y);
  }
  __syncwarp();
  const int n_here = min(W, I.n_out - ow);
  float2* y = I.y + ow;
  const bool rot = I.rot_hi != 0.f || I.rot_lo != 0.f;    // carrier term
  if ((reinterpret_cast<uintptr_t>(y) & 15) == 0) {
    for (int p = lane; 2 * p + 1 < n_here; p += 32) {
      float4 t = s4[p ^ ((p >> 3) & 7)];
      if (rot) {
        const float2 u = rotate(make_float2(t.x, t.y), I.rot_hi, I.rot_lo, ow + 2 * p);
        const float2 w = rotate(make_float2(t.z, t.w), I.rot_hi, I.rot_lo, ow + 2 * p + 1);
        t = make_float4(u.x, u.y, w.x, w.y);
      }
      __stcs(reinterpret_cast<float4*>(y) + p, t);
    }
    if ((n_here & 1) && lane == 0) {
      const int p = (n_here - 1) >> 1;
      const float4 t = s4[p ^ ((p >> 3) & 7)];
      y[n_here - 1] = rotate(make_float2(t.x, t.y), I.rot_hi, I.rot_lo, ow + n_here - 1);
    }
  } else {
    for (int p = lane; p < n_here; p += 32) {
      const int f = p >> 1;
      const float4 t = s4[f ^ ((f >> 3) & 7)];
      y[p] = rotate((p & 1) ? make_float2(t.z, t.w) : make_float2(t.x, t.y), I.rot_hi, I.rot_lo,
                    ow + p);
    }
  }
}

cudaError_t launch_resample_tiled32(const RsArgs& a, int q, cudaStream_t s) {
  if (a.n_tiles <= 0) return cudaSuccess;
  if (q == 8) resample_tiled_kernel<16, 3><<<a.n_tiles, kRsTile / 8, 0, s>>>(a);
  else if (q == 4) resample_tiled_kernel<16, 2><<<a.n_tiles, kRsTile / 4, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_freqconv(const RsArgs& a, cudaStream_t s) {
  if (a.n_tiles <= 0) return cudaSuccess;
  freqconv_kernel<<<a.n_tiles, kRsThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_resample_direct(const RsArgs& a, cudaStream_t s) {
  if (a.n_tiles <= 0) return cudaSuccess;
  resample_direct_kernel<<<a.n_tiles, kRsThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------- exact sinc, FP32 cores
// Y[p][n] = sum_m X[p][m] S[n][m], S[n][m] = sinc(alpha n - m)
//         = (-1)^(m + m_n) sin(pi e_n) / (pi ((m_n - m) + e_n)),  alpha n = m_n + e_n.
// CTA tile: 64 outputs x 32 pulses, K chunks of 32 samples; S generated in
// shared memory per chunk and reused by all 32 pulses.
constexpr int kExBN = 64, kExBP = 32, kExBK = 32;

__global__ void __launch_bounds__(256) exact_fp32_kernel(ExArgs a) {
  const ExItem& I = a.items[blockIdx.z];
  const int n0 = blockIdx.x * kExBN, p0 = blockIdx.y * kExBP;
  __shared__ float Ss[kExBK][kExBN + 4];
  __shared__ float2 Xs[kExBK][kExBP + 1];
  __shared__ float sig[kExBN], en[kExBN];
  __shared__ int mn[kExBN];
  const int tid = threadIdx.x;
  if (tid < kExBN) {
    const int n = n0 + tid;
    int fl;
    float e;
    rs_delay(I.dl_hi, I.dl_lo, (float)n, fl, e);
    const int m = n + fl;
    mn[tid] = m;
    en[tid] = e;
    const float s = sinpif(e) * kInvPi;
    sig[tid] = (m & 1) ? -s : s;
  }
  const int tn = tid & 15, tp = tid >> 4;        // 4 outputs x 2 pulses per thread
  float2 acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
  __syncthreads();

  for (int m0 = 0; m0 < a.n_in; m0 += kExBK) {
    for (int idx = tid; idx < kExBK * kExBN; idx += 256) {
      const int n = idx % kExBN, k = idx / kExBN;
      const int m = m0 + k;
      float v = 0.f;
      if (m < a.n_in) {
        if (en[n] == 0.f) {
          v = (m == mn[n]) ? 1.f : 0.f;
        } else {
          const float den = (float)(mn[n] - m) + en[n];
          v = __fdividef((m & 1) ? -sig[n] : sig[n], den);
        }
      }
      Ss[k][n] = v;
    }
    for (int idx = tid; idx < kExBK * kExBP; idx += 256) {
      const int k = idx % kExBK, p = idx / kExBK;
      const int m = m0 + k, pp = p0 + p;
      Xs[k][p] = (m < a.n_in && pp < a.n_pulses) ? __ldg(I.x + (size_t)pp * a.n_in + m)
                                                  : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kExBK; ++k) {
      const float4 s4 = *reinterpret_cast<const float4*>(&Ss[k][tn * 4]);
      const float2 x0 = Xs[k][tp * 2], x1 = Xs[k][tp * 2 + 1];
      const float s[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i][0].x = fmaf(x0.x, s[i], acc[i][0].x);
        acc[i][0].y = fmaf(x0.y, s[i], acc[i][0].y);
        acc[i][1].x = fmaf(x1.x, s[i], acc[i][1].x);
        acc[i][1].y = fmaf(x1.y, s[i], acc[i][1].y);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = n0 + tn * 4 + i;
    if (n >= a.n_out) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int p = p0 + tp * 2 + j;
      if (p < a.n_pulses) I.y[(size_t)p * a.n_out + n] = rotate(acc[i][j], I.rot_hi, I.rot_lo, n);
    }
  }
}

// The same sum for a few pulses (a matrix-vector product: one pulse per
// call of the single-pulse entry points): one warp per output sample, lanes
// striding the input, the weight computed once per (n, m) and applied to
// every pulse, lanes combined by a fixed shuffle tree (deterministic).
// One lane's share of the sum: terms m = lane, lane + 32, ... (FAST: m_n - m
// converted by exact_i2f, valid for |m_n - m| < 2^22).  Four terms per round:
// their weights, then their loads, issued together so that a warp has four
// loads in flight instead of one (the kernel is bound by the load latency);
// the terms are still added in the order m = lane, lane + 32, ...
template <bool FAST> DC_DEV float gemv_weight(int mn, int m, float e, float sgl) {
  const float den = (FAST ? exact_i2f(mn - m) : (float)(mn - m)) + e;
  return __fdividef(sgl, den);
}
template <int P, bool FAST>
DC_DEV void gemv_terms(const float2* __restrict__ x, int n_in, int np, int mn, float e, float sgl,
                       int lane, float2 (&acc)[P]) {
  int m = lane;
  for (; m + 96 < n_in; m += 128) {
    float w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) w[u] = gemv_weight<FAST>(mn, m + 32 * u, e, sgl);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      if (p < np) {
        float2 xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = __ldg(x + (size_t)p * n_in + m + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc[p].x = fmaf(xv[u].x, w[u], acc[p].x);
          acc[p].y = fmaf(xv[u].y, w[u], acc[p].y);
        }
      }
    }
  }
  for (; m < n_in; m += 32) {
    const float w = gemv_weight<FAST>(mn, m, e, sgl);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      if (p < np) {
        const float2 xv = __ldg(x + (size_t)p * n_in + m);
        acc[p].x = fmaf(xv.x, w, acc[p].x);
        acc[p].y = fmaf(xv.y, w, acc[p].y);
      }
    }
  }
}

template <int P>
__global__ void __launch_bounds__(256) exact_gemv_kernel(ExArgs a) {
  pdl_release();                        // the transform that follows may start its set-up
  const ExItem& I = a.items[blockIdx.y];
  const int n = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (n >= a.n_out) return;
  const int np = a.n_pulses;
  int fl;
  float e;
  rs_delay(I.dl_hi, I.dl_lo, (float)n, fl, e);
  const int mn = n + fl;
  if (e == 0.f) {                                  // alpha n on a sample: copy it
    if (lane < np) {
      const bool in = mn >= 0 && mn < a.n_in;
      const float2 v = in ? __ldg(I.x + (size_t)lane * a.n_in + mn) : make_float2(0.f, 0.f);
      I.y[(size_t)lane * a.n_out + n] = rotate(v, I.rot_hi, I.rot_lo, n);
    }
    return;
  }
  const float s = sinpif(e) * kInvPi;
  const float sg = (mn & 1) ? -s : s;
  const float sgl = (lane & 1) ? -sg : sg;         // (-1)^m: m steps by 32 from lane
  float2 acc[P];
#pragma unroll
  for (int p = 0; p < P; ++p) acc[p] = make_float2(0.f, 0.f);
  // m_n - m lies in (m_n - n_in, m_n]; below 2^22 in size (any Doppler
  // range rate) it converts exactly without the quarter-rate instruction
  if (mn < (1 << 22)) gemv_terms<P, true>(I.x, a.n_in, np, mn, e, sgl, lane, acc);
  else gemv_terms<P, false>(I.x, a.n_in, np, mn, e, sgl, lane, acc);
#pragma unroll
  for (int p = 0; p < P; ++p) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[p].x += __shfl_xor_sync(0xffffffffu, acc[p].x, o);
      acc[p].y += __shfl_xor_sync(0xffffffffu, acc[p].y, o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (p < np) I.y[(size_t)p * a.n_out + n] = rotate(acc[p], I.rot_hi, I.rot_lo, n);
  }
}

cudaError_t launch_exact_fp32(const ExArgs& a, int n_alpha, cudaStream_t s) {
  if (n_alpha <= 0 || a.n_out <= 0 || a.n_pulses <= 0) return cudaSuccess;
  if (a.n_pulses <= 8) {
    dim3 grid((a.n_out + 7) / 8, n_alpha);
    if (a.n_pulses == 1) exact_gemv_kernel<1><<<grid, 256, 0, s>>>(a);
    else if (a.n_pulses <= 2) exact_gemv_kernel<2><<<grid, 256, 0, s>>>(a);
    else if (a.n_pulses <= 4) exact_gemv_kernel<4><<<grid, 256, 0, s>>>(a);
    else exact_gemv_kernel<8><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  dim3 grid((a.n_out + kExBN - 1) / kExBN, (a.n_pulses + kExBP - 1) / kExBP, n_alpha);
  exact_fp32_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dc
