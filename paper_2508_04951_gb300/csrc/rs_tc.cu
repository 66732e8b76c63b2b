// Windowed-sinc resampling of one pulse for many range rates as a
// tensor-core contraction (Eq. 17 truncated to the Kaiser window, Sec. III-B
// and Table I; the Doppler bank, where every range rate reads the same input).
//
// With delta_v = alpha_v - 1 the resampled pulse is
//
//   y_v[n] = sum_u x[n + u] h(delta_v n - u),   h = sinc * Kaiser window,
//
// a sum over the input around the output's own index.  Over a tile of 128
// consecutive outputs centred at n_c, delta_v n moves by at most
// |delta_v| 64 (2e-4 of a sample at 8 km/s), so h is taken to second order
// about the centre:
//
//   h(a + tau) = h(a) + tau h'(a) + tau^2/2 h''(a),
//   a = delta_v n_c - u,  tau = delta_v (n - n_c).
//
// The tile's three sums Z_d[n][v] = sum_u x[n + u] h^(d)(delta_v n_c - u) are
// then one real GEMM per real and imaginary part: A[n][k] = x[n0 + n + u0 + k]
// (a Hankel tile of the input, shared by all range rates) times
// B[k][(d, v)] = h^(d)(e_v - j), the tap weights of range rate v at the tile
// centre (delta_v n_c = m_v + e_v, j = u0 + k - m_v in -15 .. 16, zero
// elsewhere).  The epilogue forms y = Z_0 + tau (Z_1 + tau/2 Z_2).  The
// Taylor remainder is below 2e-7 of a tap, and where the window's support
// edge falls inside the tile (h is continuous there, h' jumps by 1.4e-4)
// below 5e-7.
//
// The GEMM runs on tcgen05 (kind::f16, M = 128, N = 96: 32 range rates x 3
// derivatives, K up to 64) with fp16 hi/lo split operands and FP32
// accumulation in tensor memory: A_hi B_hi + A_hi B_lo + A_lo B_hi.  The
// input window is scaled by a power of two so its largest sample is below
// 1 (no fp16 overflow or underflow of the high parts); the epilogue undoes it.
// One CTA per (tile of 128 outputs, group of 32 range rates): 256 threads
// build the operands in shared memory (64-byte-swizzled K-major), one thread
// issues the MMAs, all eight warps read the accumulators back.
#include <cuda_fp16.h>

#include <climits>

#include "resample.cuh"
#include "tc.cuh"

namespace dc {

namespace {

constexpr int kTile = 128;              // outputs per CTA (the MMA's M)
constexpr int kV = 32;                  // range rates per CTA
constexpr int kN = 3 * kV;              // MMA N: (derivative, range rate)
constexpr int kKMax = 64;               // two 32-element swizzle atoms
constexpr int kAPlane = kTile * 64;     // 8 KiB: 128 rows x 32 fp16
constexpr int kBPlane = kN * 64;        // 6 KiB: 96 rows x 32 fp16
constexpr int kA = 2 * 4 * kAPlane;     // atoms x (re hi, re lo, im hi, im lo)
constexpr int kB = 2 * 2 * kBPlane;     // atoms x (hi, lo)
constexpr int kWin = kTile + kKMax;     // input window samples
constexpr int kSmem = kA + kB + 1024;   // + alignment slack
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 256;     // 2 x 96 accumulator columns
constexpr float kPi = 3.14159265358979f;
constexpr float kInvPi = 0.318309886183790672f;

// sinc and its first two derivatives at a = e - j, from S = sin(pi a) and
// C = cos(pi a):  sinc = S / (pi a),  sinc' = (C - sinc) / a,
// sinc'' = (-pi S - 2 sinc') / a.  Near a = 0 these cancel, so |a| < 1/4
// takes the Maclaurin series (pi a)^2 k terms to k = 5 instead.
DC_DEV void sinc_d012(float a, float S, float C, float& s0, float& s1, float& s2) {
  if (fabsf(a) < 0.25f) {
    const float z = kPi * a, z2 = z * z;
    // sinc = sum (-1)^k z^2k / (2k+1)!, and its derivatives in a
    s0 = 1.f + z2 * (-1.f / 6 + z2 * (1.f / 120 + z2 * (-1.f / 5040 + z2 * (1.f / 362880 +
                                                                          z2 * (-1.f / 39916800)))));
    const float d1 = -1.f / 3 + z2 * (1.f / 30 + z2 * (-1.f / 840 + z2 * (1.f / 45360 +
                                                                        z2 * (-1.f / 3991680))));
    s1 = kPi * z * d1;                                  // d/da = pi d/dz
    const float d2 = -1.f / 3 + z2 * (1.f / 10 + z2 * (-1.f / 168 + z2 * (1.f / 6480 +
                                                                        z2 * (-1.f / 443520))));
    s2 = kPi * kPi * d2;
  } else {
    const float ia = 1.f / a;
    s0 = S * kInvPi * ia;
    s1 = (C - s0) * ia;
    s2 = (-kPi * S - 2.f * s1) * ia;
  }
}

// Shared-memory pitch of one tap's three coefficient rows: 28 floats
// (112 bytes), so that lanes on taps up to 8 apart read different banks
// (at 24 floats, taps 4 apart collided).
constexpr int kWPitch = 3 * kWCoef + 4;

// Window w(e - j) and its first two derivatives in e from tap t's degree-7
// polynomial and its derivative polynomials (t = j + 15), staged in shared
// memory as [tap][kWPitch] (value, first- and second-derivative rows of
// kWCoef coefficients each).
DC_DEV void window_d012(const float* wp, int t, float e, float& w0, float& w1, float& w2) {
  const float4* q = reinterpret_cast<const float4*>(wp + t * kWPitch);
  const float4 a0 = q[0], a1 = q[1], b0 = q[2], b1 = q[3], c0 = q[4], c1 = q[5];
  w0 = fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(a1.w, e, a1.z), e, a1.y), e, a1.x), e, a0.w), e, a0.z), e, a0.y),
            e, a0.x);
  w1 = fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(b1.z, e, b1.y), e, b1.x), e, b0.w), e, b0.z), e, b0.y), e, b0.x);
  w2 = fmaf(fmaf(fmaf(fmaf(fmaf(c1.y, e, c1.x), e, c0.w), e, c0.z), e, c0.y), e, c0.x);
}

DC_DEV uint32_t pack_half2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// 8 values -> fp16 hi chunk and fp16 lo chunk (lo = rn(v - hi)).
DC_DEV void split8_f16(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2 a = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
    h[i] = *reinterpret_cast<const uint32_t*>(&a);
    l[i] = pack_half2(v[2 * i] - __low2float(a), v[2 * i + 1] - __high2float(a));
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__global__ void __launch_bounds__(kThreads, 2) rs_tc_kernel(RsTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ float2 win[kWin];
  __shared__ __align__(16) float s_wp[32 * kWPitch];
  __shared__ int s_m[kV], s_vidx[kV];
  __shared__ float s_e[kV], s_sin[kV], s_cos[kV], s_dl[kV];
  __shared__ int s_maxbits;
  __shared__ int s_mlo, s_kk;
  __shared__ __align__(8) unsigned long long mma_bar;
  __shared__ uint32_t tmem_base;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* A = smem;
  uint8_t* B = smem + kA;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * kTile;
  const int g0 = blockIdx.y * kV;
  const float nc = (float)n0 + 0.5f * (kTile - 1);          // tile centre (half-integer, exact)

  for (int i = threadIdx.x; i < 32 * 3 * kWCoef; i += kThreads)
    s_wp[(i / (3 * kWCoef)) * kWPitch + i % (3 * kWCoef)] = __ldg(a.wpoly + i);
  // 1. per range rate: delta_v n_c = m_v + e_v, and the K range of the tile
  if (warp == 0) {
    const int slot = g0 + lane;
    int m = 0, vidx = -1;
    float e = 0.f, dlh = 0.f;
    if (slot < a.n_slots) {
      vidx = a.vidx[slot];
      dlh = a.dl[2 * slot];
      rs_delay(dlh, a.dl[2 * slot + 1], nc, m, e);
    }
    float sn, cs;
    sincospif(e, &sn, &cs);
    s_m[lane] = m;
    s_e[lane] = e;
    s_sin[lane] = sn;
    s_cos[lane] = cs;
    s_dl[lane] = dlh;
    s_vidx[lane] = vidx;
    int lo = vidx >= 0 ? m : INT_MAX, hi = vidx >= 0 ? m : INT_MIN;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      const int span = hi - lo;                // range-rate offsets inside the tile
      s_mlo = lo;
      s_kk = span > kKMax - 32 ? -1 : ((32 + span + 15) / 16) * 16;
      s_maxbits = 0;
      mbar_init(&mma_bar, 1);
    }
  } else if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int KK = s_kk;
  const int u0 = s_mlo - 15;                   // A column k holds x[n0 + row + u0 + k]
  bool run = KK > 0;
  int ex = 0;                                  // the window's scale exponent
  if (!run && threadIdx.x == 0) atomicMax(a.err, 2);   // range rates spread too far

  if (run) {
    // 2. input window x[n0 + u0 .. + kTile + KK - 1] (zero outside the pulse)
    //    and its largest magnitude
    float mx = 0.f;
    for (int i = threadIdx.x; i < kTile + KK; i += kThreads) {
      const int gi = n0 + u0 + i;
      const float2 v = (gi >= 0 && gi < a.n_in) ? __ldg(a.x + gi) : make_float2(0.f, 0.f);
      if (DC_IN_BOUNDS(i < kWin, a.err)) win[i] = v;
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // non-negative floats (and +inf, NaN above them) order as their bit
    // patterns, so the block maximum is an integer atomic max
    if (lane == 0) atomicMax(&s_maxbits, __float_as_int(mx));
    __syncthreads();
    {
      const float m = __int_as_float(s_maxbits);
      if (m > 0.f && isfinite(m)) frexpf(m, &ex);      // m = f 2^ex, f in [0.5, 1)
    }
    const float scale = ldexpf(1.f, -ex);

    // 3. A: Hankel tile, 16-byte chunks of 8 columns, four planes per atom.
    //    A weight chunk (step 4) costs about six Hankel chunks, so the
    //    threads without one (threadIdx.x >= chunks_b) take qa Hankel chunks
    //    each and the others share the rest.
    const int chunks_a = kTile * (KK / 8);
    const int chunks_b = kV * (KK / 8);        // <= kThreads
    const int n_free = kThreads - chunks_b;
    const int qa = n_free > 0 ? min((chunks_a + 6 * chunks_b + kThreads - 1) / kThreads,
                                    chunks_a / n_free) : 0;
    const int front = qa * n_free;             // chunks [0, front): the free threads
    const bool free_t = (int)threadIdx.x >= chunks_b;
    const int c0 = free_t ? (int)threadIdx.x - chunks_b : front + (int)threadIdx.x;
    const int c_end = free_t ? front : chunks_a;
    const int c_step = free_t ? n_free : chunks_b;
    for (int c = c0; c < c_end; c += c_step) {
      const int r = c % kTile, k8 = c / kTile;  // a warp: consecutive rows, one column chunk
      const int atom = k8 >> 2, kc = k8 & 3;
      if (!DC_IN_BOUNDS(atom * 4 * kAPlane + 3 * kAPlane + sw64_offset(r, kc) + 16 <= kA &&
                            r + 8 * k8 + 8 <= kWin, a.err))
        continue;
      float re[8], im[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 v = win[r + 8 * k8 + i];
        re[i] = v.x * scale;
        im[i] = v.y * scale;
      }
      uint4 hi, lo;
      const int off = sw64_offset(r, kc);
      uint8_t* at = A + atom * 4 * kAPlane;
      split8_f16(re, hi, lo);
      *reinterpret_cast<uint4*>(at + off) = hi;
      *reinterpret_cast<uint4*>(at + kAPlane + off) = lo;
      split8_f16(im, hi, lo);
      *reinterpret_cast<uint4*>(at + 2 * kAPlane + off) = hi;
      *reinterpret_cast<uint4*>(at + 3 * kAPlane + off) = lo;
    }

    // 4. B: tap weights h, h', h'' of each range rate at the tile centre;
    //    row d * 32 + v, column k (tap j = u0 + k - m_v); one chunk per
    //    thread below chunks_b
    for (int c = threadIdx.x; c < chunks_b; c += kThreads) {
      const int v = c % kV, k8 = c / kV;
      const int atom = k8 >> 2, kc = k8 & 3;
      float w[3][8];
      const int jb = u0 + 8 * k8 - s_m[v];
      const float e = s_e[v];
      const float sn = s_sin[v], cs = s_cos[v];
      const bool live = s_vidx[v] >= 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int j = jb + i;
        float h0 = 0.f, h1 = 0.f, h2 = 0.f;
        if (live && j >= -15 && j <= 16) {
          const float sg = (j & 1) ? -1.f : 1.f;
          float s0, s1, s2, w0, w1, w2;
          sinc_d012(e - (float)j, sg * sn, sg * cs, s0, s1, s2);
          window_d012(s_wp, j + 15, e, w0, w1, w2);
          h0 = s0 * w0;
          h1 = fmaf(s1, w0, s0 * w1);
          h2 = fmaf(s2, w0, fmaf(2.f * s1, w1, s0 * w2));
        }
        w[0][i] = h0;
        w[1][i] = h1;
        w[2][i] = h2;
      }
      uint8_t* bt = B + atom * 2 * kBPlane;
      if (!DC_IN_BOUNDS(atom * 2 * kBPlane + kBPlane + sw64_offset(2 * kV + v, kc) + 16 <= kB, a.err))
        continue;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        uint4 hi, lo;
        split8_f16(w[d], hi, lo);
        const int off = sw64_offset(d * kV + v, kc);
        *reinterpret_cast<uint4*>(bt + off) = hi;
        *reinterpret_cast<uint4*>(bt + kBPlane + off) = lo;
      }
    }
    async_proxy_fence();                       // generic-proxy writes -> the MMA's async proxy
  }
  __syncthreads();

  // 5. one thread issues the split-precision products for re and im
  if (run && threadIdx.x == 0) {
    tc_fence_after();
    constexpr uint32_t idesc = f16_instr_desc(false, kTile, kN);
    const uint32_t a0 = smem_addr(A), b0 = smem_addr(B);
    for (int kk = 0; kk < KK / 16; ++kk) {
      const int atom = kk >> 1;
      const uint32_t off = (kk & 1) * 32;
      const uint32_t acc = kk > 0 ? 1u : 0u;
      const uint32_t at = a0 + atom * 4 * kAPlane + off, bt = b0 + atom * 2 * kBPlane + off;
      const uint64_t bh = sw64_desc(bt), bl = sw64_desc(bt + kBPlane);
      for (int p = 0; p < 2; ++p) {            // p = 0: real parts, 1: imaginary parts
        const uint32_t d = tmem + p * kN;
        const uint64_t ah = sw64_desc(at + 2 * p * kAPlane), al = sw64_desc(at + (2 * p + 1) * kAPlane);
        mma_f16(d, ah, bh, idesc, acc);
        mma_f16(d, ah, bl, idesc, 1u);
        mma_f16(d, al, bh, idesc, 1u);
      }
    }
    mma_commit(&mma_bar);
  }

  // 6. epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its 32 outputs) for
  //    range rates 16 (w / 4) .. + 15, eight at a time
  if (run) {
    const bool ready = mbar_wait_bounded(&mma_bar, 0, a.err);
    tc_fence_after();
    const int q = warp & 3, half = warp >> 2;
    const int r = 32 * q + lane;
    const int n = n0 + r;
    const float dn = (float)r - 0.5f * (kTile - 1);        // n - n_c
    const float unscale = ldexpf(1.f, ex);
    if (ready) {
      for (int g = 0; g < 2; ++g) {
        const int vb = 16 * half + 8 * g;
        uint32_t z[6][8];
        const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + vb;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int d = 0; d < 3; ++d) tmem_ld8_nowait(base + p * kN + d * kV, z[3 * p + d]);
        tmem_wait_ld();
        if (n < a.n_out) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int vidx = s_vidx[vb + i];
            if (vidx < 0) continue;
            const float tau = s_dl[vb + i] * dn;
            const float re = fmaf(tau, fmaf(0.5f * tau, __uint_as_float(z[2][i]), __uint_as_float(z[1][i])),
                                  __uint_as_float(z[0][i]));
            const float im = fmaf(tau, fmaf(0.5f * tau, __uint_as_float(z[5][i]), __uint_as_float(z[4][i])),
                                  __uint_as_float(z[3][i]));
            __stcs(a.y + (size_t)vidx * a.n_out + n, make_float2(re * unscale, im * unscale));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace

int rs_tc_max_span() { return kKMax - 32; }

cudaError_t launch_resample_tc(const RsTcArgs& a, cudaStream_t s) {
  if (a.n_out <= 0 || a.n_slots <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(rs_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.n_out + kTile - 1) / kTile, (a.n_slots + kV - 1) / kV);
  rs_tc_kernel<<<grid, kThreads, kSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dc
