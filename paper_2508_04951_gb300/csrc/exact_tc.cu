// Exact-sinc resampling as a tensor-core contraction (Eq. 17, Table I row 1):
//
//   Y_a[p][n] = sum_m X[p][m] S_a[n][m],   S_a[n][m] = sinc(a n - m),
//
// for many pulses p sharing one range rate a.  Treating the re/im parts of the
// pulses as 2P real columns this is the GEMM  C[n][c] = sum_m S[n][m] X^T[m][c].
// It runs on the 5th-generation tensor cores (tcgen05.mma, kind::f16) with
// split operands: every FP32 value v is written as hi + lo with hi = rn(v) in
// bf16 (or fp16) and lo = rn(v - hi); the product keeps the three significant
// terms  S_hi X_hi + S_hi X_lo + S_lo X_hi  (dropping S_lo X_lo, ~2^-16 of the
// result for bf16) with FP32 accumulation in tensor memory.  For fp16 the lo
// parts are scaled by 2^11 (they would underflow fp16's range) and summed in a
// second accumulator, C = acc1 + 2^-11 acc2.
//
// One CTA computes a 256 x 256 tile of C for bf16 (two 128-row MMA halves
// sharing each X tile, halving the X traffic per flop) or 128 x 256 for fp16:
//   warp 0     TMA: X_hi / X_lo tiles (256 columns x 32 samples, 64B swizzle)
//   warp 1     TMEM allocation (512 columns); one thread issues the MMAs
//   warps 2-17 generate the S tile (rows x 32) in the same swizzled K-major
//              layout, hi and lo, from the Cauchy form
//              S[n][m] = (-1)^(m + m_n) sin(pi e_n) / (pi ((m_n - m) + e_n)),
//              a n = m_n + e_n -- one division per element, no table
//   epilogue   TMEM -> registers (tcgen05.ld) -> complex64 outputs
// Three (bf16) or four (fp16) pipeline stages of 64 / 48 KiB, mbarriers
// between the producers and the MMA thread, every wait bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "exact_tc.cuh"
#include "tc.cuh"

namespace dc {

namespace {

constexpr int BN = 256, BK = 32;                     // N columns, K per stage
constexpr int kHalfRows = 128;                       // rows per MMA (M = 128)
constexpr int kAPlane = kHalfRows * BK * 2;          // 8 KiB: one 128-row A plane
constexpr int kBPlane = BN * BK * 2;                 // 16 KiB: one B plane
constexpr int kProducerWarps = 16;                   // S-tile producers (4 per scheduler)
constexpr int kThreads = 64 + 32 * kProducerWarps;

// bf16x3: two 128-row halves share every X tile (one accumulator each);
// fp16x3: one half with two accumulators (hi*hi and the 2^11-scaled cross
// terms).  Either way the 512 TMEM columns hold exactly the accumulators.
template <bool FP16> struct Cfg {
  static constexpr int MH = FP16 ? 1 : 2;            // 128-row halves per CTA
  static constexpr int BM = MH * kHalfRows;
  static constexpr int STAGES = FP16 ? 4 : 3;
  static constexpr int A_BYTES = 2 * MH * kAPlane;   // hi + lo planes of all halves
  static constexpr int STAGE = A_BYTES + 2 * kBPlane;
  static constexpr int SMEM = STAGES * STAGE + 1024; // + alignment slack
};
constexpr float kInvPi = 0.318309886183790672f;

// Instruction descriptor of this kernel's MMAs: N = 256, M = 128.
template <bool FP16> __host__ __device__ constexpr uint32_t instr_desc() {
  return f16_instr_desc(!FP16, kHalfRows, BN);
}

// Split 8 floats into 8 hi and 8 lo 16-bit values (one 16-byte chunk each).
template <bool FP16> DC_DEV void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if constexpr (FP16) {
      const __half2 a = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
      const __half2 b = __floats2half2_rn((v[2 * i] - __low2float(a)) * 2048.f,
                                          (v[2 * i + 1] - __high2float(a)) * 2048.f);
      h[i] = *reinterpret_cast<const uint32_t*>(&a);
      l[i] = *reinterpret_cast<const uint32_t*>(&b);
    } else {
      const __nv_bfloat162 a = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i] - __low2float(a),
                                                     v[2 * i + 1] - __high2float(a));
      h[i] = *reinterpret_cast<const uint32_t*>(&a);
      l[i] = *reinterpret_cast<const uint32_t*>(&b);
    }
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// a n = m_n + e_n with a - 1 a double-float (same arithmetic as the FP32 path).
DC_DEV void position(float dl_hi, float dl_lo, int n, int& m, float& e) {
  const float fi = (float)n;
  df p = two_prod(dl_hi, fi);
  const float lo = fmaf(dl_lo, fi, p.lo);
  float f = floorf(p.hi);
  float r = __fadd_rn(__fsub_rn(p.hi, f), lo);
  if (r < 0.f) {
    r = __fadd_rn(r, 1.f);
    f -= 1.f;
    if (r >= 1.f) { r = 0.f; f += 1.f; }
  } else if (r >= 1.f) {
    r = __fsub_rn(r, 1.f);
    f += 1.f;
  }
  m = n + (int)f;
  e = r;
}

template <bool FP16>
__global__ void __launch_bounds__(kThreads, 1)
    exact_tc_kernel(const __grid_constant__ CUtensorMap map_hi,
                    const __grid_constant__ CUtensorMap map_lo, ExTcArgs a) {
  using C = Cfg<FP16>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) unsigned long long full_bar[C::STAGES], empty_bar[C::STAGES], acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ float s_sig[C::BM], s_e[C::BM];
  __shared__ int s_m[C::BM];

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * C::BM;
  const int c0 = blockIdx.y * BN;
  const int alpha = blockIdx.z;
  const int nk = (a.n_in + BK - 1) / BK;
  constexpr uint32_t kCols = 512;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full_bar[s], 1 + kProducerWarps);   // TMA arrival + one per producer warp
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (warp >= 2 && threadIdx.x - 64 < C::BM) {
    const int nl = threadIdx.x - 64;
    int m;
    float e;
    position(a.dl[2 * alpha], a.dl[2 * alpha + 1], n0 + nl, m, e);
    const float s = sinpif(e) * kInvPi;
    s_m[nl] = m;
    s_e[nl] = e;
    s_sig[nl] = (m & 1) ? -s : s;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  bool ok = true;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      const int row0 = alpha * a.rows_per_alpha + c0;
      for (int kc = 0; kc < nk && ok; ++kc) {
        const int s = kc % C::STAGES;
        const uint32_t ph = (kc / C::STAGES) & 1;
        if (!mbar_wait_bounded(&empty_bar[s], ph ^ 1, a.err)) { ok = false; break; }
        uint8_t* st = smem + s * C::STAGE;
        mbar_expect_tx(&full_bar[s], 2 * kBPlane);
        tma_load_2d(st + C::A_BYTES, &map_hi, kc * BK, row0, &full_bar[s]);
        tma_load_2d(st + C::A_BYTES + kBPlane, &map_lo, kc * BK, row0, &full_bar[s]);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc<FP16>();
      for (int kc = 0; kc < nk && ok; ++kc) {
        const int s = kc % C::STAGES;
        const uint32_t ph = (kc / C::STAGES) & 1;
        if (!mbar_wait_bounded(&full_bar[s], ph, a.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t st = smem_addr(smem + s * C::STAGE);
        const uint32_t b_hi = st + C::A_BYTES, b_lo = b_hi + kBPlane;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t off = kk * 32;     // 16 elements of K = 32 bytes inside the swizzle atom
          const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
#pragma unroll
          for (int h = 0; h < C::MH; ++h) {
            const uint32_t a_hi = st + h * kAPlane, a_lo = st + (C::MH + h) * kAPlane;
            const uint32_t d = tmem + h * 256;
            if constexpr (FP16) {
              mma_f16(d, sw64_desc(a_hi + off), sw64_desc(b_hi + off), idesc, acc);
              mma_f16(d + 256, sw64_desc(a_hi + off), sw64_desc(b_lo + off), idesc, acc);
              mma_f16(d + 256, sw64_desc(a_lo + off), sw64_desc(b_hi + off), idesc, 1u);
            } else {
              mma_f16(d, sw64_desc(a_hi + off), sw64_desc(b_hi + off), idesc, acc);
              mma_f16(d, sw64_desc(a_hi + off), sw64_desc(b_lo + off), idesc, 1u);
              mma_f16(d, sw64_desc(a_lo + off), sw64_desc(b_hi + off), idesc, 1u);
            }
          }
        }
        mma_commit(&empty_bar[s]);
      }
      mma_commit(&acc_bar);
    }
  } else {
    // ------------------------------------------------- S tile producers
    // thread -> one of the BM rows and CHUNKS of its 4 chunks of 8 (bf16:
    // 256 rows, 2 chunks; fp16: 128 rows, 1 chunk)
    constexpr int NP = 32 * kProducerWarps;
    constexpr int CHUNKS = 4 * C::BM / NP;
    static_assert(CHUNKS >= 1 && 4 * C::BM == CHUNKS * NP, "producers cover the tile");
    const int p = threadIdx.x - 64;            // 0..NP-1
    const int nl = p % C::BM;
    const int cbase = (p / C::BM) * CHUNKS;
    const int h = nl >> 7, r = nl & 127;       // half and row inside it
    const int mn = s_m[nl];
    const float en = s_e[nl], sg = s_sig[nl];
    for (int kc = 0; kc < nk && ok; ++kc) {
      const int s = kc % C::STAGES;
      const uint32_t ph = (kc / C::STAGES) & 1;
      if (!mbar_wait_bounded(&empty_bar[s], ph ^ 1, a.err)) { ok = false; break; }
      uint8_t* st = smem + s * C::STAGE;
#pragma unroll
      for (int q = 0; q < CHUNKS; ++q) {
        const int k8 = cbase + q;              // 16-byte chunk of the 64-byte row
        float v[8];
        const int m0 = kc * BK + k8 * 8;
        // (m_n - m) + e_n with the integer part formed exactly first
        // ((m_n - m0) - i, integers below 2^22) and e_n added last, so the
        // denominator near m = m_n is e_n itself even when e_n is far below
        // the rounding unit of m_n - m0
        const float di0 = exact_i2f(mn - m0);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int m = m0 + i;
          float val = 0.f;
          if (m < a.n_in) {
            if (en == 0.f) val = (m == mn) ? 1.f : 0.f;
            else val = __fdividef((i & 1) ? -sg : sg, (di0 - (float)i) + en);
          }
          v[i] = val;
        }
        // (-1)^m: m = kc*32 + k8*8 + i has the parity of i
        uint4 hi, lo;
        split8<FP16>(v, hi, lo);
        const int off = r * 64 + ((k8 ^ ((r >> 1) & 3)) << 4);
        if (DC_IN_BOUNDS((C::MH + h) * kAPlane + off + 16 <= C::A_BYTES && off + 16 <= kAPlane, a.err)) {
          *reinterpret_cast<uint4*>(st + h * kAPlane + off) = hi;
          *reinterpret_cast<uint4*>(st + (C::MH + h) * kAPlane + off) = lo;
        }
      }
      async_proxy_fence();                     // our generic-proxy writes -> async proxy
      __syncwarp();
      if (lane == 0) bar_arrive(&full_bar[s]);
    }
    // ----------------------------------------------------------- epilogue
    if (warp < 2 + 4 * C::MH) {
      const int q = warp & 3;                   // TMEM lanes 32q .. 32q+31
      const int hh = (warp - 2) >> 2;           // accumulator half
      const bool ready = mbar_wait_bounded(&acc_bar, 0, a.err);
      tc_fence_after();
      const int n = n0 + hh * kHalfRows + 32 * q + lane;
      if (ready) {
        for (int cc = 0; cc < BN / 16; ++cc) {
          float f[16];
          const uint32_t taddr = tmem + hh * 256 + ((uint32_t)(32 * q) << 16) + cc * 16;
          tmem_ld16(taddr, f);
          if constexpr (FP16) {
            float g[16];
            tmem_ld16(taddr + 256, g);
#pragma unroll
            for (int i = 0; i < 16; ++i) f[i] = fmaf(g[i], 1.0f / 2048.f, f[i]);
          }
          if (n < a.n_out) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int pulse = (c0 + cc * 16) / 2 + i;
              if (pulse < a.n_pulses)
                a.y[((size_t)alpha * a.n_pulses + pulse) * a.n_out + n] = make_float2(f[2 * i], f[2 * i + 1]);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
  }
}

// X (complex64, pulses of n samples) -> hi / lo 16-bit planes, row 2p = re,
// row 2p + 1 = im, samples contiguous with row stride `ld` (lo scaled by 2^11
// for fp16).
template <bool FP16>
__global__ void split_planes_kernel(const float2* __restrict__ x, int n, long long rows_c, int ld,
                                    uint16_t* hi, uint16_t* lo) {
  const long long total = rows_c * n;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long pr = g / n;
    const int m = (int)(g - pr * n);
    const float2 v = x[g];
    const float vv[2] = {v.x, v.y};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      uint16_t h, l;
      if constexpr (FP16) {
        const __half a = __float2half_rn(vv[c]);
        const __half b = __float2half_rn((vv[c] - __half2float(a)) * 2048.f);
        h = __half_as_ushort(a);
        l = __half_as_ushort(b);
      } else {
        const __nv_bfloat16 a = __float2bfloat16_rn(vv[c]);
        const __nv_bfloat16 b = __float2bfloat16_rn(vv[c] - __bfloat162float(a));
        h = __bfloat16_as_ushort(a);
        l = __bfloat16_as_ushort(b);
      }
      const long long o = (2 * pr + c) * (long long)ld + m;
      hi[o] = h;
      lo[o] = l;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, void* base, bool fp16, long long rows, int n, int ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {BK, BN};      // 32 x 16-bit = 64 bytes inner: 64-byte swizzle
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base,
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

size_t exact_tc_plane_bytes(long long rows, int n) {
  const long long ld = (n + 7) / 8 * 8;
  return (size_t)rows * ld * 2;
}

cudaError_t launch_exact_tc(bool fp16, const float2* x, long long x_rows_c, int n, void* hi, void* lo,
                            const ExTcArgs& args, int n_alpha, cudaStream_t s) {
  const int ld = (n + 7) / 8 * 8;
  const long long total = x_rows_c * n;
  const int grid_c = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
  if (fp16)
    split_planes_kernel<true><<<grid_c, 256, 0, s>>>(x, n, x_rows_c, ld, (uint16_t*)hi, (uint16_t*)lo);
  else
    split_planes_kernel<false><<<grid_c, 256, 0, s>>>(x, n, x_rows_c, ld, (uint16_t*)hi, (uint16_t*)lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap mh, ml;
  if (!make_map(&mh, hi, fp16, 2 * x_rows_c, n, ld) || !make_map(&ml, lo, fp16, 2 * x_rows_c, n, ld))
    return cudaErrorInvalidValue;
  if (fp16) {
    using Cf = Cfg<true>;
    dim3 grid((args.n_out + Cf::BM - 1) / Cf::BM, (2 * args.n_pulses + BN - 1) / BN, n_alpha);
    auto k = exact_tc_kernel<true>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::SMEM))) return e;
    k<<<grid, kThreads, Cf::SMEM, s>>>(mh, ml, args);
  } else {
    using Cb = Cfg<false>;
    dim3 grid((args.n_out + Cb::BM - 1) / Cb::BM, (2 * args.n_pulses + BN - 1) / BN, n_alpha);
    auto k = exact_tc_kernel<false>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Cb::SMEM))) return e;
    k<<<grid, kThreads, Cb::SMEM, s>>>(mh, ml, args);
  }
  return cudaGetLastError();
}

}  // namespace dc
