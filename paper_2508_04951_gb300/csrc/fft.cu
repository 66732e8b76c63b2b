// Stockham FFT passes with the fused ionospheric phase multiply.
// Index conventions and the four-step split are described in fft.cuh.
#include "fft.cuh"

namespace dc {

constexpr int kThreads = 256;

// Radix of stage s of an M-point transform: radix-16 stages, then one stage
// of the remaining power of two.
template <int M> __host__ __device__ constexpr int n_stages() {
  int m = 0;
  while ((1 << m) < M) ++m;
  return m / 4 + (m % 4 ? 1 : 0);
}
template <int M> __host__ __device__ constexpr int stage_radix(int s) {
  int m = 0;
  while ((1 << m) < M) ++m;
  return s < m / 4 ? 16 : (1 << (m % 4));
}
template <int M> __host__ __device__ constexpr int stage_ns(int s) {
  int ns = 1;
  for (int i = 0; i < s; ++i) ns *= stage_radix<M>(i);
  return ns;
}

// ----------------------------------------------------------- row layout
// Line c of the CTA at c*LP, element p at p + p/16 (breaks the stride-16
// write pattern of the first stage across banks).
DC_DEV int rpad(int p) { return p + (p >> 4); }

template <int M> struct RowShape {
  static constexpr int LINES = M >= 4096 ? 1 : (M >= 16 ? 4096 / M : 256);
  static constexpr int LP = M + (M >> 4) + (M < 16 ? 0 : 0);
  static constexpr int SMEM = LINES * (M + (M >> 4) + 1);   // +1 keeps LP odd-ish for tiny M
};

// One in-place Stockham stage over all lines of the CTA (row layout).
template <int M, int R, int NS, int DIR, int LINES, int LP>
DC_DEV void row_stage(float2* sm, const float2* __restrict__ tw) {
  constexpr int NB = M / R;
  constexpr int TOTAL = NB * LINES;
  constexpr int PER = (TOTAL + kThreads - 1) / kThreads;
  float2 v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + kThreads * q;
    if (TOTAL % kThreads == 0 || b < TOTAL) {
      const int line = b / NB, j = b % NB;
      const float2* s = sm + line * LP;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = s[rpad(j + r * NB)];
      if constexpr (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r)
          v[q][r] = cmul(v[q][r], tw_m<DIR>(tw, (r * k) * (4096 / (NS * R))));
      }
      dft<R, DIR>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + kThreads * q;
    if (TOTAL % kThreads == 0 || b < TOTAL) {
      const int line = b / NB, j = b % NB;
      const int k = j % NS;
      float2* s = sm + line * LP;
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[rpad(base + r * NS)] = v[q][r];
    }
  }
  __syncthreads();
}

template <int M, int DIR, int LINES, int LP, int S = 0>
DC_DEV void row_fft(float2* sm, const float2* __restrict__ tw) {
  if constexpr (S < n_stages<M>()) {
    row_stage<M, stage_radix<M>(S), stage_ns<M>(S), DIR, LINES, LP>(sm, tw);
    row_fft<M, DIR, LINES, LP, S + 1>(sm, tw);
  }
}

// Row pass.  Line g of the launch is row (g mod L1) of item (g / L1).
template <int M, int OP>
__global__ void __launch_bounds__(kThreads) row_kernel(RowArgs a) {
  constexpr int LINES = RowShape<M>::LINES;
  constexpr int LP = M + (M >> 4) + 1;
  extern __shared__ float2 sm[];
  const int L1 = 1 << a.log2L1;
  const int total = a.n_items * L1;
  const int line0 = blockIdx.x * LINES;
  const float invL = 1.0f / (float)(1 << a.log2L);

  // ---- load (coalesced along each line)
  for (int idx = threadIdx.x; idx < LINES * M; idx += kThreads) {
    const int c = idx / M, p = idx % M;
    const int g = line0 + c;
    float2 v = make_float2(0.f, 0.f);
    if (g < total) {
      const int it = g >> a.log2L1, row = g & (L1 - 1);
      const FftItem& I = a.items[it];
      if (a.log2L1 == 0) {
        if (OP == ROW_FULL || OP == ROW_SPEC) {
          if (p < I.n_valid) v = I.src[p];
        } else {
          v = I.src[p];
        }
      } else {
        v = I.src[(size_t)row * M + p];
      }
      if (OP == ROW_APPLY) {
        const int k = row + L1 * p;
        // the table is in the spectrum's own layout: bin k at row * M + p
        if (I.ptab) v = cmul(v, __ldg(I.ptab + (size_t)row * M + p));
        else if (I.ph.enabled) v = cmul(v, iono_factor(I.ph, k));
      }
    }
    sm[c * LP + rpad(p)] = v;
  }
  __syncthreads();

  if (OP == ROW_FULL || OP == ROW_MID || OP == ROW_SPEC) row_fft<M, -1, LINES, LP>(sm, a.tw);

  if (OP == ROW_FULL || OP == ROW_MID) {
    for (int idx = threadIdx.x; idx < LINES * M; idx += kThreads) {
      const int c = idx / M, p = idx % M;
      const int g = line0 + c;
      if (g < total) {
        const int it = g >> a.log2L1, row = g & (L1 - 1);
        const FftItem& I = a.items[it];
        const int k = row + L1 * p;
        float2 w;
        if (I.ptab) w = __ldg(I.ptab + (size_t)row * M + p);   // the spectrum's layout
        else if (I.ph.enabled) w = iono_factor(I.ph, k);
        else continue;
        sm[c * LP + rpad(p)] = cmul(sm[c * LP + rpad(p)], w);
      }
    }
    __syncthreads();
  }

  if (OP != ROW_SPEC) row_fft<M, +1, LINES, LP>(sm, a.tw);

  // ---- store
  for (int idx = threadIdx.x; idx < LINES * M; idx += kThreads) {
    const int c = idx / M, p = idx % M;
    const int g = line0 + c;
    if (g >= total) continue;
    const int it = g >> a.log2L1, row = g & (L1 - 1);
    const FftItem& I = a.items[it];
    float2 v = sm[c * LP + rpad(p)];
    if (OP == ROW_SPEC) {
      I.dst[(size_t)row * M + p] = v;
    } else if (a.log2L1 == 0) {
      // single pass: scale and truncate
      if (p < I.n_out) __stcs(I.dst + p, cscale(v, invL));
    } else {
      // four-step middle / apply: twiddle W_L^(-n2 k1), n2 = p, k1 = row
      v = cmul(v, tw_big<+1>(a.tw, (uint32_t)(p * row) & ((1u << a.log2L) - 1), a.log2L));
      I.dst[(size_t)row * M + p] = v;
    }
  }
}

// ------------------------------------------------------------ column pass
// C = 4096 / M columns per CTA (32 KiB of shared memory for every M, and
// 256 butterflies per radix-16 stage), element p of column c at sm[p*C + c];
// consecutive threads take consecutive columns, so global rows of C complex
// are read and written whole.
template <int M> __host__ __device__ constexpr int col_width() { return 4096 / M; }

template <int M, int R, int NS, int DIR>
DC_DEV void col_stage(float2* sm, const float2* __restrict__ tw) {
  constexpr int C = col_width<M>();
  constexpr int NB = M / R;
  constexpr int TOTAL = NB * C;
  constexpr int PER = (TOTAL + kThreads - 1) / kThreads;
  float2 v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + kThreads * q;
    if (TOTAL % kThreads == 0 || b < TOTAL) {
      const int c = b % C, j = b / C;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = sm[(j + r * NB) * C + c];
      if constexpr (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r)
          v[q][r] = cmul(v[q][r], tw_m<DIR>(tw, (r * k) * (4096 / (NS * R))));
      }
      dft<R, DIR>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + kThreads * q;
    if (TOTAL % kThreads == 0 || b < TOTAL) {
      const int c = b % C, j = b / C;
      const int k = j % NS;
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[(base + r * NS) * C + c] = v[q][r];
    }
  }
  __syncthreads();
}

template <int M, int DIR, int S = 0>
DC_DEV void col_fft(float2* sm, const float2* __restrict__ tw) {
  if constexpr (S < n_stages<M>()) {
    col_stage<M, stage_radix<M>(S), stage_ns<M>(S), DIR>(sm, tw);
    col_fft<M, DIR, S + 1>(sm, tw);
  }
}

// Column pass for M = L1 in [32, 256] (shared memory).
template <int M, int OP>
__global__ void __launch_bounds__(kThreads) col_kernel_smem(ColArgs a) {
  constexpr int C = col_width<M>();
  __shared__ float2 sm[M * C];
  const int L2 = 1 << (a.log2L - a.log2L1);
  const int cta_per_item = L2 / C;
  const int it = blockIdx.x / cta_per_item;
  const int col0 = (blockIdx.x % cta_per_item) * C;
  const FftItem& I = a.items[it];
  const float invL = 1.0f / (float)(1 << a.log2L);

  // all of a thread's loads first (the global source may not be proven
  // apart from shared memory, which would serialise load/store pairs)
  constexpr int PER = M * C / kThreads;
  const int c = threadIdx.x % C, p0 = threadIdx.x / C;
  constexpr int PSTEP = kThreads / C;
  const int n2 = col0 + c;
  float2 v[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int p = p0 + PSTEP * q;
    if (OP == COL_F1) {
      const int n = n2 + L2 * p;
      v[q] = n < I.n_valid ? __ldg(I.src + n) : make_float2(0.f, 0.f);
    } else {
      v[q] = __ldg(I.src + (size_t)p * L2 + n2);
    }
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) sm[(p0 + PSTEP * q) * C + c] = v[q];
  __syncthreads();
  col_fft<M, OP == COL_F1 ? -1 : +1>(sm, a.tw);
#pragma unroll
  for (int q = 0; q < PER; ++q) v[q] = sm[(p0 + PSTEP * q) * C + c];
  if (OP == COL_F1) {
    // twiddle W_L^(n2 k1), k1 = p0 + PSTEP q: W_L^(n2 p0) times the q-th
    // power of W_L^(n2 PSTEP) (powers from the table values for 1, 2, 4, 8)
    static_assert(PER == 16, "16 rows per thread");
    const uint32_t mask = (1u << a.log2L) - 1;
    float2 b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = tw_big<-1>(a.tw, (uint32_t)(n2 * (PSTEP << i)) & mask, a.log2L);
    const float2 w0 = tw_big<-1>(a.tw, (uint32_t)(n2 * p0) & mask, a.log2L);
    apply_powers<PER>(v, b);
#pragma unroll
    for (int q = 0; q < PER; ++q) I.dst[(size_t)(p0 + PSTEP * q) * L2 + n2] = cmul(v[q], w0);
  } else {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int n = n2 + L2 * (p0 + PSTEP * q);
      if (n < I.n_out) __stcs(I.dst + n, cscale(v[q], invL));
    }
  }
}

// Column pass for M = L1 in [2, 16]: one column per thread, all in registers.
template <int M, int OP>
__global__ void __launch_bounds__(kThreads) col_kernel_reg(ColArgs a) {
  const int L2 = 1 << (a.log2L - a.log2L1);
  const int cta_per_item = L2 / kThreads;
  const int it = blockIdx.x / cta_per_item;
  const int n2 = (blockIdx.x % cta_per_item) * kThreads + threadIdx.x;
  const FftItem& I = a.items[it];
  float2 v[M];
#pragma unroll
  for (int p = 0; p < M; ++p) {
    if (OP == COL_F1) {
      const int n = n2 + L2 * p;
      v[p] = n < I.n_valid ? I.src[n] : make_float2(0.f, 0.f);
    } else {
      v[p] = I.src[(size_t)p * L2 + n2];
    }
  }
  dft<M, OP == COL_F1 ? -1 : +1>(v);
  if (OP == COL_F1) {
#pragma unroll
    for (int p = 0; p < M; ++p)
      I.dst[(size_t)p * L2 + n2] =
          cmul(v[p], tw_big<-1>(a.tw, (uint32_t)(n2 * p) & ((1u << a.log2L) - 1), a.log2L));
  } else {
    const float invL = 1.0f / (float)(1 << a.log2L);
#pragma unroll
    for (int p = 0; p < M; ++p) {
      const int n = n2 + L2 * p;
      if (n < I.n_out) __stcs(I.dst + n, cscale(v[p], invL));
    }
  }
}

// ---------------------------------------------------------------- launchers
template <int M, int OP>
static cudaError_t launch_row_m(const RowArgs& a, cudaStream_t s) {
  constexpr int LINES = RowShape<M>::LINES;
  constexpr int LP = M + (M >> 4) + 1;
  const size_t smem = sizeof(float2) * LINES * LP;
  const long long lines = (long long)a.n_items << a.log2L1;
  const long long grid = (lines + LINES - 1) / LINES;
  if (grid <= 0) return cudaSuccess;
  auto k = row_kernel<M, OP>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<(unsigned)grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_row_op(const RowArgs& a, cudaStream_t s) {
  const int m = a.log2L - a.log2L1;   // row length log2
  switch (m) {
    case 0: return launch_row_m<1, OP>(a, s);
    case 1: return launch_row_m<2, OP>(a, s);
    case 2: return launch_row_m<4, OP>(a, s);
    case 3: return launch_row_m<8, OP>(a, s);
    case 4: return launch_row_m<16, OP>(a, s);
    case 5: return launch_row_m<32, OP>(a, s);
    case 6: return launch_row_m<64, OP>(a, s);
    case 7: return launch_row_m<128, OP>(a, s);
    case 8: return launch_row_m<256, OP>(a, s);
    case 9: return launch_row_m<512, OP>(a, s);
    case 10: return launch_row_m<1024, OP>(a, s);
    case 11: return launch_row_m<2048, OP>(a, s);
    case 12: return launch_row_m<4096, OP>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_row(int op, const RowArgs& a, cudaStream_t s) {
  switch (op) {
    case ROW_FULL: return launch_row_op<ROW_FULL>(a, s);
    case ROW_MID: return launch_row_op<ROW_MID>(a, s);
    case ROW_SPEC: return launch_row_op<ROW_SPEC>(a, s);
    case ROW_APPLY: return launch_row_op<ROW_APPLY>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int M, int OP>
static cudaError_t launch_col_m(const ColArgs& a, cudaStream_t s) {
  const int L2 = 1 << (a.log2L - a.log2L1);
  if (a.n_items <= 0) return cudaSuccess;
  if constexpr (M <= 16) {
    const long long grid = (long long)a.n_items * (L2 / kThreads);
    col_kernel_reg<M, OP><<<(unsigned)grid, kThreads, 0, s>>>(a);
  } else {
    const long long grid = (long long)a.n_items * (L2 / col_width<M>());
    col_kernel_smem<M, OP><<<(unsigned)grid, kThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_col_op(const ColArgs& a, cudaStream_t s) {
  switch (a.log2L1) {
    case 1: return launch_col_m<2, OP>(a, s);
    case 2: return launch_col_m<4, OP>(a, s);
    case 3: return launch_col_m<8, OP>(a, s);
    case 4: return launch_col_m<16, OP>(a, s);
    case 5: return launch_col_m<32, OP>(a, s);
    case 6: return launch_col_m<64, OP>(a, s);
    case 7: return launch_col_m<128, OP>(a, s);
    case 8: return launch_col_m<256, OP>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col(int op, const ColArgs& a, cudaStream_t s) {
  return op == COL_F1 ? launch_col_op<COL_F1>(a, s) : launch_col_op<COL_B>(a, s);
}

}  // namespace dc
