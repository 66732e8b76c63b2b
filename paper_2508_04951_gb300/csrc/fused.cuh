// Cluster-fused FFT correction for 4096 <= L <= 65536 (Sec. II-B, Eq. 16).
//
// L = L1 x 4096 with L1 = L / 4096 <= 16 rows of 4096 points.  One thread
// block cluster owns one transform: each CTA holds one row in shared memory,
// 256 threads per row run the three radix-16 Stockham stages of a row with
// the data in registers, and the column DFTs of length L1 exchange data
// with the other CTAs through distributed shared memory.  The
// four-step intermediate never leaves the SMs, so a transform reads its input
// once and writes its output once.
//
//   FUSED_APPLY : rows of a stored spectrum (bin k1 + L1 k2 at k1*4096 + k2)
//                 times a phase table in the same layout (already scaled by
//                 1/L) -> inverse rows -> written into the column owners'
//                 shared memory (plain remote stores, delivered by a
//                 cluster barrier) -> W_L^(-n2 k1) -> inverse columns -> out;
//                 at L >= 32768 optionally two rows per CTA; or, without
//                 clusters, rows and columns as tasks of one persistent grid
//                 meeting in an L2-resident scratch
//   FUSED_FULL  : y (zero-padded) -> forward columns written to the row
//                 owners (remote stores) -> forward rows -> exp(-i phi_k) / L
//                 -> inverse rows written to the column owners -> inverse
//                 columns -> out (truncated to n_out); one padded row
//                 buffer per CTA
//   FUSED_SPEC  : y -> forward columns written to the row owners (remote
//                 stores) -> forward rows -> spectrum rows
#pragma once

#include "fft.cuh"

namespace dc {

enum FusedOp : int { FUSED_APPLY = 0, FUSED_FULL = 1, FUSED_SPEC = 2 };

struct FusedArgs {
  const FftItem* items;   // one per transform (cluster)
  int n_items;
  int log2L;              // 12..16
  const float2* tw;
  int* err;               // device error flag (bounded waits)
  // Four-step twiddles W_L^(-q n2) = exp(+2 pi i q n2 / L) (L1 > 1)
  // for q = 2^b < L1, n2 < 4096, at t4 + kT4Offset(L1) + b * 4096 + n2
  // (the other q are products of these rows).
  const float2* t4;
  // FUSED_APPLY at L >= 32768: two rows per CTA (512 threads, clusters of
  // L1 / 2 CTAs) instead of one.
  int apply_rows2;
  // FUSED_APPLY at L >= 8192 in two passes through L2 instead of clusters:
  // scratch for kApplyL2Slots * chunk transforms (L float2 each), counters
  // (1 + 2 * n_items ints, zero at launch), transforms per chunk.
  float2* scratch;
  int* ctr;
  int chunk;
  // FUSED_APPLY over a grid of transforms (the bank): with grid_src set,
  // transform p = i * grid_n_tec + t reads the spectrum grid_src + i L and
  // the factors grid_ptab + t L and writes grid_n_out samples to
  // grid_dst + p grid_n_out; `items` is not read.
  const float2* grid_src;
  const float2* grid_ptab;
  float2* grid_dst;
  int grid_n_tec;
  int grid_n_out;
  // FUSED_FULL: launched with programmatic serialization (set only when no
  // item has a factor table, so that everything the kernel reads from the
  // kernel before it -- the resampled input -- is read after pdl_wait).
  int pdl;
};

// Four-step twiddle rows for L1 = 2, 4, 8, 16: log2(L1) rows of 4096 per L1.
__host__ __device__ constexpr int kT4Log2(int l1) { return l1 >= 16 ? 4 : l1 >= 8 ? 3 : l1 >= 4 ? 2 : 1; }
__host__ __device__ constexpr int kT4Offset(int l1) {
  return kT4Log2(l1) * (kT4Log2(l1) - 1) / 2 * 4096;
}
constexpr int kT4Size = 10 * 4096;

// Scratch slots of the two-pass apply, in chunks (the queue's lag between a
// chunk's rows and its columns, plus two).
constexpr int kApplyL2Slots = 4;

// Launch; returns cudaErrorInvalidValue for L outside [4096, 65536].
cudaError_t launch_fused(int op, const FusedArgs& a, cudaStream_t s);

// Middle (row) pass of the three-pass path for 2^17 <= L <= 2^20: forward
// row, phase, inverse row, four-step twiddle, in place (RowArgs as for
// ROW_MID, rows of 4096).
cudaError_t launch_row_mid_4096(const RowArgs& a, cudaStream_t s);

}  // namespace dc
