// Stockham autosort FFT passes and the ionospheric correction built on them
// (Sec. II-B, Eqs. 15-16: forward DFT, multiply by exp(-i phi_k), inverse DFT).
//
// Transform lengths L = 2^m up to 2^20.  L <= 4096 runs as one "row" pass in
// shared memory.  Larger L uses the four-step split L = L1 x L2 with
// L2 = 4096, n = n2 + L2 n1, k = k1 + L1 k2:
//   F1  (column pass): DFT over n1 of x[n2 + L2 n1], times W_L^(n2 k1),
//                      stored at T[n2 + L2 k1]
//   F2  (row pass)   : DFT over n2 of row k1 of T  -> bin k1 + L1 k2 sits at
//                      T[k1 L2 + k2] (transposed spectrum, never reordered)
//   phase multiply on that layout, then the inverse in mirror order:
//   A   (row pass)   : inverse DFT over k2, times W_L^(-n2 k1), back to T
//   B   (column pass): inverse DFT over k1, times 1/L, out[n2 + L2 n1]
// F2, the phase multiply and A run in one row kernel, so a corrected pulse
// costs three passes over the data.
#pragma once

#include "common.cuh"
#include "phase.cuh"

namespace dc {

// One transform of a launch.  All items of one launch share L.
struct FftItem {
  const float2* src;     // input of this pass
  float2* dst;           // output of this pass
  const float2* ptab;    // per-bin factors (length L): exp(-i phi_k), times a
                         // matched filter's conjugate replica spectrum when
                         // compressing, in the spectrum's layout (bin
                         // k1 + L1 k2 at k1*4096 + k2 for L > 4096, natural
                         // order below); null -> exp(-i phi_k) computed from
                         // `ph`
  PhaseParams ph;
  int n_valid;           // samples of src that are data (zero beyond), first pass
  int n_out;             // samples stored by the last pass (truncation)
};

enum RowOp : int {
  ROW_FULL = 0,   // L <= 4096: load (zero-pad), fwd, phase, inv, 1/L, store n < n_out
  ROW_MID = 1,    // four-step middle: fwd, phase, inv, W_L^(-n2 k1); in place on T
  ROW_SPEC = 2,   // forward only: L <= 4096 from y (zero-pad), else row of T (F2)
  ROW_APPLY = 3,  // phase + inverse: L <= 4096 -> 1/L, store n < n_out; else twiddle, store T
};
enum ColOp : int {
  COL_F1 = 0,     // forward first pass, from y (zero-pad) to T
  COL_B = 1,      // inverse last pass, from T to out (1/L, n < n_out)
};

struct RowArgs {
  const FftItem* items;
  int n_items;
  int log2L;       // transform length
  int log2L1;      // rows per transform (0 for L <= 4096)
  const float2* tw;
};
struct ColArgs {
  const FftItem* items;
  int n_items;
  int log2L;
  int log2L1;      // column length M = L1
  const float2* tw;
};

// Launchers (fft.cu).  Return cudaSuccess or the launch error.
cudaError_t launch_row(int op, const RowArgs& a, cudaStream_t s);
cudaError_t launch_col(int op, const ColArgs& a, cudaStream_t s);

}  // namespace dc
