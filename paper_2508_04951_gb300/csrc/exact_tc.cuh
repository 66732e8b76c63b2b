// Exact-sinc resampling on tcgen05 tensor cores with hi/lo split operands
// (see exact_tc.cu).
#pragma once

#include "common.cuh"

namespace dc {

struct ExTcArgs {
  int n_in, n_out, n_pulses;
  int rows_per_alpha;      // rows of the split planes between alpha groups (0: shared pulses)
  float2* y;               // [n_alpha][n_pulses][n_out]
  const float* dl;         // per alpha: (alpha - 1) as hi, lo floats
  int* err;                // device error flag (bounded waits)
};

// Bytes of one 16-bit split plane for `rows` real rows of n samples.
size_t exact_tc_plane_bytes(long long rows, int n);

// Split x (x_rows_c complex pulses of n samples) into hi / lo planes (two
// buffers of exact_tc_plane_bytes(2 x_rows_c, n)), then run the contraction.
cudaError_t launch_exact_tc(bool fp16, const float2* x, long long x_rows_c, int n, void* hi, void* lo,
                            const ExTcArgs& args, int n_alpha, cudaStream_t s);

}  // namespace dc
