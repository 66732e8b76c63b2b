// Predistorted LFM transmit waveforms on the device (Sec. II-A, II-C,
// Appendix B); see predist.cu.
#pragma once

#include <algorithm>

#include "../../include/dc.h"
#include "common.cuh"

namespace dc {

// Per-waveform constants (FP64, from the host).
struct PredistParams {
  int kind;                 // dc_lfm_kind
  double fs, f0, f_mix;
  double half_rate;         // B / (2T): the plain LFM's t^2 coefficient (cycles)
  double P0, slope, Q;      // Eq. 4: P = P0 + slope t, Q
  double f2, t2, c1, gamma; // pseudo-Chebyshev: f = f2 + c1 (t - t2) + gamma (t - t2)^2
};

PredistParams predist_params(int kind, double fs, double f0, double B, double T, double K2,
                             double c_light, double f_mix);
// Scratch the cubic kind needs for n samples (FP64 frequencies, block totals).
size_t predist_scratch_bytes(long long n);
cudaError_t launch_predist(const PredistParams& p, float2* y, long long n, void* scratch,
                           cudaStream_t s);

}  // namespace dc
