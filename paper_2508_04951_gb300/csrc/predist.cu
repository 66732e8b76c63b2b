// Predistorted LFM transmit waveforms (Sec. II-A, Sec. II-C, Appendix B):
// the comparison methods of the paper's FFT correction, generated on the
// device.  s[m] = exp(i (phi(t_m) - 2 pi f_mix t_m)), t_m = m / fs:
//
//   DC_LFM_PLAIN          phi = 2 pi (f0 t + B t^2 / (2T))          (no ionosphere)
//   DC_LFM_CUBIC          f(t) the real root of Eq. 4 by Eqs. 11-14, phi by the
//                         trapezoidal rule over the samples (Sec. II-A)
//   DC_LFM_POLY           pseudo-Chebyshev quadratic f(t) (Eqs. 5-10), phi in
//                         closed form
//   DC_LFM_POLY_ORIGINAL  the same with the factor-4 coefficients (Appendix B)
//
// The phases reach ~10^5 rad (f0 ~ 400 MHz over 100 us), so they are carried
// in FP64 as cycles, reduced to a fraction of a cycle, and only then turned
// into the FP32 output by sincospif.  The trapezoidal phase is a prefix sum:
// one kernel evaluates f(t_m) - f0 per sample (FP64) and each 1024-sample
// block's total, a one-block kernel scans the block totals, and a third
// kernel scans within blocks and writes the samples.
#include <cmath>

#include "predist.cuh"

namespace dc {

namespace {

constexpr int kPdBlock = 1024;      // samples per block of the trapezoid scan

// Real root of Eq. 4, f^3 - P f^2 - Q = 0, by Eqs. 11-14 (chi = P^2,
// psi = -2 P^3 - 27 Q, omega = cbrt((psi + sqrt(psi^2 - 4 chi^3)) / 2),
// f = (P - omega - chi / omega) / 3).  The radicand is formed as
// 108 P^3 Q + 729 Q^2, which equals psi^2 - 4 chi^3 without its cancellation.
__device__ double cubic_root_eq4(double P, double Q) {
  const double chi = P * P;
  const double P3 = chi * P;
  const double psi = -2.0 * P3 - 27.0 * Q;
  const double rad = fmax(108.0 * P3 * Q + 729.0 * Q * Q, 0.0);
  const double omega = cbrt(0.5 * (psi + sqrt(rad)));
  return (P - omega - chi / omega) / 3.0;
}

__device__ float2 cycles_to_sample(double cyc) {
  const double r = cyc - rint(cyc);
  float s, c;
  sincospif(2.0f * (float)r, &s, &c);
  return make_float2(c, s);
}

// Closed-form phases (PLAIN, POLY, POLY_ORIGINAL).
__global__ void predist_closed_kernel(PredistParams p, float2* __restrict__ y, long long n) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n;
       m += (long long)gridDim.x * blockDim.x) {
    const double t = (double)m / p.fs;
    double cyc;
    if (p.kind == DC_LFM_PLAIN) {
      cyc = (p.f0 - p.f_mix) * t + p.half_rate * t * t;
    } else {
      // f = f2 + c1 s + gamma s^2, s = t - t2; int_0^t f = f2 t + c1 (s^2 - s0^2)/2
      // + gamma (s^3 - s0^3)/3, s0 = -t2, with s^2 - s0^2 = t (s + s0) and
      // s^3 - s0^3 = t (s^2 + s s0 + s0^2) (no cancellation)
      const double s = t - p.t2, s0 = -p.t2;
      cyc = (p.f2 - p.f_mix) * t + 0.5 * p.c1 * t * (s + s0) +
            p.gamma * t * (s * s + s * s0 + s0 * s0) * (1.0 / 3.0);
    }
    y[m] = cycles_to_sample(cyc);
  }
}

// CUBIC, pass 1: F[m] = f(t_m) - f0 and the block totals.
__global__ void __launch_bounds__(kPdBlock) predist_cubic_freq_kernel(PredistParams p, double* F,
                                                                     double* totals, long long n) {
  __shared__ double red[kPdBlock / 32];
  const long long m = blockIdx.x * (long long)kPdBlock + threadIdx.x;
  double f = 0.0;
  if (m < n) {
    const double t = (double)m / p.fs;
    f = cubic_root_eq4(p.P0 + p.slope * t, p.Q) - p.f0;
    F[m] = f;
  }
  double v = f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) totals[blockIdx.x] = v;
  }
}

// CUBIC, pass 2: exclusive prefix sums of the block totals (one CTA; each
// thread owns consecutive totals, a warp scan joins them).
__global__ void __launch_bounds__(kPdBlock) predist_scan_totals_kernel(double* totals, int nb) {
  __shared__ double warp_sum[kPdBlock / 32];
  const int per = (nb + kPdBlock - 1) / kPdBlock;
  const int b0 = threadIdx.x * per;
  double own = 0.0;
  for (int i = 0; i < per; ++i)
    if (b0 + i < nb) own += totals[b0 + i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double inc = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_sum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    double w = warp_sum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    warp_sum[lane] = w;                           // inclusive over warps
  }
  __syncthreads();
  double run = inc - own + (warp ? warp_sum[warp - 1] : 0.0);   // exclusive prefix of b0
  for (int i = 0; i < per; ++i) {
    if (b0 + i < nb) {
      const double t = totals[b0 + i];
      totals[b0 + i] = run;
      run += t;
    }
  }
}

// CUBIC, pass 3: S[m] = sum_{i <= m} F[i] (block prefix + in-block scan);
// the trapezoid over t_0 .. t_m is dt (S[m] - (F[0] + F[m]) / 2), and
// phi / 2 pi = f0 t_m + that - f_mix t_m.
__global__ void __launch_bounds__(kPdBlock) predist_cubic_out_kernel(PredistParams p, const double* F,
                                                                    const double* prefix,
                                                                    float2* __restrict__ y,
                                                                    long long n) {
  __shared__ double warp_sum[kPdBlock / 32];
  const long long m = blockIdx.x * (long long)kPdBlock + threadIdx.x;
  const double f = m < n ? F[m] : 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double inc = f;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_sum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    double w = warp_sum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    warp_sum[lane] = w;
  }
  __syncthreads();
  if (m >= n) return;
  const double S = prefix[blockIdx.x] + (warp ? warp_sum[warp - 1] : 0.0) + inc;
  const double dt = 1.0 / p.fs;
  const double t = (double)m * dt;
  const double cyc = (p.f0 - p.f_mix) * t + dt * (S - 0.5 * (F[0] + f));
  y[m] = cycles_to_sample(cyc);
}

}  // namespace

size_t predist_scratch_bytes(long long n) {
  const long long nb = (n + kPdBlock - 1) / kPdBlock;
  return (size_t)n * sizeof(double) + 256 + (size_t)nb * sizeof(double);
}

cudaError_t launch_predist(const PredistParams& p, float2* y, long long n, void* scratch,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (p.kind != DC_LFM_CUBIC) {
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 8);
    predist_closed_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, y, n);
    return cudaGetLastError();
  }
  const long long nb = (n + kPdBlock - 1) / kPdBlock;
  double* F = static_cast<double*>(scratch);
  double* totals = reinterpret_cast<double*>(static_cast<char*>(scratch) +
                                             (((size_t)n * sizeof(double) + 255) & ~(size_t)255));
  predist_cubic_freq_kernel<<<(unsigned)nb, kPdBlock, 0, s>>>(p, F, totals, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  predist_scan_totals_kernel<<<1, kPdBlock, 0, s>>>(totals, (int)nb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  predist_cubic_out_kernel<<<(unsigned)nb, kPdBlock, 0, s>>>(p, F, totals, y, n);
  return cudaGetLastError();
}

// Host: per-waveform constants in FP64.
PredistParams predist_params(int kind, double fs, double f0, double B, double T, double K2,
                             double c_light, double f_mix) {
  PredistParams p{};
  p.kind = kind;
  p.fs = fs;
  p.f0 = f0;
  p.f_mix = f_mix;
  p.half_rate = 0.5 * B / T;
  // Eq. 4 as f^3 - P f^2 - Q = 0: P = f0 + B t/T - 2 K2 B/(c f0^2 T), Q = 2 K2 B/(c T)
  p.P0 = f0 - 2.0 * K2 * B / (c_light * f0 * f0 * T);
  p.slope = B / T;
  p.Q = 2.0 * K2 * B / (c_light * T);
  if (kind == DC_LFM_POLY || kind == DC_LFM_POLY_ORIGINAL) {
    // Eqs. 6-10 (factor 2; Appendix B's original: 4).  Nodes f1, f2, f3 =
    // f0 + B (1 -+ a)/2, f0 + B/2 with a = sqrt(3)/2; T1 (Eq. 9) and T3 (its
    // mirror at the third node, used by Eqs. 7-8) are the nodes' transmit
    // times relative to that of f2, T2 = T1 + T3 (Eq. 10).  The quadratic
    // through (T1, -aB/2), (0, 0), (T3, aB/2) about node 2 gives the slope
    // c1 = mu0 + delta_mu and the curvature gamma (Eq. 8).
    const double a = std::sqrt(3.0) / 2.0;
    const double g = (kind == DC_LFM_POLY ? 2.0 : 4.0) * K2 / c_light;
    const double f1 = f0 + B * (1.0 - a) / 2.0, f2 = f0 + B / 2.0, f3 = f0 + B * (1.0 + a) / 2.0;
    const double i1 = 1.0 / (f1 * f1), i2 = 1.0 / (f2 * f2), i3 = 1.0 / (f3 * f3);
    const double T1 = -a * T / 2.0 + g * (i2 - i1);
    const double T3 = a * T / 2.0 + g * (i2 - i3);
    const double T2 = g * (2.0 * i2 - i1 - i3);
    const double den = T1 * T3 * (T3 - T1);
    p.gamma = (a * B / 2.0) * T2 / den;
    p.c1 = -(a * B / 2.0) * (T1 * T1 + T3 * T3) / den;
    p.f2 = f2;
    p.t2 = T / 2.0 + g * (1.0 / (f0 * f0) - i2);
  }
  return p;
}

}  // namespace dc
