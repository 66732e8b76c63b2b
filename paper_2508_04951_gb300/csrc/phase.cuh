// Ionospheric phase phi_k = 4 pi K2 / (c f_k) of the FFT correction
// (Eqs. 15-16), evaluated and range-reduced in double-float arithmetic before
// the FP32 sincos.  phi reaches thousands of radians at TEC ~ 1e2 TECU and
// f ~ 1 GHz, where one float ulp is ~2.4e-4 rad; the double-float path keeps
// ~48 bits, so the reduced angle is good to float rounding.
#pragma once

#include "common.cuh"

namespace dc {

// Per-pulse constants, split on the host from FP64 into hi + lo floats.
struct PhaseParams {
  float a_hi, a_lo;     // A = 4 pi kappa E / c      [rad Hz]
  float fc_hi, fc_lo;   // carrier fc                [Hz]; 0 = RF sampling
  float d_hi, d_lo;     // bin spacing fs / L        [Hz]
  int log2L;            // transform length L = 2^log2L
  int enabled;          // 0 when E == 0 (identity)
};

// 2 pi = TWO_PI_HI + TWO_PI_LO
constexpr float kTwoPiHi = 6.28318548202514648f;
constexpr float kTwoPiLo = -1.74845560007448833e-07f;
constexpr float kInvTwoPi = 0.159154943091895336f;

// theta(phi) = phi - 2 pi n, one reduction round in double-float
DC_DEV df reduce_2pi(df p) {
  float n = rintf(p.hi * kInvTwoPi);
  df q = two_prod(n, kTwoPiHi);
  float hi = __fsub_rn(p.hi, q.hi);        // exact (Sterbenz) when p ~ q
  float lo = __fsub_rn(__fadd_rn(p.lo, -q.lo), n * kTwoPiLo);
  return two_sum(hi, lo);
}

// Reduced phase angle theta in about [-pi, pi] for bin k of an L-point DFT:
// f_k = fc + (fs/L) kt with kt = k (k < L/2) or k - L (fftfreq order).
// A bin at f_k == 0 (DC under RF sampling) gets 0.
DC_DEV float iono_theta(const PhaseParams& P, int k) {
  const int L = 1 << P.log2L;
  const float kt = (float)(k < (L >> 1) ? k : k - L);
  df f = df_add(df{P.fc_hi, P.fc_lo}, df_mul_f(df{P.d_hi, P.d_lo}, kt));
  if (f.hi == 0.0f) return 0.0f;
  df phi = df_div(df{P.a_hi, P.a_lo}, f);
  phi = reduce_2pi(phi);
  phi = reduce_2pi(phi);                   // second round for very large phi
  return phi.hi + phi.lo;
}

// Correction factor exp(-i phi_k) (Eq. 16).
DC_DEV float2 iono_factor(const PhaseParams& P, int k) {
  float s, c;
  __sincosf(iono_theta(P, k), &s, &c);
  return make_float2(c, -s);
}

}  // namespace dc
