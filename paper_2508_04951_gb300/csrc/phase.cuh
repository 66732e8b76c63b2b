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
  // 16: runs of 16 bins k0 + s i (s d = fs / 4096) may step the phase from
  // its first bin (iono_apply_run16); 1: every bin evaluated in full.  Set by
  // the host where the stepped error bound stays below 1e-7 rad.
  int run;
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

DC_DEV float bin_kt(const PhaseParams& P, int k) {
  const int L = 1 << P.log2L;
  return (float)(k < (L >> 1) ? k : k - L);
}

// Reduced phase angle theta in about [-pi, pi] for bin k of an L-point DFT,
// as a double-float: f_k = fc + (fs/L) kt with kt = k (k < L/2) or k - L
// (fftfreq order).  A bin at f_k == 0 (DC under RF sampling) gets 0.
DC_DEV df iono_theta_df(const PhaseParams& P, int k) {
  const float kt = bin_kt(P, k);
  df f = df_add(df{P.fc_hi, P.fc_lo}, df_mul_f(df{P.d_hi, P.d_lo}, kt));
  if (f.hi == 0.0f) return df{0.0f, 0.0f};
  df phi = df_div(df{P.a_hi, P.a_lo}, f);
  phi = reduce_2pi(phi);
  phi = reduce_2pi(phi);                   // second round for very large phi
  return phi;
}
DC_DEV float iono_theta(const PhaseParams& P, int k) {
  const df t = iono_theta_df(P, k);
  return t.hi + t.lo;
}

// Correction factor exp(-i phi_k) (Eq. 16).
DC_DEV float2 iono_factor(const PhaseParams& P, int k) {
  float s, c;
  __sincosf(iono_theta(P, k), &s, &c);
  return make_float2(c, -s);
}

// v[i] *= exp(-i phi_k) for the 16 bins k = k0 + s i, all on one side of L/2,
// with s (fs / L) = fs / 4096.  With P.run == 16 only k0 is evaluated in
// full; each next phase adds phi_k - phi_(k-s) = -A s d / (f_(k-s) f_k), the
// exact difference of Eq. 16's phase between neighbouring bins, computed in
// float and accumulated in double-float (|step| <= 0.02 rad, relative error
// of a step ~3e-7, so 15 steps stay within 1e-7 rad; the host checks the
// bound).  The angle is left unreduced across the run (it moves < 0.3 rad).
DC_DEV void iono_apply_run16(const PhaseParams& P, int k0, int s, float2 (&v)[16]) {
  if (P.run != 16) {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = cmul(v[i], iono_factor(P, k0 + s * i));
    return;
  }
  df th = iono_theta_df(P, k0);
  float kt = bin_kt(P, k0);
  float fprev = fmaf(P.d_hi, kt, P.fc_hi);
  const float c = P.a_hi * ((float)s * P.d_hi);
  const float fs_step = (float)s;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (i) {
      kt += fs_step;
      const float f = fmaf(P.d_hi, kt, P.fc_hi);
      const float step = -__fdividef(c, fprev * f);
      const df t = two_sum(th.hi, step);
      th = df{t.hi, t.lo + th.lo};
      fprev = f;
    }
    float sn, cs;
    __sincosf(th.hi + th.lo, &sn, &cs);
    v[i] = cmul(v[i], make_float2(cs, -sn));
  }
}

}  // namespace dc
