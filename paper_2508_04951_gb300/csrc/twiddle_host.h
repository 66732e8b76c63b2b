// Host-side construction of the device twiddle table (layout in common.cuh):
// every entry computed in double precision and rounded once to float.
#pragma once

#include <cmath>

#include "common.cuh"
#include "fused.cuh"

namespace dc {

inline void fill_twiddles(float2* tw) {
  const double pi = 3.14159265358979323846;
  auto w = [pi](double num, double den) {
    const double a = -2.0 * pi * num / den;
    return make_float2((float)std::cos(a), (float)std::sin(a));
  };
  for (int t = 0; t < 4096; ++t) tw[t] = w(t, 4096.0);
  for (int j = 0; j < 1024; ++j) {
    tw[kTwLo + j] = w(j, (double)(1 << 20));
    tw[kTwHi + j] = w(j, 1024.0);
  }
  for (int r = 1; r < 16; ++r) {
    for (int k = 0; k < 16; ++k) tw[kTwS2 + (r - 1) * 16 + k] = w((r * k) % 256, 256.0);
    for (int j = 0; j < 256; ++j) tw[kTwS3 + (r - 1) * 256 + j] = w((r * j) % 4096, 4096.0);
  }
}

// Four-step twiddles of the spectrum-apply kernel (layout in fused.cuh):
// exp(+2 pi i m / L) with m = 2^b n2 mod L, in double, rounded once.
inline void fill_four_step(float2* t4) {
  const double pi = 3.14159265358979323846;
  for (int l1 = 2; l1 <= 16; l1 *= 2) {
    const long long L = 4096LL * l1;
    for (int b = 0; b < kT4Log2(l1); ++b)
      for (int n2 = 0; n2 < 4096; ++n2) {
        const long long q = 1LL << b;
        const double a = 2.0 * pi * (double)((q * n2) % L) / (double)L;
        t4[kT4Offset(l1) + b * 4096 + n2] = make_float2((float)std::cos(a), (float)std::sin(a));
      }
  }
}

}  // namespace dc
