// Device-side building blocks shared by the library's kernels: complex
// arithmetic on float2, error-free float transforms (double-float), the
// in-register DFTs of radix 2/4/8/16 used by the Stockham stages, and the
// twiddle tables' layout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define DC_DEV __device__ __forceinline__

namespace dc {

// ---------------------------------------------------------------- complex
// Complex add and subtract as packed two-lane FP32 instructions (one issue
// for both parts; each part rounds as the scalar add or subtract does).
DC_DEV float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
DC_DEV float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 pa, pb, pr;\n mov.b64 pa, {%2, %3};\n mov.b64 pb, {%4, %5};\n"
      " sub.rn.f32x2 pr, pa, pb;\n mov.b64 {%0, %1}, pr;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
DC_DEV float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
DC_DEV float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (DIR < 0) or +i (DIR > 0)
template <int DIR> DC_DEV float2 mul_i(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
template <int DIR> DC_DEV float2 conj_if(float2 w) {
  return DIR < 0 ? w : make_float2(w.x, -w.y);
}

// (float)i for |i| < 2^22, exactly, on the full-rate integer and FP32 pipes:
// i added into the mantissa of 1.5 * 2^23 (whose ulp is 1), then 1.5 * 2^23
// subtracted exactly.  The conversion instruction runs at a quarter of that
// rate, which matters in loops that convert once per term.
DC_DEV float exact_i2f(int i) {
  return __int_as_float(i + 0x4B400000) - 12582912.0f;
}

// ------------------------------------------- programmatic dependent launch
// A kernel launched with the programmatic-serialization attribute may start
// while the kernel before it in the stream is still running; pdl_wait()
// blocks until that kernel has completed and its memory is visible, so it
// must come before the first access to anything the earlier kernel writes
// or reads.  pdl_release() lets such a dependent start once every CTA of the
// calling grid has executed it (or exited).  Both are no-ops for kernels
// launched without the attribute or without a dependent.
DC_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
DC_DEV void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------ double-float
// Dekker/Knuth error-free transforms: a value is hi + lo with |lo| <= ulp(hi)/2.
struct df { float hi, lo; };
DC_DEV df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
DC_DEV df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
DC_DEV df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return two_sum(s.hi, lo);
}
// (a.hi + a.lo) * k for a float k
DC_DEV df df_mul_f(df a, float k) {
  df p = two_prod(a.hi, k);
  return two_sum(p.hi, fmaf(a.lo, k, p.lo));
}
// a / b, both double-float.  One reciprocal of b.hi serves both quotient
// steps: q1 = a.hi / b.hi to a couple of ulps, the remainder
// a - q1 b is formed exactly (two_prod, Sterbenz), and its quotient q2 only
// needs float accuracy relative to itself (|q2| ~ 2^-23 |q1|).
DC_DEV df df_div(df a, df b) {
  const float rb = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, rb);
  df p = two_prod(q1, b.hi);
  float r = __fsub_rn(a.hi, p.hi);          // exact: q1*b.hi is within a few ulps of a.hi
  r = __fsub_rn(r, p.lo);
  r = __fadd_rn(r, a.lo);
  r = fmaf(-q1, b.lo, r);
  const float q2 = __fmul_rn(r, rb);
  return two_sum(q1, q2);
}

// exp(2 pi i g n) for a rotation rate g (cycles per sample) held as the
// double-float g_hi + g_lo and an output index n < 2^24: g n is formed as a
// double-float (two_prod, exact for the high part), its integer part removed
// exactly (rintf of the high part), and the remaining fraction of a cycle
// goes to sincospif.  Used for the carrier term of a passband dilation and
// for frequency conversion, whose phases reach thousands of cycles.
DC_DEV float2 cycles_rot(float g_hi, float g_lo, int n) {
  const float fn = (float)n;
  const df p = two_prod(g_hi, fn);
  const float r = __fadd_rn(__fsub_rn(p.hi, rintf(p.hi)), fmaf(g_lo, fn, p.lo));
  float s, c;
  sincospif(2.0f * r, &s, &c);
  return make_float2(c, s);
}

// --------------------------------------------------------- radix-R DFTs
// DIR = -1: forward, exp(-2 pi i kn/R); DIR = +1: inverse (no 1/R).
// Output in natural order, in place.
template <int DIR> DC_DEV void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int DIR> DC_DEV void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  float2 t0 = cadd(v0, v2), t1 = csub(v0, v2);
  float2 t2 = cadd(v1, v3), d = csub(v1, v3);
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  // v1, v3 = t1 +- (-/+ i) d: the parts cross, so these four stay scalar
  if constexpr (DIR < 0) {
    v1 = make_float2(t1.x + d.y, t1.y - d.x);
    v3 = make_float2(t1.x - d.y, t1.y + d.x);
  } else {
    v1 = make_float2(t1.x - d.y, t1.y + d.x);
    v3 = make_float2(t1.x + d.y, t1.y - d.x);
  }
}

// exp(DIR * 2 pi i m / 16) for a compile-time m (folded by the compiler)
template <int DIR, int M> DC_DEV float2 w16() {
  constexpr int m = ((M % 16) + 16) % 16;
  constexpr float c[16] = {
      1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
      0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
      -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
      0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
  constexpr float cs = c[m];
  constexpr float sn = c[(m + 12) % 16];    // sin(x) = cos(x - pi/2)
  return make_float2(cs, DIR < 0 ? -sn : sn);
}

template <int DIR, int M> DC_DEV float2 tw16(float2 a) {
  constexpr int m = ((M % 16) + 16) % 16;
  if constexpr (m == 0) return a;
  else if constexpr (m == 4) return mul_i<DIR>(a);
  else if constexpr (m == 8) return make_float2(-a.x, -a.y);
  else if constexpr (m == 12) return mul_i<-DIR>(a);
  else return cmul(a, w16<DIR, M>());
}

template <int DIR> DC_DEV void dft8(float2 (&v)[8]) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  o1 = tw16<DIR, 2>(o1);
  o2 = tw16<DIR, 4>(o2);
  o3 = tw16<DIR, 6>(o3);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <int DIR> DC_DEV void dft16(float2 (&v)[16]) {
  // 16 = 4 x 4: columns n2 (stride 4 in n), twiddle W16^(n2 k1), rows.
  float2 a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 x0 = v[n2], x1 = v[n2 + 4], x2 = v[n2 + 8], x3 = v[n2 + 12];
    dft4<DIR>(x0, x1, x2, x3);
    a[n2][0] = x0; a[n2][1] = x1; a[n2][2] = x2; a[n2][3] = x3;
  }
  a[1][1] = tw16<DIR, 1>(a[1][1]);
  a[1][2] = tw16<DIR, 2>(a[1][2]);
  a[1][3] = tw16<DIR, 3>(a[1][3]);
  a[2][1] = tw16<DIR, 2>(a[2][1]);
  a[2][2] = tw16<DIR, 4>(a[2][2]);
  a[2][3] = tw16<DIR, 6>(a[2][3]);
  a[3][1] = tw16<DIR, 3>(a[3][1]);
  a[3][2] = tw16<DIR, 6>(a[3][2]);
  a[3][3] = tw16<DIR, 9>(a[3][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 x0 = a[0][k1], x1 = a[1][k1], x2 = a[2][k1], x3 = a[3][k1];
    dft4<DIR>(x0, x1, x2, x3);
    v[k1] = x0; v[k1 + 4] = x1; v[k1 + 8] = x2; v[k1 + 12] = x3;
  }
}

template <int R, int DIR> DC_DEV void dft(float2 (&v)[R]) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<DIR>(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4<DIR>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    dft8<DIR>(v);
  } else {
    static_assert(R == 16, "radix must be 1, 2, 4, 8 or 16");
    dft16<DIR>(v);
  }
}

// Bounds checks of the checked build (compiled with -DDC_CHECKED).  A failed
// check raises the context's error flag to 3 (flags only rise: 3 bounds, 2
// parameters out of range, 1 a bounded wait ran out) and the caller skips the
// access -- never a trap.  In the normal build every check is `true`.
DC_DEV void bounds_fail(int* err) {
  if (err) atomicMax(err, 3);
}
#ifdef DC_CHECKED
#define DC_IN_BOUNDS(cond, err) ((cond) ? true : (::dc::bounds_fail(err), false))
#else
#define DC_IN_BOUNDS(cond, err) true
#endif

// v[q] *= w^q for q = 1 .. N-1 (N = 2, 4, 8, 16) from correctly rounded
// b[0] = w, b[1] = w^2, b[2] = w^4, b[3] = w^8 (entries past log2 N unused):
// w^q is the product of the bases of q's set bits, so every factor carries
// at most three roundings beyond the table's own.
template <int N> DC_DEV void apply_powers(float2 (&v)[N], const float2 (&b)[4]) {
  static_assert(N == 2 || N == 4 || N == 8 || N == 16, "N must be 2, 4, 8 or 16");
  float2 p[N];
  p[1] = b[0];
  if constexpr (N > 2) {
    p[2] = b[1];
    p[3] = cmul(b[1], b[0]);
  }
  if constexpr (N > 4) {
    p[4] = b[2];
#pragma unroll
    for (int q = 1; q < 4; ++q) p[4 + q] = cmul(b[2], p[q]);
  }
  if constexpr (N > 8) {
    p[8] = b[3];
#pragma unroll
    for (int q = 1; q < 8; ++q) p[8 + q] = cmul(b[3], p[q]);
  }
#pragma unroll
  for (int q = 1; q < N; ++q) v[q] = cmul(v[q], p[q]);
}

// --------------------------------------------------------------- twiddles
// One device table of roots of unity, filled once per context in FP64 on the
// host and rounded to float (fill_twiddles in twiddle_host.h):
//   [0, 4096)          W4096^t = exp(-2 pi i t / 4096)
//   [4096, 5120)       W(2^20)^j        j in [0, 1024)
//   [5120, 6144)       W(2^20)^(1024 i) i in [0, 1024)
//   [6144, 6384)       W256^(r k)   at 6144 + (r-1)*16 + k,  r in [1,16), k in [0,16)
//   [6384, 10224)      W4096^(r j)  at 6384 + (r-1)*256 + j, r in [1,16), j in [0,256)
// W_M^t for M | 4096 is W4096^(t 4096/M); W_L^t for L | 2^20 is
// W(2^20)^s with s = t 2^20/L, split as s = 1024 i + j.  The last two blocks
// are the per-stage twiddles of a 4096-point radix-16 row, laid out so a
// warp's 32 consecutive butterflies read consecutive entries.
constexpr int kTwMax = 4096;
constexpr int kTwLo = 4096;
constexpr int kTwHi = 5120;
constexpr int kTwS2 = 6144;
constexpr int kTwS3 = 6384;
constexpr int kTwSize = 10224;
constexpr int kLog2Big = 20;

template <int DIR> DC_DEV float2 tw_m(const float2* __restrict__ tw, int t4096) {
  return conj_if<DIR>(__ldg(tw + t4096));
}
// W_L^e for the four-step, e in [0, L), L = 2^log2L <= 2^20
template <int DIR> DC_DEV float2 tw_big(const float2* __restrict__ tw, uint32_t e, int log2L) {
  uint32_t s = e << (kLog2Big - log2L);
  float2 w = cmul(__ldg(tw + kTwHi + (s >> 10)), __ldg(tw + kTwLo + (s & 1023u)));
  return conj_if<DIR>(w);
}

}  // namespace dc
