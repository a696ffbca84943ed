// ff.cuh -- float-float ("double-single") arithmetic: a value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 executes FP64 at 1/73 of its FP32 rate; the chemical-potential passes
// need about 1e-12 relative accuracy and run in this arithmetic on the FP32
// pipes.  Building blocks are the error-free transformations TwoSum (Knuth),
// Fast2Sum (Dekker) and TwoProduct through a fused multiply-add.  exp follows
// the table method (Tang, ACM TOMS 15(2), 1989): x = (32 m + j) ln2/32 + r,
// exp(x) = 2^m 2^(j/32) exp(r) with |r| <= ln2/64 and a degree-6 Taylor
// polynomial for exp(r); the 32 values 2^(j/32) are split into float pairs
// from their FP64 values when the library starts.
#pragma once

#include <cuda_runtime.h>

namespace mxe {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // constants of the kernels ((R)0, (R)2, (R)(1.0/12.0), ...)
  __host__ __device__ explicit ff(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};

__device__ __forceinline__ ff ff_make(float h, float l = 0.f) { return ff{h, l}; }

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  const float e = (a - (s - bp)) + (b - bp);
  return ff{s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return ff{s, b - (s - a)};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = a * b;
  return ff{p, fmaf(a, b, -p)};
}

// a + b with one TwoSum on the high parts: the error is bounded by about
// 2^-47 max(|a|, |b|) -- enough wherever absolute accuracy relative to the
// operands is what matters (exponent arguments, sums of positive terms, per
// pair sums that are then added in FP64).
__device__ __forceinline__ ff operator+(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff operator-(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.hi, b);
  s.lo += a.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ bool operator<(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) {
  a = a * b;
  return a;
}

// 1 / a: y = 1/hi, one Newton correction y + y (1 - a y)
__device__ __forceinline__ ff ff_recip(ff a) {
  const float y = 1.0f / a.hi;
  const ff ay = ff_mul_f(a, y);
  const float e = (1.0f - ay.hi) - ay.lo;
  return fast_two_sum(y, y * e);
}

__device__ __forceinline__ ff ff_from_double(double x) {
  const float h = (float)x;
  return ff{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// sqrt: y = sqrt(hi) in FP32, one Newton correction y + (a - y^2) / (2 y).
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.hi > 0.f)) return ff{0.f, 0.f};
  const float y = sqrtf(a.hi);
  const ff y2 = two_prod(y, y);
  const float r = ((a.hi - y2.hi) - y2.lo + a.lo) * (0.5f / y);
  return fast_two_sum(y, r);
}

// 2^(j/32), j = 0..31, as float pairs (filled from FP64 values at start-up).
struct FFExpTable {
  float hi[32], lo[32];
};

// exp(x) for |x| < 87 (inputs of the radial terms are far smaller).
// tab(j) returns 2^(j/32) as a float pair.  The absolute error of the reduced
// argument r is the relative error of the result, so r is formed to about
// 1e-16 and exp(r) to about 1e-14.
template <typename Tab>
__device__ __forceinline__ ff ff_exp_t(ff x, const Tab& tab) {
  // ln2/32 = c1 + c2 + c3: c1 has 12 significant bits, so n * c1 is exact for
  // |n| < 2^12 (|x| < 88); c2 and c3 are the next float-sized pieces.
  const float kInvLn2x32 = 46.16624069213867f;           // 32 / ln 2
  const float c1 = 0.02165985107421875f;
  const float c2 = 9.983182280848268e-07f;
  const float c3 = 5.14560928046269e-14f;
  const float n = rintf(x.hi * kInvLn2x32);
  const int ni = (int)n;
  const int j = ni & 31;
  const int m = (ni - j) / 32;
  // r = x - n ln2/32.  x.hi - n c1 is exact: n c1 is, and for n != 0 the two
  // lie within a factor of two of each other (Sterbenz).  n c2 is split
  // exactly by TwoProduct; x.lo (up to 2e-6) and -n c2 enter by TwoSum, and
  // the remaining pieces are below 1e-9.
  const float s = fmaf(-n, c1, x.hi);
  const ff p2 = two_prod(n, c2);
  const ff t = two_sum(s, -p2.hi);
  const ff u = two_sum(t.hi, x.lo);
  const ff r = fast_two_sum(u.hi, (t.lo + u.lo) - (p2.lo + n * c3));
  // exp(r) = 1 + r + r^2/2 + r^3 (1/6 + r/24 + r^2/120 + r^3/720), |r| <= ln2/64.
  // The cubic tail (below 2.2e-7) in FP32 from r.hi; r^2/2 from TwoProduct
  // plus the cross term; r + r^2/2 by Fast2Sum (|r| > r^2/2); every remaining
  // piece is below 3e-7, so one float sums them to about 1e-14.
  const float q = r.hi;
  const float q2 = q * q;
  const float tail = q2 * q * fmaf(fmaf(fmaf(q, 1.0f / 720.0f, 1.0f / 120.0f), q, 1.0f / 24.0f), q, 1.0f / 6.0f);
  const float e2 = fmaf(q, q, -q2) + 2.0f * q * r.lo;  // r^2 = q2 + e2 (to 1e-19)
  const ff s1 = fast_two_sum(q, 0.5f * q2);
  const float small = ((s1.lo + r.lo) + 0.5f * e2) + tail;
  ff pe = fast_two_sum(1.0f, s1.hi);
  pe = fast_two_sum(pe.hi, pe.lo + small);
  const ff pt = pe * tab(j);
  // 2^m by its exponent bits (|m| <= 126 for |x| < 87; clamped to the normal
  // range beyond)
  const float sc = __int_as_float((min(max(m, -126), 127) + 127) << 23);
  return ff{pt.hi * sc, pt.lo * sc};
}

// with the table in constant memory (uniform indices are broadcast, distinct
// ones are served one after another)
__device__ __forceinline__ ff ff_exp(ff x, const FFExpTable& T) {
  return ff_exp_t(x, [&](int j) { return ff{T.hi[j], T.lo[j]}; });
}

// with the table copied to shared memory as 32 (hi, lo) pairs: the 32 entries
// fall in distinct banks, so lanes with different indices read in one pass
__device__ __forceinline__ ff ff_exp(ff x, const float2* T) {
  return ff_exp_t(x, [&](int j) {
    const float2 v = T[j];
    return ff{v.x, v.y};
  });
}

}  // namespace mxe
