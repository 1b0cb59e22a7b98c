// ff.cuh -- float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The building blocks are the error-free
// transformations of Knuth (TwoSum: a + b = s + e exactly) and of the fused
// multiply-add (TwoProd: a * b = p + e exactly, e = fma(a, b, -p)); sums of
// products use the compensated dot product of Ogita, Rump and Oishi (2005).
//
// GB300 runs FP32 at about 64x the FP64 rate, so FP64-class accuracy is
// cheaper this way than on the FP64 pipe.  Exponent range is that of float:
// callers keep values O(1) (the GMLS tiles are eps-scaled).
#pragma once
#include <cuda_runtime.h>

namespace gmls {

struct ff {
  float h, l;
  ff() = default;
  __host__ __device__ constexpr ff(float a, float b) : h(a), l(b) {}
  // split a double: h = fl32(d), l = fl32(d - h)
  __device__ __forceinline__ explicit ff(double d) {
    h = __double2float_rn(d);
    l = __double2float_rn(d - (double)h);
  }
};

// s + e == a + b exactly (Knuth)
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff(s, e);
}

// s + e == a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff(s, e);
}

// p + e == a * b exactly
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return ff(p, e);
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  ff s = two_sum(a.h, b.h);
  float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return quick_two_sum(s.h, e);
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.h, -a.l); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  ff p = two_prod(a.h, b.h);
  float e = __fmaf_rn(a.h, b.l, p.l);
  e = __fmaf_rn(a.l, b.h, e);
  return quick_two_sum(p.h, e);
}

__device__ __forceinline__ ff mul_f(ff a, float b) {
  ff p = two_prod(a.h, b);
  float e = __fmaf_rn(a.l, b, p.l);
  return quick_two_sum(p.h, e);
}

__device__ __forceinline__ ff add_f(ff a, float b) {
  ff s = two_sum(a.h, b);
  float e = __fadd_rn(s.l, a.l);
  return quick_two_sum(s.h, e);
}

// 1 / a: one Newton step on the float reciprocal
__device__ __forceinline__ ff recip(ff a) {
  float q = 1.0f / a.h;
  ff r = ff(1.0f, 0.0f) - a * ff(q, 0.0f);  // residual 1 - a q, tiny
  float c = __fmul_rn(r.h, q);
  return quick_two_sum(q, c);
}

// sqrt(a), a >= 0: one Newton step on the float square root (the step's
// quotient only needs float accuracy: it is about 2^-24 of the result)
__device__ __forceinline__ ff sqrt_ff(ff a) {
  if (!(a.h > 0.0f)) return ff(0.0f, 0.0f);
  float s = sqrtf(a.h);
  ff ss = two_prod(s, s);
  float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, ss.h), ss.l), a.l);
  float c = __fdividef(r, __fmul_rn(2.0f, s));
  return quick_two_sum(s, c);
}

// float -> double by re-biasing the exponent field with integer ops (exact for
// normal floats and zeros; denormals and inf/nan take the conversion
// instruction), so that the float-float -> FP64 store costs one FP64 add
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) {
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)(u & 0x80000000u) << 32);
    return (double)f;
  }
  const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double to_double(ff a) { return f2d_exact(a.h) + f2d_exact(a.l); }

// constant with float-float split (h, l), and x * p for a power of two p
// (exact: both parts scale); used by the generated basis evaluation
__device__ __forceinline__ ff gmls_cst(ff, double, float h, float l) { return ff(h, l); }
__device__ __forceinline__ ff gmls_scale2(ff x, float p) { return ff(x.h * p, x.l * p); }

// Float-float split of a double without FP64 conversions: h is d cut to 24
// significant bits (exact in a float), l the remaining 29 bits rounded to a
// float by an integer -> float conversion, so |d - (h + l)| <= 2^-48 |d| and
// |l| < ulp(h).  The integer path covers 2^-74 <= |d| < 2^127 (h and the scale
// 2^(e - 1075) are then normal floats); other values take the conversions.
__device__ __forceinline__ ff split_d(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  if (e < 949u || e > 1150u) {
    const float h = __double2float_rn(d);
    return ff(h, __double2float_rn(d - (double)h));
  }
  const unsigned s = (unsigned)(b >> 63) << 31;
  const float h = __uint_as_float(s | ((e - 896u) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
  const float lo = __uint2float_rn((unsigned)(b & 0x1fffffffu));
  const float sc = __uint_as_float((e - 948u) << 23);  // 2^(e - 1075)
  return ff(h, __uint_as_float(__float_as_uint(__fmul_rn(lo, sc)) | s));
}

// x_j - x_T as float-float: the FP64 difference (the same rounded value the
// exact neighbour distances use) split by split_d.  Independent of where the
// cloud sits: no float copy of the absolute coordinates is involved.
__device__ __forceinline__ ff diff_ff(double xj, double xt) { return split_d(__dsub_rn(xj, xt)); }

// Compensated accumulation of products (Ogita-Rump-Oishi Dot2 with
// float-float factors): acc_h + acc_l tracks sum(a_i * b_i) to about 2^-48.
struct Dot2 {
  float h = 0.0f, l = 0.0f;
  __device__ __forceinline__ void init(ff v) {
    h = v.h;
    l = v.l;
  }
  __device__ __forceinline__ void add_prod(ff a, ff b) {
    ff p = two_prod(a.h, b.h);
    float e = __fmaf_rn(a.h, b.l, p.l);
    e = __fmaf_rn(a.l, b.h, e);
    ff s = two_sum(h, p.h);
    h = s.h;
    l = __fadd_rn(l, __fadd_rn(s.l, e));
  }
  // a * b with b a plain float (one product term fewer)
  __device__ __forceinline__ void add_prod_f(ff a, float b) {
    ff p = two_prod(a.h, b);
    float e = __fmaf_rn(a.l, b, p.l);
    ff s = two_sum(h, p.h);
    h = s.h;
    l = __fadd_rn(l, __fadd_rn(s.l, e));
  }
  __device__ __forceinline__ ff value() const { return quick_two_sum(h, l); }
};

}  // namespace gmls
