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

// (a_h + a_l) - (b_h + b_l) for coordinates stored as float pairs
__device__ __forceinline__ ff sub_pair(float ah, float al, float bh, float bl) {
  ff s = two_sum(ah, -bh);
  float e = __fadd_rn(s.l, __fsub_rn(al, bl));
  return quick_two_sum(s.h, e);
}

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
  __device__ __forceinline__ ff value() const { return quick_two_sum(h, l); }
};

}  // namespace gmls
