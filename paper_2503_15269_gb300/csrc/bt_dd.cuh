// Double-float arithmetic: a value is an unevaluated pair hi + lo of float32
// numbers with |lo| <= ulp(hi) / 2, about 48 significand bits.  Float64
// issues at 1/64 of the float32 rate on this part, so the dense float64
// work of the LQR formation runs on the float32 pipe in this form.
//
// Building blocks (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2; the FMA form of
// the exact product):
//   two_sum(a, b)      s + e = a + b exactly, s = fl(a + b)
//   fast_two_sum(a, b) the same for |a| >= |b| (or a = 0)
//   two_prod(a, b)     p + e = a * b exactly, p = fl(a * b), e = fma(a, b, -p)
// Every operation below uses the explicitly rounded intrinsics, which the
// compiler never contracts or reassociates: a product folded into a later
// addition as one FMA would break the exactness these rely on.
#pragma once
#include <cuda_runtime.h>

namespace bt {

struct dd {
  float h, l;
};

__device__ __forceinline__ dd dd_make(float h, float l) {
  dd r;
  r.h = h;
  r.l = l;
  return r;
}

__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return dd_make(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

// x + y, both pairs (the accurate form: the low parts are summed with their
// own error term, so cancellation of the high parts keeps full precision)
__device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = two_sum(x.h, y.h);
  const dd t = two_sum(x.l, y.l);
  s.l = __fadd_rn(s.l, t.h);
  s = fast_two_sum(s.h, s.l);
  s.l = __fadd_rn(s.l, t.l);
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ dd dd_neg(dd x) { return dd_make(-x.h, -x.l); }

// x * y: exact product of the high parts plus the two cross terms (the
// lo * lo term is below 2^-48 of the result)
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return fast_two_sum(p, e);
}

// Dot-product accumulator: the high parts of the exact products are summed
// by two_sum into s (exact), and every rounding error, the low parts of the
// products and the cross terms go to the float32 correction c.  One term
// costs 12 float32 operations; the sum of n terms is within about n 2^-48
// of the sum of their magnitudes.
struct DDAcc {
  float s, c;
  __device__ __forceinline__ void init(dd x) {
    s = x.h;
    c = x.l;
  }
  __device__ __forceinline__ void init0() { s = c = 0.f; }
  // += a * b
  __device__ __forceinline__ void fma(dd a, dd b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  }
  // -= a * b
  __device__ __forceinline__ void fms(dd a, dd b) { fma(dd_neg(a), b); }
  __device__ __forceinline__ void add(dd x) {
    const dd t = two_sum(s, x.h);
    s = t.h;
    c = __fadd_rn(c, __fadd_rn(t.l, x.l));
  }
  __device__ __forceinline__ dd value() const { return fast_two_sum(s, c); }
};

// sqrt(a) for a > 0: the float32 root plus one Newton correction computed
// with the exact square of the root: s + (a - s^2) / (2 s)
__device__ __forceinline__ dd dd_sqrt(dd a) {
  const float s = __fsqrt_rn(a.h);
  const float p = __fmul_rn(s, s);
  const float pe = __fmaf_rn(s, s, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), pe), a.l);
  return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}

// 1 / a: the float32 reciprocal x plus one Newton correction x (1 - a x),
// with a x formed exactly in its high part
__device__ __forceinline__ dd dd_rcp(dd a) {
  const float x = __fdiv_rn(1.f, a.h);
  const float p = __fmul_rn(a.h, x);
  const float pe = __fmaf_rn(a.h, x, -p);
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), pe), __fmul_rn(a.l, x));
  return fast_two_sum(x, __fmul_rn(x, e));
}

// float64 <-> float32 conversions on the integer pipes.  A conversion
// instruction runs on the float64 pipe (1/64 of the float32 rate here), and
// the formation converts every input and output element, so these rebuild
// the IEEE 754 encodings from the bits instead; values outside the normal
// range of the narrower format take the hardware conversion.
//
// float -> double is exact: the sign, the exponent rebiased by 1023 - 127
// and the 23 fraction bits shifted up by 29.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;  // zeros, subnormals, infinities, NaN
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// double -> float, round to nearest even: for a normal float result (biased
// float64 exponent 897 .. 1150) the sign, the rebiased exponent and the top
// 23 of the 52 fraction bits, plus one unit in the last place when the 29
// dropped bits are above half, or exactly half with an odd kept part (a
// carry out of the fraction moves into the exponent, reaching infinity from
// the largest binade as IEEE rounding does).
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u > 253u) return __double2float_rn(x);
  unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
  return __uint_as_float(f);
}

// float64 <-> pair: hi = fl32(x), lo = fl32(x - hi) (x - hi is exact in
// float64), so hi + lo is within 2^-48 of x; the merge rounds hi + lo once to
// float64.  One float64 operation each.
__device__ __forceinline__ dd dd_from(double x) {
  const float h = d2f_rn(x);
  return dd_make(h, d2f_rn(x - f2d_exact(h)));
}

__device__ __forceinline__ double dd_to(dd x) { return f2d_exact(x.h) + f2d_exact(x.l); }

}  // namespace bt
