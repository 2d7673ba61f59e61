// Double-float ("double-word") arithmetic: a real number as the unevaluated
// sum hi + lo of two FP32 values with |lo| <= ulp(hi) / 2 (about 48
// significant bits), and complex numbers as pairs of them.  The mixed search
// keeps the per-pixel state of its per-flip chain (diag W, e, the rows of T,
// the port amplitudes and the objective) in this form so that the chain runs
// on the FP32 pipe: on GB300 an SM retires ~76x more FP32 than FP64 lanes per
// clock, and a dependent FP64 instruction costs a 64-cycle issue slot.
//
// Building blocks (each operation rounds to nearest, no contraction):
//   Fast2Sum (Dekker 1971): s + e = a + b exactly when |a| >= |b|;
//   2Sum (Knuth / Moller): s + e = a + b exactly, any order;
//   2ProdFMA: p + e = a b exactly, e = fma(a, b, -p).
// Double-word operations follow Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic"
// (ACM TOMS 44, 2017): the accurate sum of two double-words (relative error
// below 3 u^2, u = 2^-24, also under cancellation), the product of two
// double-words with FMA (below 5 u^2) and of a double-word by a float.  The
// reciprocal and the square root take one Newton step from the correctly
// rounded FP32 value, with the residual formed exactly by an FMA.
//
// The header also compiles as plain C++ (host), so that the CPU tests can
// check every operation against exact rational arithmetic; compile the host
// side with floating-point contraction off.
#pragma once

#if defined(__CUDACC__)
#define DD_FN __host__ __device__ __forceinline__
#else
#include <cmath>
#define DD_FN static inline
#endif

namespace pngf {

#if defined(__CUDA_ARCH__)
DD_FN float dd_fadd(float a, float b) { return __fadd_rn(a, b); }
DD_FN float dd_fsub(float a, float b) { return __fsub_rn(a, b); }
DD_FN float dd_fmul(float a, float b) { return __fmul_rn(a, b); }
DD_FN float dd_ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
DD_FN float dd_frcp(float a) { return __frcp_rn(a); }
DD_FN float dd_fsqrt(float a) { return __fsqrt_rn(a); }
#else
DD_FN float dd_fadd(float a, float b) { return a + b; }
DD_FN float dd_fsub(float a, float b) { return a - b; }
DD_FN float dd_fmul(float a, float b) { return a * b; }
DD_FN float dd_ffma(float a, float b, float c) { return std::fmaf(a, b, c); }
DD_FN float dd_frcp(float a) { return 1.0f / a; }
DD_FN float dd_fsqrt(float a) { return std::sqrt(a); }
#endif

struct dd {
  float hi, lo;
};
struct cdd {
  dd re, im;
};

// ---- error-free transformations
DD_FN dd fast2sum(float a, float b) {  // |a| >= |b| (or a == 0)
  const float s = dd_fadd(a, b);
  return dd{s, dd_fsub(b, dd_fsub(s, a))};
}
DD_FN dd two_sum(float a, float b) {
  const float s = dd_fadd(a, b);
  const float bv = dd_fsub(s, a);
  return dd{s, dd_fadd(dd_fsub(a, dd_fsub(s, bv)), dd_fsub(b, bv))};
}

// ---- real double-words
DD_FN dd dd_of(float a) { return dd{a, 0.0f}; }
DD_FN dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
// accurate sum of two double-words
DD_FN dd dd_add(dd x, dd y) {
  const dd s = two_sum(x.hi, y.hi);
  const dd t = two_sum(x.lo, y.lo);
  const dd v = fast2sum(s.hi, dd_fadd(s.lo, t.hi));
  return fast2sum(v.hi, dd_fadd(t.lo, v.lo));
}
DD_FN dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }
// product of two double-words (FMA)
DD_FN dd dd_mul(dd x, dd y) {
  const float ch = dd_fmul(x.hi, y.hi);
  const float cl1 = dd_ffma(x.hi, y.hi, -ch);
  const float cl2 = dd_ffma(x.lo, y.hi, dd_fmul(x.hi, y.lo));
  return fast2sum(ch, dd_fadd(cl1, cl2));
}
// product of a double-word and a float (FMA)
DD_FN dd dd_mul_f(dd x, float y) {
  const float ch = dd_fmul(x.hi, y);
  const float cl = dd_ffma(x.lo, y, dd_ffma(x.hi, y, -ch));
  return fast2sum(ch, cl);
}
// 1 / x: y0 = fl(1 / x.hi), r = 1 - x y0 (the first FMA is exact), y = y0 + y0 r
DD_FN dd dd_rcp(dd x) {
  const float y0 = dd_frcp(x.hi);
  const float r = dd_ffma(-x.lo, y0, dd_ffma(-x.hi, y0, 1.0f));
  return fast2sum(y0, dd_fmul(y0, r));
}
// sqrt(x), x >= 0: s0 = fl(sqrt(x.hi)), r = x - s0^2 (exact by FMA, plus x.lo), s = s0 + r / (2 s0)
DD_FN dd dd_sqrt(dd x) {
  if (!(x.hi > 0.0f)) return dd{0.0f, 0.0f};
  const float s0 = dd_fsqrt(x.hi);
  const float r = dd_fadd(dd_ffma(-s0, s0, x.hi), x.lo);
  return fast2sum(s0, dd_fmul(r, dd_fmul(0.5f, dd_frcp(s0))));
}
// x > y for normalised double-words
DD_FN bool dd_gt(dd x, dd y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }
DD_FN bool dd_lt(dd x, dd y) { return dd_gt(y, x); }
DD_FN dd dd_abs(dd x) { return (x.hi < 0.0f || (x.hi == 0.0f && x.lo < 0.0f)) ? dd_neg(x) : x; }

// ---- complex double-words
DD_FN cdd cdd_of(float re, float im) { return cdd{dd_of(re), dd_of(im)}; }
DD_FN cdd cdd_add(cdd a, cdd b) { return cdd{dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
DD_FN cdd cdd_sub(cdd a, cdd b) { return cdd{dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
DD_FN cdd cdd_mul(cdd a, cdd b) {
  return cdd{dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}
// c + a b
DD_FN cdd cdd_fma(cdd a, cdd b, cdd c) { return cdd_add(c, cdd_mul(a, b)); }
// a b for a complex float b
DD_FN cdd cdd_mul_cf(cdd a, float bre, float bim) {
  return cdd{dd_sub(dd_mul_f(a.re, bre), dd_mul_f(a.im, bim)), dd_add(dd_mul_f(a.re, bim), dd_mul_f(a.im, bre))};
}
DD_FN dd cdd_abs2(cdd a) { return dd_add(dd_mul(a.re, a.re), dd_mul(a.im, a.im)); }

}  // namespace pngf
