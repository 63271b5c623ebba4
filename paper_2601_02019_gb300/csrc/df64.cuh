// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  On this
// part FP64 throughput is a small fraction of FP32 throughput, so the
// eigensolver's O(n^3) loops run in df64 on the FP32 pipes.
//
// The building blocks are the error-free transformations: Knuth's TwoSum
// (s + e = a + b exactly), Dekker's FastTwoSum (the same when |a| >= |b|) and
// the FMA form of Dekker's TwoProduct (p + e = a * b exactly).  Sums and
// products are then formed as in the double-double literature (Dekker 1971;
// Hida, Li and Bailey 2001): the high parts through an error-free step, the
// low-order terms gathered in plain FP32, one renormalisation at the end.
#pragma once

#include <cuda_runtime.h>

namespace as {

struct df64 {
  float hi, lo;
};

__device__ __forceinline__ df64 df_make(float hi, float lo) { return df64{hi, lo}; }

// s + e = a + b exactly (any a, b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| (or a = 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// p + e = a * b exactly (FMA computes the rounding error of the product).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df64 df_renorm(float s, float e) {
  df64 r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// Conversions.  from_double: hi = fl32(x), lo = fl32(x - hi).
__device__ __forceinline__ df64 df_from_double(double x) {
  const float hi = (float)x;
  const float lo = (float)(x - (double)hi);
  return df64{hi, lo};
}
__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df64 df_neg(df64 a) { return df64{-a.hi, -a.lo}; }

// a + b
__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_renorm(s, e);
}

// a - b
__device__ __forceinline__ df64 df_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }

// a * b
__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_renorm(p, e);
}

// c + a * b with one renormalisation.
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  float s, f;
  two_sum(c.hi, p, s, f);
  f = __fadd_rn(f, e);
  f = __fmaf_rn(a.hi, b.lo, f);
  f = __fmaf_rn(a.lo, b.hi, f);
  f = __fadd_rn(f, c.lo);
  return df_renorm(s, f);
}

// One step of a compensated dot product of df64 vectors (the scheme of Ogita,
// Rump and Oishi's Dot2, extended by the cross terms of the low parts): the
// running value is s + e, where s is the FP32 sum of the high-part products
// (each added through TwoSum) and e gathers the TwoProduct and TwoSum errors
// and a.hi b.lo + a.lo b.hi.  Only the two adds into s and e carry over to
// the next step; df_dot_finish renormalises at the end.
__device__ __forceinline__ void df_dot_step(df64 a, df64 b, float& s, float& e) {
  float p, pe;
  two_prod(a.hi, b.hi, p, pe);
  float t, te;
  two_sum(s, p, t, te);
  s = t;
  e = __fadd_rn(e, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fadd_rn(te, pe))));
}
__device__ __forceinline__ df64 df_dot_finish(float s, float e) {
  float hi, lo;
  two_sum(s, e, hi, lo);
  return df64{hi, lo};
}

// a - (u * v + w * z): the two-sided rank-2 update of one matrix entry.
__device__ __forceinline__ df64 df_rank2(df64 a, df64 u, df64 v, df64 w, df64 z) {
  float p1, e1, p2, e2;
  two_prod(u.hi, v.hi, p1, e1);
  two_prod(w.hi, z.hi, p2, e2);
  float s, f1, s2, f2;
  two_sum(a.hi, -p1, s, f1);
  two_sum(s, -p2, s2, f2);
  float lo = __fsub_rn(a.lo, __fadd_rn(e1, e2));
  lo = __fadd_rn(lo, __fadd_rn(f1, f2));
  lo = __fmaf_rn(-u.hi, v.lo, lo);
  lo = __fmaf_rn(-u.lo, v.hi, lo);
  lo = __fmaf_rn(-w.hi, z.lo, lo);
  lo = __fmaf_rn(-w.lo, z.hi, lo);
  return df_renorm(s2, lo);
}

// a / b (one correction step of the FP32 quotient).
__device__ __forceinline__ df64 df_div(df64 a, df64 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  // r = a - q1 * b, exactly enough for the correction
  float p, e;
  two_prod(q1, b.hi, p, e);
  float s, f;
  two_sum(a.hi, -p, s, f);
  f = __fsub_rn(f, e);
  f = __fadd_rn(f, a.lo);
  f = __fmaf_rn(-q1, b.lo, f);
  const float r = __fadd_rn(s, f);
  const float q2 = __fdiv_rn(r, b.hi);
  return df_renorm(q1, q2);
}

// sqrt(a) for a >= 0: the FP32 root and one Newton correction
// (a - r^2) / (2 r), with r^2 formed exactly.
__device__ __forceinline__ df64 df_sqrt(df64 a) {
  if (!(a.hi > 0.f)) return df64{0.f, 0.f};
  const float r = sqrtf(a.hi);
  float p, e;
  two_prod(r, r, p, e);
  float s, f;
  two_sum(a.hi, -p, s, f);
  f = __fsub_rn(f, e);
  f = __fadd_rn(f, a.lo);
  const float corr = __fdiv_rn(__fadd_rn(s, f), __fmul_rn(2.f, r));
  return df_renorm(r, corr);
}

// 1 / sqrt(a) for a > 0 without a division.  a is first scaled by an exact
// power of two, a = a' 2^(2k) with a' in [1/2, 2), so that no intermediate
// leaves the FP32 range (the scale comes from the exponent bits, with
// frexpf/ldexpf only for a subnormal or huge a.hi).  Then the FP32 estimate r0 = rsqrtf(a'.hi) (relative
// error below 2^-21) is refined by the binomial series of (1 - h)^(-1/2),
// with h = 1 - a' r0^2 formed in df64:
//   1/sqrt(a') = r0 (1 + h/2 + 3h^2/8 + O(h^3)),
// one step of the third-order Newton-Householder iteration for the
// reciprocal square root.  The correction is small, so FP32 suffices for it;
// the result carries about 46 significant bits.
__device__ __forceinline__ df64 df_rsqrt(df64 a) {
  if (!(a.hi > 0.f)) return df64{0.f, 0.f};
  // the exponent from the bits (a normal a.hi; otherwise frexpf/ldexpf)
  const int eb = (__float_as_int(a.hi) >> 23) & 0xff;
  const int k = (eb - 126) >> 1;   // floor(ex / 2) for a.hi = m 2^ex, m in [1/2, 1)
  const bool fast = eb >= 1 && eb <= 254 && 127 - 2 * k >= 1 && 127 - 2 * k <= 254;
  df64 as;
  if (fast) {
    const float sc = __int_as_float((127 - 2 * k) << 23);   // 2^-2k, exact
    as = df64{a.hi * sc, a.lo * sc};
  } else {
    int ex;
    (void)frexpf(a.hi, &ex);
    const int kk = ex >> 1;
    as = df64{ldexpf(a.hi, -2 * kk), ldexpf(a.lo, -2 * kk)};
    const float r0s = rsqrtf(as.hi);
    float p, e;
    two_prod(r0s, r0s, p, e);
    const df64 h = df_sub(df64{1.f, 0.f}, df_mul(as, df64{p, e}));
    const float hh = __fadd_rn(h.hi, h.lo);
    const df64 r = df_renorm(r0s, __fmul_rn(r0s, __fmaf_rn(0.375f * hh, hh, 0.5f * hh)));
    return df64{ldexpf(r.hi, -kk), ldexpf(r.lo, -kk)};
  }
  const float r0 = rsqrtf(as.hi);
  float p, e;
  two_prod(r0, r0, p, e);    // r0^2 = p + e exactly
  const df64 t = df_mul(as, df64{p, e});
  const df64 h = df_sub(df64{1.f, 0.f}, t);
  const float hh = __fadd_rn(h.hi, h.lo);
  const float corr = __fmul_rn(r0, __fmaf_rn(0.375f * hh, hh, 0.5f * hh));
  const df64 r = df_renorm(r0, corr);
  const float sk = __int_as_float((127 - k) << 23);   // 2^-k, exact (127 - k in [64, 190])
  return df64{r.hi * sk, r.lo * sk};
}

}  // namespace as
