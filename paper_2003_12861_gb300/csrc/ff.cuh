// Float-float ("double-float") arithmetic and elementary functions on the
// FP32 pipe.  On GB300 an FP64 operation costs about 58 FP32 operations of
// issue throughput, so a value carried as an unevaluated sum hi + lo of two
// floats (~48 significant bits) and the error-free transformations of
// Knuth (two-sum), Dekker (fast two-sum) and the FMA two-product are far
// cheaper than FP64 while accurate to a few 1e-15 relative.
//
// Elementary functions (tables in ff_tables.h, generated from the
// mathematics by gen_ff_tables.py):
//   ff_exp  Tang's table-driven exponential (ACM TOMS 1989): x = k ln2/256 + r,
//           exp(x) = 2^(k>>8) 2^((k&255)/256) (1 + r + r^2/2 + r^3/6 + r^4/24).
//   ff_log  Tang's table-driven logarithm (ACM TOMS 1990): x = 2^e m with
//           m in [sqrt2/2, sqrt2), m = F (1 + r), F = 1 + j/256, log1p(r) to r^5.
//   ff_rcp  one Newton step from the hardware reciprocal estimate.
//   ff_erfcx exp(y^2) erfc(y), y >= 0: piecewise Chebyshev interpolants.
// Each function sets ok = false when its argument or result leaves the
// range in which the pair keeps its precision; callers then take an FP64
// path.  Plain float operations below use the _rn intrinsics wherever an
// error-free transformation must not be contracted into an FMA.
#pragma once

#include <cuda_runtime.h>

#include "ff_tables.h"

namespace rf {

struct ff {
  float hi, lo;
};

// Shared-memory copy of the tables (filled by ff_load_tables), the layout
// of kFFTablesFlat: 514-entry tables padded to 516, the six erfcx pieces'
// per-piece values to 8.
struct __align__(16) FFTables {
  float exp_tab[512];
  float log_tab[516];
  float invf_tab[516];
  float erfcx[6 * 17 * 2];
  float erfcx_mid[8], erfcx_ihalf[8];
  float erfcx_kf[8];  // small integers
};
static_assert(sizeof(FFTables) == sizeof(kFFTablesFlat), "table layout");

// Every 16-byte load is issued before the first store, so staging costs one
// memory round trip (blocks of at least 111 threads; smaller ones loop).
__device__ __forceinline__ void ff_load_tables(FFTables& t) {
  constexpr int kN4 = (int)(sizeof(FFTables) / 16), kPer = 4;
  const uint4* src = reinterpret_cast<const uint4*>(kFFTablesFlat);
  uint4* dst = reinterpret_cast<uint4*>(&t);
  const int nt = blockDim.x;
  uint4 r[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = threadIdx.x + j * nt;
    if (i < kN4) r[j] = __ldg(src + i);
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = threadIdx.x + j * nt;
    if (i < kN4) dst[i] = r[j];
  }
  for (int i = threadIdx.x + kPer * nt; i < kN4; i += nt) dst[i] = __ldg(src + i);
}

__device__ __forceinline__ ff ff_from_double(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// ---------------------------------------------------- error-free transforms
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b| (or a == 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// ------------------------------------------------------------- arithmetic
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
// The product without the final renormalisation: |lo| may reach 2^-22 |hi|
// instead of 2^-24.  Such a pair is as accurate as an operand of ff_mul,
// ff_acc and ff_acc_mul; other functions take normalised pairs.
__device__ __forceinline__ ff ff_mul_u(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return p;
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// a b + c with one renormalisation: the product's error terms join the
// sum's low word (the accuracy of ff_add(ff_mul(a, b), c), three fewer
// operations).
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) {
  const ff p = two_prod(a.hi, b.hi);
  const ff s = two_sum(p.hi, c.hi);
  float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  lo = __fadd_rn(lo, __fadd_rn(c.lo, s.lo));
  return fast_two_sum(s.hi, lo);
}
// ff_fma without the final renormalisation, for an argument of the
// exponential only: its reduction adds the low word by an exact two-sum, so
// a low word that cancellation has left as large as the high word costs
// nothing.  (A product would see that low word rounded to a float.)
__device__ __forceinline__ ff ff_fma_u(ff a, ff b, ff c) {
  const ff p = two_prod(a.hi, b.hi);
  const ff s = two_sum(p.hi, c.hi);
  const float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return {s.hi, __fadd_rn(lo, __fadd_rn(c.lo, s.lo))};
}
__device__ __forceinline__ ff ff_sqr(ff a) {
  ff p = two_prod(a.hi, a.hi);
  p.lo = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_scale(ff a, float pow2) { return {__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)}; }

// Running sum without renormalisation per step: hi accumulates through an
// exact two-sum, lo collects the errors and the addends' low parts.
__device__ __forceinline__ void ff_acc(ff& acc, ff x) {
  const ff s = two_sum(acc.hi, x.hi);
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, x.lo));
  acc.hi = s.hi;
}

// acc += a b: the product's hi word through the exact two-sum, its error
// terms into the low word.
__device__ __forceinline__ void ff_acc_mul(ff& acc, ff a, ff b) {
  const ff p = two_prod(a.hi, b.hi);
  const ff s = two_sum(acc.hi, p.hi);
  const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
  acc.hi = s.hi;
}

// Variants with one operand a plain float (an FP32 observable: its low word
// is zero, known at compile time).  Each gives the result of the pair
// variant with {b, 0}, with the product or sum terms of the zero word left
// out.
__device__ __forceinline__ float ff_neg(float a) { return -a; }
__device__ __forceinline__ float ff_hi(float a) { return a; }
__device__ __forceinline__ float ff_hi(ff a) { return a.hi; }
__device__ __forceinline__ ff ff_sub(float a, ff b) {
  ff s = two_sum(a, -b.hi);
  s.lo = __fsub_rn(s.lo, b.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_mul_u(ff a, float b) {
  ff p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return p;
}
__device__ __forceinline__ ff ff_fma(ff a, float b, ff c) {
  const ff p = two_prod(a.hi, b);
  const ff s = two_sum(p.hi, c.hi);
  float lo = __fmaf_rn(a.lo, b, p.lo);
  lo = __fadd_rn(lo, __fadd_rn(c.lo, s.lo));
  return fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ ff ff_fma(float a, ff b, ff c) { return ff_fma(b, a, c); }
__device__ __forceinline__ ff ff_fma_u(ff a, float b, ff c) {
  const ff p = two_prod(a.hi, b);
  const ff s = two_sum(p.hi, c.hi);
  const float lo = __fmaf_rn(a.lo, b, p.lo);
  return {s.hi, __fadd_rn(lo, __fadd_rn(c.lo, s.lo))};
}
__device__ __forceinline__ ff ff_fma_u(float a, ff b, ff c) { return ff_fma_u(b, a, c); }
__device__ __forceinline__ void ff_acc_mul(ff& acc, ff a, float b) {
  const ff p = two_prod(a.hi, b);
  const ff s = two_sum(acc.hi, p.hi);
  const float e = __fmaf_rn(a.lo, b, p.lo);
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
  acc.hi = s.hi;
}

// ---------------------------------------------------------------- exp
// The reduction and reconstruction for an integer kk = k = rint(x 256/ln2)
// whose 2^(k >> 8) scale is a normal float.
__device__ __forceinline__ ff ff_exp_k(const FFTables& T, ff x, int k, float kk) {
  // r = x - k ln2/256, the large cancellation exact
  const float t1 = __fmaf_rn(-kk, kLn2_256_1, x.hi);
  const ff p2 = two_prod(kk, kLn2_256_2);
  const ff s = two_sum(t1, -p2.hi);
  const ff s2 = two_sum(s.hi, x.lo);  // the input's low word can exceed |r| * 2^-24
  float lo = __fadd_rn(s.lo, s2.lo);
  lo = __fsub_rn(lo, p2.lo);
  lo = __fmaf_rn(-kk, kLn2_256_3, lo);
  const ff r = fast_two_sum(s2.hi, lo);
  // exp(r) - 1 = r + r^2/2 + r^3/6 + r^4/24, |r| <= ln2/512
  ff sq = two_prod(r.hi, r.hi);
  sq.lo = __fmaf_rn(__fmul_rn(2.0f, r.hi), r.lo, sq.lo);
  const float q = __fmul_rn(__fmul_rn(r.hi, sq.hi), __fmaf_rn(r.hi, 1.0f / 24.0f, 1.0f / 6.0f));
  ff pp = fast_two_sum(r.hi, __fmul_rn(0.5f, sq.hi));
  pp.lo = __fadd_rn(pp.lo, __fadd_rn(r.lo, __fmaf_rn(0.5f, sq.lo, q)));
  // 2^(j/256) (1 + p)
  const int j = k & 255, m = k >> 8;
  const ff t = {T.exp_tab[2 * j], T.exp_tab[2 * j + 1]};
  ff tp = two_prod(t.hi, pp.hi);
  tp.lo = __fmaf_rn(t.hi, pp.lo, __fmaf_rn(t.lo, pp.hi, tp.lo));
  ff res = fast_two_sum(t.hi, tp.hi);
  res.lo = __fadd_rn(res.lo, __fadd_rn(t.lo, tp.lo));
  res = fast_two_sum(res.hi, res.lo);
  return ff_scale(res, __int_as_float((m + 127) << 23));
}

__device__ __forceinline__ ff ff_exp(const FFTables& T, ff x, bool& ok) {
  const float kf = rintf(__fmul_rn(x.hi, kExpK));
  ok = ok && fabsf(x.hi) < 80.0f;
  const int k = ok ? (int)kf : 0;
  ok = ok && (k >> 8) >= -100 && (k >> 8) <= 100;
  return ff_exp_k(T, x, ok ? k : 0, ok ? kf : 0.0f);
}

// exp for |x.hi| <= 69, which the caller has checked: |k| <= 25484, so
// 2^(k >> 8) is within 2^+-100 and no further range test is needed.
__device__ __forceinline__ ff ff_exp_in_range(const FFTables& T, ff x) {
  const float kf = rintf(__fmul_rn(x.hi, kExpK));
  return ff_exp_k(T, x, (int)kf, kf);
}

// ---------------------------------------------------------------- log
__device__ __forceinline__ ff ff_log(const FFTables& T, ff a, bool& ok) {
  ok = ok && a.hi > 7.9e-31f && a.hi < 1.2e30f;  // 2^-100 .. 2^100
  const float ah = ok ? a.hi : 1.0f, al = ok ? a.lo : 0.0f;
  const int bits = __float_as_int(ah);
  int e = ((bits >> 23) & 0xff) - 127;
  float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);
  float ml = __fmul_rn(al, __int_as_float((127 - e) << 23));
  if (m > 1.41421356f) {  // m in [sqrt2/2, sqrt2): no cancellation of e ln2 against log F near 1
    m = __fmul_rn(m, 0.5f);
    ml = __fmul_rn(ml, 0.5f);
    e += 1;
  }
  const int j = __float2int_rn(__fmul_rn(__fsub_rn(m, 1.0f), 256.0f));  // -75 .. 106
  const float F = __fmaf_rn((float)j, 1.0f / 256.0f, 1.0f);
  const ff f = two_sum(__fsub_rn(m, F), ml);
  const int jt = j + 128;
  const ff iF = {T.invf_tab[2 * jt], T.invf_tab[2 * jt + 1]};
  const ff r = ff_mul(f, iF);
  // log1p(r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5, |r| <= 1/362
  ff sq = two_prod(r.hi, r.hi);
  sq.lo = __fmaf_rn(__fmul_rn(2.0f, r.hi), r.lo, sq.lo);
  const float q = __fmul_rn(__fmul_rn(r.hi, sq.hi),
                            __fmaf_rn(r.hi, __fmaf_rn(r.hi, 0.2f, -0.25f), 1.0f / 3.0f));
  ff lp = fast_two_sum(r.hi, __fmul_rn(-0.5f, sq.hi));
  lp.lo = __fadd_rn(lp.lo, __fadd_rn(r.lo, __fmaf_rn(-0.5f, sq.lo, q)));
  // + e ln2 + log F
  const float ef = (float)e;
  const ff lf = {T.log_tab[2 * jt], T.log_tab[2 * jt + 1]};
  const ff e2 = two_prod(ef, kLn2_2);
  ff s = two_sum(__fmul_rn(ef, kLn2_1), lf.hi);  // e*ln2_1 exact (16-bit constant)
  s.lo = __fadd_rn(s.lo, __fadd_rn(lf.lo, __fmaf_rn(ef, kLn2_3, e2.lo)));
  ff s2 = two_sum(s.hi, e2.hi);
  s2.lo = __fadd_rn(s2.lo, s.lo);
  s2 = fast_two_sum(s2.hi, s2.lo);
  ff out = two_sum(s2.hi, lp.hi);
  out.lo = __fadd_rn(out.lo, __fadd_rn(s2.lo, lp.lo));
  return fast_two_sum(out.hi, out.lo);
}

// ------------------------------------------------------- log of a product
// A running product m 2^e of positive float-float factors, m kept in
// [1, 2) by exact power-of-two scaling: sum_i log p_i = log(prod_i p_i)
// costs one logarithm per product instead of one per factor.
struct LogProd {
  ff m;
  int e;
};
__device__ __forceinline__ LogProd logprod_init() { return {{1.0f, 0.0f}, 0}; }
// p in [2^-100, 2^100] (the caller checks); m is kept unnormalised.
__device__ __forceinline__ void logprod_mul(LogProd& L, ff p) {
  const ff m = ff_mul_u(L.m, p);
  const int ex = ((__float_as_int(m.hi) >> 23) & 0xff) - 127;
  const float sc = __int_as_float((127 - ex) << 23);  // 2^-ex, exact
  L.m = {__fmul_rn(m.hi, sc), __fmul_rn(m.lo, sc)};
  L.e += ex;
}
// log(m 2^e) = log(m) + e ln2, |e| < 2^12.
__device__ __forceinline__ ff logprod_log(const FFTables& T, const LogProd& L, bool& ok) {
  const ff lm = ff_log(T, fast_two_sum(L.m.hi, L.m.lo), ok);
  const float ef = (float)L.e;
  const ff e2 = two_prod(ef, kLn2e_2);
  ff s = two_sum(__fmul_rn(ef, kLn2e_1), e2.hi);  // e ln2_1 exact (12-bit constant)
  s.lo = __fadd_rn(s.lo, __fmaf_rn(ef, kLn2e_3, e2.lo));
  return ff_add(fast_two_sum(s.hi, s.lo), lm);
}

// ---------------------------------------------------------------- rcp
// y0 (1 + e) with e = 1 - a y0, unnormalised (see ff_mul_u)
__device__ __forceinline__ ff ff_rcp_u(ff a) {
  float y0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(a.hi));
  const ff p = two_prod(a.hi, y0);
  float e = __fsub_rn(1.0f, p.hi);
  e = __fsub_rn(e, p.lo);
  e = __fmaf_rn(-a.lo, y0, e);
  return {y0, __fmul_rn(y0, e)};
}
__device__ __forceinline__ ff ff_rcp(ff a) {
  const ff r = ff_rcp_u(a);
  return fast_two_sum(r.hi, r.lo);
}

// -------------------------------------------------------------- erfcx
// y >= 0.  Pieces 0-2: y in [0,0.5), [0.5,1), [1,2); pieces 3-5: w = 1/y in
// (0.25,0.5], (0.125,0.25], [0,0.125] with erfcx(y) = w h(w).
__device__ __forceinline__ ff ff_erfcx(const FFTables& T, ff y, bool& ok) {
  ok = ok && y.hi >= 0.0f && y.hi < 1e30f;
  int piece;
  ff v;
  if (y.hi < 2.0f) {
    piece = y.hi < 0.5f ? 0 : (y.hi < 1.0f ? 1 : 2);
    v = y;
  } else {
    v = ff_rcp(y);
    piece = v.hi > 0.25f ? 3 : (v.hi > 0.125f ? 4 : 5);
  }
  // x = (v - mid) / half, exact scaling by a power of two
  const ff x = ff_scale(ff_add_f(v, -T.erfcx_mid[piece]), T.erfcx_ihalf[piece]);
  const float* c = T.erfcx + piece * 34;
  const int kf = (int)T.erfcx_kf[piece];  // 1 <= kf <= 16: tail a_16..a_kf in float
  float s = c[2 * 16];
  for (int k = 15; k >= kf; --k) s = __fmaf_rn(s, x.hi, c[2 * k]);
  ff acc = {s, 0.0f};
  for (int k = kf - 1; k >= 0; --k) acc = ff_fma(acc, x, ff{c[2 * k], c[2 * k + 1]});
  return piece >= 3 ? ff_mul(acc, v) : acc;
}

}  // namespace rf
