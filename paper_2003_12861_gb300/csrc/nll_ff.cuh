// Float-float event programs of the graph shapes the library specialises.
//
// The event pass is the hot loop of the likelihood (Sec. 4: every
// observable-dependent node is recomputed for every event).  For the shapes
// below the whole per-event program runs in float-float arithmetic (ff.cuh)
// on the FP32 pipe.  The gradient is not accumulated per parameter: every
// parameter derivative of log p_i is a linear combination, with
// parameter-point constants, of a few per-event moments (1/p_i, t_i/p_i,
// e_i/p_i, ...), so the kernel sums the moments and one matrix K per set maps
// the summed moments to (sum log p, d/dtheta_slot) at the end of each chunk.
// K and the per-event constants are computed in FP64 once per parameter point.
//
// (PROD3's moment 13 is the count of events the pass summed, not a moment.)
// Shapes (program order = the topological order of rf_model_create):
//   DECAY     SUM(GAUSSEXP(t; tau,mu,sigma), CHEB2(t; c1,c2); f)      Q = 7
//   GP1       SUM(GAUSS(x; mu,sigma), POLY1(x; a1); f)                 Q = 5
//   PROD3     PROD(SUM(GAUSS(m), CHEB1(m); fm), DECAY(t), POLY2(c))    Q = 13
#pragma once

#include "ff.cuh"
#include "nll_kernels.cuh"

namespace rf {

constexpr int kFFConst = 512;  // floats per set: per-event constants, then K (Q x NACC pairs)
// Below this z the resolution term of the decay is dropped: erfc(z) = 2 -
// erfc(-z) with erfc(5.5) / 2 < 4e-15 (below the float-float precision of
// the other terms) and the derivative ratio carries exp(-z^2) < 8e-14, far
// below the gradient tolerance.
constexpr float kSlowZf = -5.5f;

// Number of moment accumulators (index 0 = log p) and of output quantities.
__host__ __device__ constexpr int ff_nacc(int shape) {
  return shape == SHAPE_SUM_GAUSSEXP_CHEB2 ? 8 : shape == SHAPE_SUM_GAUSS_POLY1 ? 6 : shape == SHAPE_PROD3 ? 16 : 0;
}
__host__ __device__ constexpr int ff_q(int shape) {
  return shape == SHAPE_SUM_GAUSSEXP_CHEB2 ? 7 : shape == SHAPE_SUM_GAUSS_POLY1 ? 5 : shape == SHAPE_PROD3 ? 13 : 0;
}
// Offset of K in the set's float block, after the per-event constants.
__host__ __device__ constexpr int ff_koff(int shape) {
  return shape == SHAPE_SUM_GAUSSEXP_CHEB2 ? 24 : shape == SHAPE_SUM_GAUSS_POLY1 ? 16 : shape == SHAPE_PROD3 ? 44 : 0;
}

// ------------------------------------------------ parameter-point side (FP64)

// A double observable as a float pair, from its bits (no FP64 instruction):
// hi = the top 24 significand bits, lo = the remaining 29 rounded to a float.
// ok = false for values the pair cannot hold (|d| < 2^-74 except 0, >= 2^128).
__device__ __forceinline__ ff ff_split(double d, bool& ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
  const int ex = (int)((hi32 >> 20) & 0x7ffu);
  if ((b << 1) == 0ull) return {0.0f, 0.0f};
  ok = ok && ex >= 949 && ex <= 1150;
  const int exs = ok ? ex : 1023;
  const unsigned sign = hi32 & 0x80000000u;
  const unsigned m23 = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const float h = __uint_as_float(sign | ((unsigned)(exs - 896) << 23) | m23);
  const float scale = __uint_as_float(sign | ((unsigned)(exs - 948) << 23));
  const float l = __fmul_rn(__uint2float_rn(lo32 & 0x1fffffffu), scale);
  return {h, l};
}

// A parameter-point constant as a float pair at o[0], o[1].  The split
// works on the bits (integer pipe); only values outside the pair's range
// take the FP64 conversions, whose warp instructions are slow on this GPU.
__device__ __forceinline__ void put_ff(float* o, double v) {
  bool ok = true;
  const ff p = ff_split(v, ok);
  if (ok) {
    o[0] = p.hi;
    o[1] = p.lo;
    return;
  }
  const float h = __double2float_rn(v);
  o[0] = h;
  o[1] = __double2float_rn(v - (double)h);
}

// Per-event constants of a decay sub-model (22 floats at o) and its rows of K.
// ge: GAUSSEXP constants [mu, 1/sigma, s, 1/tau, 1/I, dlogI/dtau, dlogI/dmu,
// dlogI/dsigma]; ch: CHEB2 [2/(b-a), (a+b)/(b-a), 1/I, dlogI/dc1, dlogI/dc2,
// c1, c2]; sm: SUM [f, 1-f].  The kernel evaluates the normalised signal
// density v = shape/I with log(1/I) folded into the exponent, so that no
// factor leaves the float range while the product matters.  Moments at
// column m0: E = v/p, E t, 1/p, t/p, t^2/p, E R, E R u (u = (t - mu)/sigma).
// Rows r0.. for tau, mu, sigma, c1, c2, f.
// The background polynomial of CHEB2 in powers of t: S[j] t^j = 1 + c1
// T1(x') + c2 T2(x'), x' = c0 t - c1p.
__device__ __forceinline__ void cheb2_power(const double* ch, double S[3]) {
  const double c0 = ch[0], c1p = ch[1], a1 = ch[5], a2 = ch[6];
  S[0] = 1.0 - a1 * c1p + a2 * (2.0 * c1p * c1p - 1.0);
  S[1] = a1 * c0 - 4.0 * a2 * c0 * c1p;
  S[2] = 2.0 * a2 * c0 * c0;
}
// The per-event constants (job 0 of a decay sub-model).
static __device__ void prep_decay_consts(const double* ge, const double* ch, const double* sm, float* o) {
  const double mu = ge[0], is = ge[1], s = ge[2], it = ge[3], iIs = ge[4];
  const double iIb = ch[2];
  const double f = sm[0], fl = sm[1];
  const double lIs = log(iIs);
  double S[3];
  cheb2_power(ch, S);
  const double r2 = 0.70710678118654752440;
  put_ff(o + 0, 0.5 * s * s + mu * it + lIs);  // log v = A + log(1/I), A = s^2/2 + mu/tau - t/tau
  put_ff(o + 2, it);
  put_ff(o + 4, f);
  for (int j = 0; j < 3; ++j) put_ff(o + 6 + 2 * j, fl * iIb * S[j]);
  o[12] = (float)((s + mu * is) * r2);  // z ~ zc - t zs (decides the slow path only)
  o[13] = (float)(is * r2);
  put_ff(o + 14, mu);
  put_ff(o + 16, is);
  put_ff(o + 18, s);
  put_ff(o + 20, lIs);
}
// Its rows of K (job 1).
static __device__ void prep_decay_K(const double* ge, const double* ch, const double* sm, double* K, int nacc, int r0,
                                    int m0) {
  const double mu = ge[0], is = ge[1], s = ge[2], it = ge[3];
  const double dIt = ge[5], dIm = ge[6], dIs = ge[7];
  const double c0 = ch[0], c1p = ch[1], iIb = ch[2], dI1 = ch[3], dI2 = ch[4];
  const double f = sm[0], fl = sm[1];
  double S[3];
  cheb2_power(ch, S);
  const double T1[3] = {-c1p, c0, 0.0};
  const double T2[3] = {2.0 * c1p * c1p - 1.0, -4.0 * c0 * c1p, 2.0 * c0 * c0};
  const double r2 = 0.70710678118654752440;
  double* rt = K + (r0 + 0) * nacc;  // tau
  rt[m0 + 1] = f * s * is * it;
  rt[m0 + 0] = -f * (s * mu * is * it + s * s * it + dIt);
  rt[m0 + 5] = f * s * it * r2;
  double* rm = K + (r0 + 1) * nacc;  // mu
  rm[m0 + 0] = f * (it - dIm);
  rm[m0 + 5] = -f * is * r2;
  double* rs = K + (r0 + 2) * nacc;  // sigma: dz/dsigma = (1/tau + u/sigma)/sqrt2
  rs[m0 + 0] = f * (s * it - dIs);
  rs[m0 + 5] = -f * it * r2;
  rs[m0 + 6] = -f * is * r2;
  for (int j = 0; j < 3; ++j) {
    K[(r0 + 3) * nacc + m0 + 2 + j] = fl * iIb * (T1[j] - dI1 * S[j]);
    K[(r0 + 4) * nacc + m0 + 2 + j] = fl * iIb * (T2[j] - dI2 * S[j]);
    K[(r0 + 5) * nacc + m0 + 2 + j] = -iIb * S[j];
  }
  K[(r0 + 5) * nacc + m0 + 0] = 1.0;
}

// Gauss + linear background (POLY1 or CHEB1) sub-model: constants (16
// floats) and rows for mu, sigma, background coefficient, fraction.  The
// kernel evaluates the normalised Gaussian density (log(1/I) folded into the
// exponent); the moments are centred so that their combination does not
// cancel: at m0, G = v/p, G u, G u^2 (u = (x - mu)/sigma), 1/p, y/p, with
// y = c0 x - c1 the background's own variable (x for POLY1, the mapped x'
// for CHEB1), in which its shape is 1 + b y.  bg = (c0, c1, b, iIb, dIb).
static __device__ void prep_gauss_lin_consts(const double* g, const double* bg, const double* sm, float* o) {
  const double mu = g[0], is = g[1], iIg = g[2];
  const double c0 = bg[0], c1 = bg[1], b = bg[2], iIb = bg[3];
  const double f = sm[0], fl = sm[1];
  put_ff(o + 0, mu);
  put_ff(o + 2, is);
  put_ff(o + 4, f);
  put_ff(o + 6, fl * iIb);
  put_ff(o + 8, fl * iIb * b);
  put_ff(o + 10, c0);
  put_ff(o + 12, c1);
  put_ff(o + 14, log(iIg));
}
static __device__ void prep_gauss_lin_K(const double* g, const double* bg, const double* sm, double* K, int nacc,
                                        int r0, int m0) {
  const double is = g[1], dIm = g[3], dIs = g[4];
  const double b = bg[2], iIb = bg[3], dIb = bg[4];
  const double f = sm[0], fl = sm[1];
  K[(r0 + 0) * nacc + m0 + 1] = f * is;  // mu: u/sigma - dlogI/dmu
  K[(r0 + 0) * nacc + m0 + 0] = -f * dIm;
  K[(r0 + 1) * nacc + m0 + 2] = f * is;  // sigma: u^2/sigma - dlogI/dsigma
  K[(r0 + 1) * nacc + m0 + 0] = -f * dIs;
  K[(r0 + 2) * nacc + m0 + 3] = -fl * iIb * dIb;  // background: y - (1 + b y) dlogI/db
  K[(r0 + 2) * nacc + m0 + 4] = fl * iIb * (1.0 - dIb * b);
  K[(r0 + 3) * nacc + m0 + 0] = 1.0;  // fraction
  K[(r0 + 3) * nacc + m0 + 3] = -iIb;
  K[(r0 + 3) * nacc + m0 + 4] = -iIb * b;
}

// The set's float block (per-event constants, then K as float pairs) is
// written in independent jobs, so that K1 can run them on separate warps:
// ff_jobs(shape) jobs each fill their part of `out` or rows of K (a zeroed
// Q x NACC double array with K[0] = 1), then ff_convert_K writes K as float
// pairs, entry by entry.
__host__ __device__ constexpr int ff_jobs(int shape) { return shape == SHAPE_PROD3 ? 5 : 2; }

static __device__ void prepare_ff_job(const Program& P, int shape, const double* C, float* out, double* K, int job) {
  const int nacc = ff_nacc(shape);
  if (shape == SHAPE_SUM_GAUSSEXP_CHEB2) {
    const double *ge = C + P.node[0].cofs, *ch = C + P.node[1].cofs, *sm = C + P.node[2].cofs;
    if (job == 0) prep_decay_consts(ge, ch, sm, out);
    else prep_decay_K(ge, ch, sm, K, nacc, 1, 1);
  } else if (shape == SHAPE_SUM_GAUSS_POLY1) {
    const double* pl = C + P.node[1].cofs;  // POLY1 [1/I, dlogI/da1, a1]
    const double bg[5] = {1.0, 0.0, pl[2], pl[0], pl[1]};
    if (job == 0) prep_gauss_lin_consts(C + P.node[0].cofs, bg, C + P.node[2].cofs, out);
    else prep_gauss_lin_K(C + P.node[0].cofs, bg, C + P.node[2].cofs, K, nacc, 1, 1);
  } else if (shape == SHAPE_PROD3) {
    const double* cb = C + P.node[1].cofs;  // CHEB1 [c0, c1', 1/I, dlogI/dc, c]
    const double bg[5] = {cb[0], cb[1], cb[4], cb[2], cb[3]};
    const double *ge = C + P.node[3].cofs, *ch = C + P.node[4].cofs, *sm = C + P.node[5].cofs;
    const double* pa = C + P.node[6].cofs;  // POLY2 [1/I, dlogI/da1, dlogI/da2, a1, a2]
    const double Sa[3] = {1.0, pa[3], pa[4]};
    switch (job) {
      case 0: prep_gauss_lin_consts(C + P.node[0].cofs, bg, C + P.node[2].cofs, out); break;
      case 1: prep_gauss_lin_K(C + P.node[0].cofs, bg, C + P.node[2].cofs, K, nacc, 1, 1); break;
      case 2: prep_decay_consts(ge, ch, sm, out + 16); break;
      case 3: prep_decay_K(ge, ch, sm, K, nacc, 5, 6); break;
      default:
        // d log p_c / d a_k = c^k / (I p_c) - dlogI/da_k, and moment 13 is
        // the count of events (not sum 1/p_c)
        for (int j = 0; j < 3; ++j) put_ff(out + 38 + 2 * j, pa[0] * Sa[j]);
        for (int k = 0; k < 2; ++k) {
          K[(11 + k) * nacc + 13] = -pa[1 + k];
          K[(11 + k) * nacc + 13 + 1 + k] = pa[0];
        }
    }
  }
}

// K entries [i0, end) with stride, as float pairs after the constants.
static __device__ void ff_convert_K(int shape, const double* K, float* out, int i0, int stride) {
  float* Ko = out + ff_koff(shape);
  for (int i = i0; i < ff_q(shape) * ff_nacc(shape); i += stride) put_ff(Ko + 2 * i, K[i]);
}

// All jobs in turn (one thread).
static __device__ void prepare_ff(const Program& P, int shape, const double* C, float* out) {
  double K[13 * 16];
  const int nacc = ff_nacc(shape), Q = ff_q(shape);
  for (int i = 0; i < Q * nacc; ++i) K[i] = 0.0;
  K[0] = 1.0;  // sum log p
  for (int j = 0; j < ff_jobs(shape); ++j) prepare_ff_job(P, shape, C, out, K, j);
  ff_convert_K(shape, K, out, 0, 1);
}

// ----------------------------------------------------- event side (FF)

__device__ __forceinline__ ff ld_ff(const Columns& cols, int c, int64_t e, bool& ok) {
  if (cols.is_f32[c]) return {__ldg((const float*)cols.ptr[c] + e), 0.0f};
  return ff_split(__ldg((const double*)cols.ptr[c] + e), ok);
}

__device__ __forceinline__ ff ldc(const float* k, int i) { return {k[i], k[i + 1]}; }

// exp, with arguments below -69 giving 0 and setting `dropped`: such a term
// (a normalised density below 1e-30) is negligible when the event's total
// density is at least 1e-14, which the caller then checks.  Arguments above
// 69 (or NaN) clear ok.
__device__ __forceinline__ ff ff_exp0(const FFTables& T, ff x, bool& ok, bool& dropped) {
  if (x.hi < -69.0f) {
    dropped = true;
    return {0.0f, 0.0f};
  }
  if (!(x.hi <= 69.0f)) {
    ok = false;
    return {1.0f, 0.0f};
  }
  return ff_exp_in_range(T, x);
}

// Normalised decay signal density v and the derivative ratio R at t (the
// constants fold log(1/I) into every exponent).  Fast path (z < -5.5):
// v = exp(A)/I, R = 0.  Otherwise the resolution region:
// z >= 0: v = exp(-u^2/2) erfcx(z) / (2I), R = 2 / (sqrt(pi) erfcx(z));
// z < 0:  v = exp(A)/I - exp(-u^2/2) erfcx(|z|) / (2I),
//         R = 2 q / (sqrt(pi) (2 - q erfcx(|z|))), q = exp(-z^2).
template <bool kSlow, class OT>
__device__ __forceinline__ ff decay_shape(const FFTables& T, const float* k, OT t, ff* R, ff* uo, bool& ok,
                                          bool& dropped) {
  const ff logv = ff_fma_u(ff_neg(t), ldc(k, 2), ldc(k, 0));
  if (!kSlow) {
    *R = {0.0f, 0.0f};
    return ff_exp0(T, logv, ok, dropped);
  }
  const ff u = ff_mul(ff_sub(t, ldc(k, 14)), ldc(k, 16));
  *uo = u;
  const ff z = ff_mul(ff_sub(ldc(k, 18), u), ff{kSqrt1_2_hi, kSqrt1_2_lo});
  const bool neg = z.hi < 0.0f;
  const ff y = neg ? ff_neg(z) : z;
  const ff ex = ff_erfcx(T, y, ok);
  const ff G = ff_exp0(T, ff_fma_u(ff_scale(u, -0.5f), u, ldc(k, 20)), ok, dropped);
  const ff half_g_ex = ff_scale(ff_mul_u(G, ex), 0.5f);
  const ff two_over_sqrtpi = {kTwoInvSqrtPi_hi, kTwoInvSqrtPi_lo};
  if (!neg) {
    *R = ff_mul_u(two_over_sqrtpi, ff_rcp_u(ex));
    return half_g_ex;
  }
  const ff ev = ff_exp0(T, logv, ok, dropped);
  // q = exp(-z^2) = G / exp(logv): both exponents carry log(1/I), and
  // A - z^2 = -u^2/2 (one reciprocal instead of an exponential; q only
  // scales R)
  ff q;
  if (G.hi > 0.0f && ev.hi > 0.0f) {
    q = ff_mul_u(G, ff_rcp_u(ev));
  } else {
    bool dq = false;
    q = ff_exp0(T, ff_neg(ff_sqr(z)), ok, dq);
  }
  *R = ff_mul_u(ff_mul_u(two_over_sqrtpi, q), ff_rcp_u(ff_fma(ff_neg(q), ex, ff{2.0f, 0.0f})));
  return ff_sub(ev, half_g_ex);
}

// Per-shape event programs.  Each adds the event's moments to acc and
// returns 0, or returns 1 (needs the decay slow path) / 2 (outside the
// float-float range: take the FP64 fallback) without touching acc.
// The event's observables, split to float-float: x[0] (DECAY, GP1) or
// (m, t, c) (PROD3); ok is false if one is outside the float-float range.
template <int kShape>
struct FFIn {
  ff x[kShape == SHAPE_PROD3 ? 3 : 1];
  bool ok;
};
// The raw bits of an event's observables (a double, or a float in the low
// word), loaded ahead of use; ff_split_in converts them when needed, so a
// prefetch does not make the warp wait for its load early.  kF32: every
// column of the dataset is FP32 (known at compile time: no per-event dtype
// test, and the observables' low words are zero).
template <int kShape>
struct FFRaw {
  unsigned long long b[kShape == SHAPE_PROD3 ? 3 : 1];
};
template <bool kF32>
__device__ __forceinline__ unsigned long long ld_raw(const Columns& cols, int c, int64_t e) {
  if (kF32 || cols.is_f32[c]) return (unsigned long long)__float_as_uint(__ldg((const float*)cols.ptr[c] + e));
  return (unsigned long long)__double_as_longlong(__ldg((const double*)cols.ptr[c] + e));
}
template <bool kF32>
__device__ __forceinline__ ff split_raw(const Columns& cols, int c, unsigned long long b, bool& ok) {
  if (kF32 || cols.is_f32[c]) return {__uint_as_float((unsigned)b), 0.0f};
  return ff_split(__longlong_as_double((long long)b), ok);
}
template <int kShape, bool kF32>
__device__ __forceinline__ FFRaw<kShape> ff_load_raw(const Columns& cols, const int* col, int64_t e) {
  FFRaw<kShape> r;
  r.b[0] = ld_raw<kF32>(cols, col[0], e);
  if constexpr (kShape == SHAPE_PROD3) {
    r.b[1] = ld_raw<kF32>(cols, col[1], e);
    r.b[2] = ld_raw<kF32>(cols, col[2], e);
  }
  return r;
}
template <int kShape, bool kF32>
__device__ __forceinline__ FFIn<kShape> ff_split_in(const Columns& cols, const int* col, const FFRaw<kShape>& r) {
  FFIn<kShape> in;
  in.ok = true;
  in.x[0] = split_raw<kF32>(cols, col[0], r.b[0], in.ok);
  if constexpr (kShape == SHAPE_PROD3) {
    in.x[1] = split_raw<kF32>(cols, col[1], r.b[1], in.ok);
    in.x[2] = split_raw<kF32>(cols, col[2], r.b[2], in.ok);
  }
  return in;
}
template <int kShape, bool kF32>
__device__ __forceinline__ FFIn<kShape> ff_load(const Columns& cols, const int* col, int64_t e) {
  return ff_split_in<kShape, kF32>(cols, col, ff_load_raw<kShape, kF32>(cols, col, e));
}

// An observable as the program uses it: a plain float for an all-FP32
// dataset (kF32), else the pair.
template <bool kF32>
__device__ __forceinline__ auto obs_value(ff x) {
  if constexpr (kF32) return x.hi;
  else return x;
}

// p_i goes into the lane's running product L (its log is taken once per
// part: sum log p_i = log prod p_i); the moments into acc[1..].
template <int kShape, bool kGrad, bool kSlow, bool kF32 = false>
__device__ __forceinline__ int ff_event(const FFTables& T, const float* k, const FFIn<kShape>& in, ff* acc,
                                        LogProd& L) {
  bool ok = in.ok, dropped = false;
  if constexpr (kShape == SHAPE_SUM_GAUSSEXP_CHEB2) {
    const auto t = obs_value<kF32>(in.x[0]);
    if (!kSlow && __fmaf_rn(-ff_hi(t), k[13], k[12]) >= kSlowZf) return ok ? 1 : 2;
    ff R, u;
    const ff vs = decay_shape<kSlow>(T, k, t, &R, &u, ok, dropped);
    const ff pb = ff_fma(ff_fma(ldc(k, 10), t, ldc(k, 8)), t, ldc(k, 6));
    const ff p = ff_fma(ldc(k, 4), vs, pb);
    ok = ok && p.hi > 7.9e-31f && p.hi < 1.2e30f;  // 2^-100 .. 2^100
    if (!ok || (dropped && p.hi < 1e-14f)) return 2;
    logprod_mul(L, p);
    if constexpr (kGrad) {
      const ff ip = ff_rcp_u(p);
      const ff E = ff_mul_u(vs, ip);
      const ff ipt = ff_mul_u(ip, t);
      ff_acc(acc[1], E);
      ff_acc_mul(acc[2], E, t);
      ff_acc(acc[3], ip);
      ff_acc(acc[4], ipt);
      ff_acc_mul(acc[5], ipt, t);
      if (kSlow) {
        const ff ER = ff_mul_u(E, R);
        ff_acc(acc[6], ER);
        ff_acc_mul(acc[7], ER, u);
      }
    }
    return 0;
  } else if constexpr (kShape == SHAPE_SUM_GAUSS_POLY1) {
    const auto x = obs_value<kF32>(in.x[0]);
    const ff u = ff_mul(ff_sub(x, ldc(k, 0)), ldc(k, 2));
    const ff g = ff_exp0(T, ff_fma_u(ff_scale(u, -0.5f), u, ldc(k, 14)), ok, dropped);
    const ff p = ff_fma(ldc(k, 4), g, ff_fma(ldc(k, 8), x, ldc(k, 6)));
    ok = ok && p.hi > 7.9e-31f && p.hi < 1.2e30f;
    if (!ok || (dropped && p.hi < 1e-14f)) return 2;
    logprod_mul(L, p);
    if constexpr (kGrad) {
      const ff ip = ff_rcp_u(p);
      const ff G = ff_mul_u(g, ip);
      const ff Gu = ff_mul_u(G, u);
      ff_acc(acc[1], G);
      ff_acc(acc[2], Gu);
      ff_acc_mul(acc[3], Gu, u);
      ff_acc(acc[4], ip);
      ff_acc_mul(acc[5], ip, x);
    }
    return 0;
  } else {  // PROD3
    // The factors are over disjoint observables, so log p = log p_m + log
    // p_t + log p_c and each factor's moments depend on its own density
    // only.  The fast pass (kSlow = false) takes the mass and angle factors
    // of every event, and the decay factor of the events outside its
    // resolution region; an event in the region returns 1 after its mass and
    // angle terms are summed, and the slow pass (kSlow = true) then adds its
    // decay factor alone.  2 in the fast pass: nothing of the event was
    // summed, the whole event takes the FP64 path; 2 in the slow pass: the
    // decay factor alone takes it.
    const auto t = obs_value<kF32>(in.x[1]);
    const float* kd = k + 16;
    if constexpr (!kSlow) {
      const auto m = obs_value<kF32>(in.x[0]);
      const auto c = obs_value<kF32>(in.x[2]);
      const ff um = ff_mul(ff_sub(m, ldc(k, 0)), ldc(k, 2));
      bool dm = false;
      const ff g = ff_exp0(T, ff_fma_u(ff_scale(um, -0.5f), um, ldc(k, 14)), ok, dm);
      const ff ym = ff_fma(m, ldc(k, 10), ff_neg(ldc(k, 12)));
      const ff pm = ff_fma(ldc(k, 4), g, ff_fma(ldc(k, 8), ym, ldc(k, 6)));
      const ff pa = ff_fma(ff_fma(ldc(k, 42), c, ldc(k, 40)), c, ldc(k, 38));
      const bool slow = __fmaf_rn(-ff_hi(t), kd[13], kd[12]) >= kSlowZf;
      // the decay's fast formula for every lane, used where not slow
      ff R, u;
      bool okd = true;
      const ff vsf = decay_shape<false>(T, kd, t, &R, &u, okd, dropped);
      const ff ptf = ff_fma(ldc(kd, 4), vsf, ff_fma(ff_fma(ldc(kd, 10), t, ldc(kd, 8)), t, ldc(kd, 6)));
      const ff vs = slow ? ff{0.0f, 0.0f} : vsf;
      const ff pt = slow ? ff{1.0f, 0.0f} : ptf;
      okd = slow || (okd && !(dropped && pt.hi < 1e-14f));
      const ff p = ff_mul_u(ff_mul_u(pm, pt), pa);  // logprod_mul takes it unnormalised
      ok = ok && okd && p.hi > 7.9e-31f && p.hi < 1.2e30f && pm.hi > 7.9e-31f && pa.hi > 7.9e-31f &&
           pm.hi < 1.2e30f && pa.hi < 1.2e30f && pt.hi < 1.2e30f;
      if (!ok || (dm && pm.hi < 1e-14f)) return 2;
      logprod_mul(L, p);
      if constexpr (kGrad) {
        const ff ipm = ff_rcp_u(pm), ipa = ff_rcp_u(pa);
        const ff iptf = ff_rcp_u(pt);
        const ff ipt = slow ? ff{0.0f, 0.0f} : iptf;
        const ff G = ff_mul_u(g, ipm);
        const ff Gu = ff_mul_u(G, um);
        ff_acc(acc[1], G);
        ff_acc(acc[2], Gu);
        ff_acc_mul(acc[3], Gu, um);
        ff_acc(acc[4], ipm);
        ff_acc_mul(acc[5], ipm, ym);
        const ff E = ff_mul_u(vs, ipt);
        const ff it_ = ff_mul_u(ipt, t);
        ff_acc(acc[6], E);
        ff_acc_mul(acc[7], E, t);
        ff_acc(acc[8], ipt);
        ff_acc(acc[9], it_);
        ff_acc_mul(acc[10], it_, t);
        // the angle factor (1 + a1 c + a2 c^2)/I needs only sum c/p_c and
        // sum c^2/p_c: its sum of 1/p_c times 1/I equals the event count
        // less the rest, so slot 13 carries the count (set per part)
        const ff iac = ff_mul_u(ipa, c);
        ff_acc(acc[14], iac);
        ff_acc_mul(acc[15], iac, c);
      }
      return slow ? 1 : 0;
    } else {
      ff R, u;
      const ff vs = decay_shape<true>(T, kd, t, &R, &u, ok, dropped);
      const ff pt = ff_fma(ldc(kd, 4), vs, ff_fma(ff_fma(ldc(kd, 10), t, ldc(kd, 8)), t, ldc(kd, 6)));
      ok = ok && pt.hi > 7.9e-31f && pt.hi < 1.2e30f;
      if (!ok || (dropped && pt.hi < 1e-14f)) return 2;
      logprod_mul(L, pt);
      if constexpr (kGrad) {
        const ff ipt = ff_rcp_u(pt);
        const ff E = ff_mul_u(vs, ipt);
        const ff it_ = ff_mul_u(ipt, t);
        ff_acc(acc[6], E);
        ff_acc_mul(acc[7], E, t);
        ff_acc(acc[8], ipt);
        ff_acc(acc[9], it_);
        ff_acc_mul(acc[10], it_, t);
        const ff ER = ff_mul_u(E, R);
        ff_acc(acc[11], ER);
        ff_acc_mul(acc[12], ER, u);
      }
      return 0;
    }
  }
}

}  // namespace rf
