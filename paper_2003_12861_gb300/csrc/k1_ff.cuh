// K1's float-float path for the decay sub-model SUM(GAUSSEXP(t; tau, mu,
// sigma), CHEB2(t; c1, c2); f).
//
// The parameter-point work of K1 is a chain of transcendentals (erfc, exp,
// log) and divisions.  In FP64 each warp instruction holds a sub-partition's
// FP64 unit for ~64 cycles, so a single chain takes ~15 us; on the FP32 pipe
// the same chain in float-float arithmetic (ff.cuh) is several times
// shorter.  The expressions are those of node_consts / end_vals (the
// normalisation integral of the decay convolved with the Gaussian
// resolution, Sec. 4's "values that depend only on parameters") and of
// prep_decay_consts / prep_decay_K (the per-event constants and the moment
// matrix K), with the same output layouts.  A set whose values leave the
// float-float range, or whose differences would lose more than a factor ten
// of the pair's ~1e-14 precision, returns false and takes the FP64 path.
#pragma once

#include "nll_ff.cuh"

namespace rf {

// erfc(y) for y >= 0 as exp(-y^2) erfcx(y); 0 for y > 8.3 (erfc < 1.4e-31),
// where the callers only add it to terms that the guards keep far larger.
__device__ __forceinline__ ff ff_erfc_pos(const FFTables& T, ff y, bool& ok) {
  if (y.hi > 8.3f) return {0.0f, 0.0f};
  return ff_mul(ff_exp(T, ff_neg(ff_sqr(y)), ok), ff_erfcx(T, y, ok));
}

// exp(x), 0 below e^-69 (likewise only added to far larger terms)
__device__ __forceinline__ ff ff_exp_or0(const FFTables& T, ff x, bool& ok) {
  if (x.hi < -69.0f) return {0.0f, 0.0f};
  return ff_exp(T, x, ok);
}

// The decay node's parameters at the point, split to float pairs.
struct DecayFF {
  ff tau, mu, sg, isg, it, s, al, be;
  int cs;  // mass case of [al, be] (mass_case)
  bool ok;
};

__device__ __forceinline__ DecayFF decay_setup(const PNode& q, double tau, double mu, double sg) {
  DecayFF d;
  d.ok = true;
  d.tau = ff_split(tau, d.ok);
  d.mu = ff_split(mu, d.ok);
  d.sg = ff_split(sg, d.ok);
  const ff lo = ff_split(q.lo, d.ok), hi = ff_split(q.hi, d.ok);
  d.ok = d.ok && d.tau.hi > 0.0f && d.sg.hi > 0.0f;  // else the FP64 path flags the point
  if (!d.ok) return d;
  d.isg = ff_rcp(d.sg);
  d.it = ff_rcp(d.tau);
  d.s = ff_mul(d.sg, d.it);
  d.al = ff_mul(ff_sub(lo, d.mu), d.isg);
  d.be = ff_mul(ff_sub(hi, d.mu), d.isg);
  d.cs = d.al.hi >= 0.0f ? 0 : d.be.hi <= 0.0f ? 1 : 2;
  return d;
}

// What the decay node needs at one end x (standardised, = u at that end):
// the mass term e, p = exp(-x^2/2), the convolution f = 1/2 exp(A) erfc(z)
// and df/d(tau, mu, sigma) (gaussexp_point).
struct EndFF {
  ff e, p, f, df[3];
};

__device__ __forceinline__ void decay_end_ff(const FFTables& T, const DecayFF& d, ff x, EndFF& v, bool& ok) {
  const ff r2 = {kSqrt1_2_hi, kSqrt1_2_lo};
  const ff xr = ff_mul(x, r2);
  if (d.cs == 2) {  // erf(xr) = sign(xr) (1 - erfc(|xr|))
    const bool neg = xr.hi < 0.0f;
    const ff e1 = ff_add_f(ff_neg(ff_erfc_pos(T, neg ? ff_neg(xr) : xr, ok)), 1.0f);
    v.e = neg ? ff_neg(e1) : e1;
  } else {
    v.e = ff_erfc_pos(T, d.cs == 0 ? xr : ff_neg(xr), ok);
  }
  const ff g = ff_exp_or0(T, ff_scale(ff_sqr(x), -0.5f), ok);
  v.p = g;
  const ff A = ff_mul(d.s, ff_sub(ff_scale(d.s, 0.5f), x));
  const ff z = ff_mul(ff_sub(d.s, x), r2);
  ff val;
  if (z.hi > 0.0f)
    val = ff_scale(ff_mul(g, ff_erfcx(T, z, ok)), 0.5f);
  else
    val = ff_scale(ff_mul(ff_exp_or0(T, A, ok), ff_add_f(ff_neg(ff_erfc_pos(T, ff_neg(z), ok)), 2.0f)), 0.5f);
  const ff sit = ff_mul(d.s, d.it);
  const ff dA[3] = {ff_mul(sit, ff_sub(x, d.s)), d.it, sit};
  const ff dz[3] = {ff_neg(ff_mul(sit, r2)), ff_mul(r2, d.isg), ff_mul(ff_fma(x, d.isg, d.it), r2)};
  const ff gi = ff_mul(g, ff{kInvSqrtPi_hi, kInvSqrtPi_lo});
  v.f = val;
  for (int k = 0; k < 3; ++k) v.df[k] = ff_sub(ff_mul(val, dA[k]), ff_mul(gi, dz[k]));
}

__device__ __forceinline__ void put_pair(float* o, ff v) {
  o[0] = v.hi;
  o[1] = v.lo;
}

// The node's constants ge[8] (node_consts' GAUSSEXP layout: mu, 1/sigma,
// sigma/tau, 1/tau, 1/I, dlogI/d(tau, mu, sigma)) from the two ends, then
// the set's per-event constants and K (nacc = 8, rows tau, mu, sigma, c1,
// c2, f at 1..6, moments at 1..7) into out.  ch, sm: the CHEB2 and SUM
// constants (FP64, node_consts' layout).  False: take the FP64 path.
__device__ __forceinline__ bool decay_point_ff(const FFTables& T, const DecayFF& d, const EndFF& A,
                                               const EndFF& B, const double* ch, const double* sm, ff* ge,
                                               float* out) {
  bool ok = true;
  const ff D = ff_scale(d.cs == 0 ? ff_sub(A.e, B.e) : ff_sub(B.e, A.e), 0.5f);
  // the Gaussian mass in range and the integral keep their precision
  const float ref = d.cs == 0 ? A.e.hi : d.cs == 1 ? B.e.hi : 1.0f;
  ok = ok && D.hi >= 0.05f * ref;
  const ff br = ff_add(ff_sub(D, B.f), A.f);
  ok = ok && br.hi >= 0.1f * (D.hi + A.f.hi) && br.hi > 1e-15f;
  if (!ok) return false;
  const ff I = ff_mul(d.tau, br), iI = ff_rcp(I);
  const ff is2p = {kInvSqrt2Pi_hi, kInvSqrt2Pi_lo};
  const ff pa = ff_mul(A.p, is2p), pb = ff_mul(B.p, is2p);
  const ff dD1 = ff_neg(ff_mul(ff_sub(pb, pa), d.isg));
  const ff dD2 = ff_neg(ff_mul(ff_sub(ff_mul(d.be, pb), ff_mul(d.al, pa)), d.isg));
  ge[0] = d.mu;
  ge[1] = d.isg;
  ge[2] = d.s;
  ge[3] = d.it;
  ge[4] = iI;
  ge[5] = ff_mul(ff_add(br, ff_mul(d.tau, ff_sub(A.df[0], B.df[0]))), iI);
  ge[6] = ff_mul(ff_mul(d.tau, ff_add(ff_sub(dD1, B.df[1]), A.df[1])), iI);
  ge[7] = ff_mul(ff_mul(d.tau, ff_add(ff_sub(dD2, B.df[2]), A.df[2])), iI);
  // per-event constants (prep_decay_consts' layout)
  const ff c0 = ff_split(ch[0], ok), c1p = ff_split(ch[1], ok), iIb = ff_split(ch[2], ok);
  const ff dI1 = ff_split(ch[3], ok), dI2 = ff_split(ch[4], ok), a1 = ff_split(ch[5], ok), a2 = ff_split(ch[6], ok);
  const ff f = ff_split(sm[0], ok), fl = ff_split(sm[1], ok);
  const ff lIs = ff_log(T, iI, ok);
  if (!ok) return false;
  const ff one = {1.0f, 0.0f};
  const ff T2_0 = ff_add_f(ff_scale(ff_sqr(c1p), 2.0f), -1.0f);
  const ff S[3] = {ff_add(ff_sub(one, ff_mul(a1, c1p)), ff_mul(a2, T2_0)),
                   ff_sub(ff_mul(a1, c0), ff_scale(ff_mul(ff_mul(a2, c0), c1p), 4.0f)),
                   ff_scale(ff_mul(a2, ff_sqr(c0)), 2.0f)};
  const ff r2 = {kSqrt1_2_hi, kSqrt1_2_lo};
  put_pair(out + 0, ff_add(ff_fma(d.mu, d.it, ff_scale(ff_sqr(d.s), 0.5f)), lIs));
  put_pair(out + 2, d.it);
  put_pair(out + 4, f);
  const ff flb = ff_mul(fl, iIb);
  for (int j = 0; j < 3; ++j) put_pair(out + 6 + 2 * j, ff_mul(flb, S[j]));
  out[12] = ff_mul(ff_fma(d.mu, d.isg, d.s), r2).hi;  // z ~ zc - t zs (decides the slow path only)
  out[13] = ff_mul(d.isg, r2).hi;
  put_pair(out + 14, d.mu);
  put_pair(out + 16, d.isg);
  put_pair(out + 18, d.s);
  put_pair(out + 20, lIs);
  // K (prep_decay_K's entries), zero elsewhere
  constexpr int nacc = 8, Q = 7;
  float* K = out + ff_koff(SHAPE_SUM_GAUSSEXP_CHEB2);
  for (int i = 0; i < 2 * Q * nacc; ++i) K[i] = 0.0f;
  auto put = [&](int r, int m, ff v) { put_pair(K + 2 * (r * nacc + m), v); };
  put(0, 0, one);
  const ff sit = ff_mul(d.s, d.it), fs = ff_mul(f, sit);
  put(1, 2, ff_mul(fs, d.isg));
  put(1, 1, ff_neg(ff_mul(f, ff_add(ff_add(ff_mul(ff_mul(sit, d.mu), d.isg), ff_mul(sit, d.s)), ge[5]))));
  put(1, 6, ff_mul(fs, r2));
  put(2, 1, ff_mul(f, ff_sub(d.it, ge[6])));
  put(2, 6, ff_neg(ff_mul(ff_mul(f, d.isg), r2)));
  put(3, 1, ff_mul(f, ff_sub(sit, ge[7])));
  put(3, 6, ff_neg(ff_mul(ff_mul(f, d.it), r2)));
  put(3, 7, ff_neg(ff_mul(ff_mul(f, d.isg), r2)));
  const ff T1[3] = {ff_neg(c1p), c0, {0.0f, 0.0f}};
  const ff T2[3] = {T2_0, ff_scale(ff_mul(c0, c1p), -4.0f), ff_scale(ff_sqr(c0), 2.0f)};
  for (int j = 0; j < 3; ++j) {
    put(4, 3 + j, ff_mul(flb, ff_sub(T1[j], ff_mul(dI1, S[j]))));
    put(5, 3 + j, ff_mul(flb, ff_sub(T2[j], ff_mul(dI2, S[j]))));
    put(6, 3 + j, ff_neg(ff_mul(iIb, S[j])));
  }
  put(6, 1, one);
  return true;
}

}  // namespace rf
