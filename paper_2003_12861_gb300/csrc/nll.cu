// Likelihood kernels: parameter-point constants (K1), the fused per-event
// evaluation with its adjoint (K2), and the deterministic reduction tree over
// event chunks (K3, fused into K2's epilogue).
//
// Paper, Sec. 4: a likelihood needs the probability of every event; RooFit
// loads one event at a time into the graph's leaves and re-evaluates every
// observable-dependent node, with parameter-only branches cached.  Sec. 4.1
// batches all events per node, Sec. 4.2 vectorises with no data dependencies,
// register-only work, few branches and simple reductions.  On the GPU the
// batch is a 4096-event chunk, the "vector" is a warp, and a whole graph is
// evaluated per event in registers; normalisation integrals and all other
// parameter-only quantities are computed once per parameter point (K1).
#include <cmath>
#include <cstdio>

#include "expr.cuh"
#include "k1_ff.cuh"
#include "nll_ff.cuh"
#include "nll_kernels.cuh"

namespace rf {

namespace {

constexpr double kSqrt1_2 = 0.70710678118654752440;
constexpr double kSqrt2Pi = 2.50662827463100050242;
constexpr double kInvSqrt2Pi = 0.39894228040143267794;
constexpr double kInvSqrtPi = 0.56418958354775628695;
constexpr double kTwoInvSqrtPi = 1.12837916709551257390;
// Below this z the erfc factor of the decay-resolution convolution equals 2
// to better than 1e-22 relative and its derivative term is below 1e-21 of
// the exponential's, so the event takes the one-exponential fast path.
constexpr double kSlowZ = -7.0;

// Programmatic dependent launch: K1 lets the event kernel be scheduled at
// once; the event kernel stages its tables, then waits for K1's completion
// (and memory) before it reads anything K1 writes.  Without a programmatic
// dependency (a plain launch) the wait returns at once.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ double param_of(const PNode& q, int j, const double* th) {
  return q.pfree[j] >= 0 ? th[q.pfree[j]] : q.pfixed[j];
}

// Phi(be) - Phi(al) from one term per end, using erfc on the tail side to
// keep far-tail precision: case 0 (al >= 0) e(x) = erfc(x/sqrt2), mass
// (e(al) - e(be))/2; case 1 (be <= 0) e(x) = erfc(-x/sqrt2), case 2
// e(x) = erf(x/sqrt2), both with mass (e(be) - e(al))/2.
__device__ __forceinline__ int mass_case(double al, double be) { return al >= 0.0 ? 0 : be <= 0.0 ? 1 : 2; }
__device__ __forceinline__ double mass_term(int cs, double x) {
  return cs == 0 ? erfc(x * kSqrt1_2) : cs == 1 ? erfc(-x * kSqrt1_2) : erf(x * kSqrt1_2);
}
__device__ __forceinline__ double mass_of(int cs, double ea, double eb) {
  return cs == 0 ? 0.5 * (ea - eb) : 0.5 * (eb - ea);
}

// Decay (x) resolution at one point t, with d/d(tau, mu, sigma).
// f = 1/2 exp(A) erfc(z), A = s(s/2 - u), z = (s - u)/sqrt2, u = (t-mu)/sigma,
// s = sigma/tau; A - z^2 = -u^2/2 gives df = f dA - exp(-u^2/2)/sqrt(pi) dz.
__device__ void gaussexp_point(double t, double tau, double mu, double sigma, double* f, double df[3]) {
  const double u = (t - mu) / sigma, s = sigma / tau;
  const double A = s * (0.5 * s - u), z = (s - u) * kSqrt1_2;
  const double g = exp(-0.5 * u * u);
  const double val = z > 0.0 ? 0.5 * g * erfcx(z) : 0.5 * exp(A) * erfc(z);
  const double it = 1.0 / tau;
  const double dA[3] = {s * (u - s) * it, it, s * it};
  const double dz[3] = {-s * it * kSqrt1_2, kSqrt1_2 / sigma, (it + u / sigma) * kSqrt1_2};
  *f = val;
  for (int k = 0; k < 3; ++k) df[k] = val * dA[k] - g * kInvSqrtPi * dz[k];
}

// What a Gaussian or decay-resolution node needs at one end of its range:
// x the standardised end (al or be), t the end itself.  e = the mass term,
// p = exp(-x^2/2), and for the decay the convolution f(t) with d/d(tau, mu,
// sigma).
struct EndVals {
  double e, p, f, df[3];
};
__device__ __forceinline__ void end_vals(int cs, double x, bool decay, double t, double tau, double mu, double sg,
                                         EndVals& v) {
  v.e = mass_term(cs, x);
  v.p = exp(-0.5 * x * x);
  if (decay) {
    gaussexp_point(t, tau, mu, sg, &v.f, v.df);
  } else {
    v.f = 0.0;
    v.df[0] = v.df[1] = v.df[2] = 0.0;
  }
}
// One part of an end's work, for K1's job split: part 0 the mass term and
// p, part 1 the decay convolution; end 0 = lo, 1 = hi.  The same expressions
// as end_vals, so the split does not change any bit.
__device__ __forceinline__ void end_part(int cs, double x, bool decay, double t, double tau, double mu, double sg,
                                         int part, EndVals& v) {
  if (part == 0) {
    v.e = mass_term(cs, x);
    v.p = exp(-0.5 * x * x);
  } else if (decay) {
    gaussexp_point(t, tau, mu, sg, &v.f, v.df);
  } else {
    v.f = 0.0;
    v.df[0] = v.df[1] = v.df[2] = 0.0;
  }
}

// Mean of exp(y w) on w in [0, 1]: 1/(1 - e^-y) - 1/y; series near 0.
__device__ double trunc_exp_mean01(double y) {
  if (fabs(y) < 1e-3) return 0.5 + y * (1.0 / 12.0) - y * y * y * (1.0 / 720.0);
  return -1.0 / expm1(-y) - 1.0 / y;
}

// ------------------------------------------------------------------- K1

// Constants of pdf node q at the parameter point th into c (the layout in
// rf_internal.h); returns false if th is outside the node's domain.  A
// Gaussian or decay node takes its two range ends from `ends` when K1 has
// computed them as separate jobs, else computes them in turn.
__device__ bool node_consts(const PNode& q, const double* th, double* c, const EndVals* ends) {
  bool bad = false;
  const double lo = q.lo, hi = q.hi;
  switch (q.kind) {
    case GAUSS: {
      const double mu = param_of(q, 0, th), sg = param_of(q, 1, th);
      if (!(sg > 0.0)) { bad = true; break; }
      const double isg = 1.0 / sg;
      const double al = (lo - mu) * isg, be = (hi - mu) * isg;
      const int cs = mass_case(al, be);
      EndVals A, B;
      if (ends) {
        A = ends[0];
        B = ends[1];
      } else {
        end_vals(cs, al, false, lo, 1.0, mu, sg, A);
        end_vals(cs, be, false, hi, 1.0, mu, sg, B);
      }
      const double I = sg * kSqrt2Pi * mass_of(cs, A.e, B.e);
      const double dmu = A.p - B.p;
      const double dsg = I * isg - (be * B.p - al * A.p);
      if (!(I > 0.0)) bad = true;
      const double iI = 1.0 / I;
      c[0] = mu; c[1] = isg; c[2] = iI; c[3] = dmu * iI; c[4] = dsg * iI;
      break;
    }
    case EXPO: {
      const double cc = param_of(q, 0, th), L = hi - lo;
      const double xref = cc > 0.0 ? hi : lo;
      double Iref;
      if (cc == 0.0) Iref = L;
      else if (cc > 0.0) Iref = -expm1(-cc * L) / cc;
      else Iref = expm1(cc * L) / cc;
      c[0] = cc; c[1] = xref; c[2] = 1.0 / Iref; c[3] = lo + L * trunc_exp_mean01(cc * L);
      break;
    }
    case GAUSSEXP: {
      const double tau = param_of(q, 0, th), mu = param_of(q, 1, th), sg = param_of(q, 2, th);
      if (!(tau > 0.0) || !(sg > 0.0)) { bad = true; break; }
      const double isg = 1.0 / sg;
      const double al = (lo - mu) * isg, be = (hi - mu) * isg;
      const int cs = mass_case(al, be);
      EndVals A, B;
      if (ends) {
        A = ends[0];
        B = ends[1];
      } else {
        end_vals(cs, al, true, lo, tau, mu, sg, A);
        end_vals(cs, be, true, hi, tau, mu, sg, B);
      }
      const double D = mass_of(cs, A.e, B.e);
      const double br = D - B.f + A.f;
      const double I = tau * br;
      const double pa = A.p * kInvSqrt2Pi, pb = B.p * kInvSqrt2Pi;
      const double dD[3] = {0.0, -(pb - pa) * isg, -(be * pb - al * pa) * isg};
      if (!(I > 0.0)) bad = true;
      const double iI = 1.0 / I;
      c[0] = mu; c[1] = isg; c[2] = sg / tau; c[3] = 1.0 / tau; c[4] = iI;
      for (int k = 0; k < 3; ++k) c[5 + k] = ((k == 0 ? br : 0.0) + tau * (dD[k] - B.df[k] + A.df[k])) * iI;
      break;
    }
    case CHEB: {
      const int np = q.n_par;
      double sum = 2.0;
      for (int k = 1; k <= np; ++k) {
        const double ck = param_of(q, k - 1, th);
        const double Tk = (k % 2 == 0) ? 2.0 / (1.0 - (double)k * k) : 0.0;
        sum += ck * Tk;
        c[3 + np + k - 1] = ck;
        c[3 + k - 1] = 0.5 * (hi - lo) * Tk;  // dI/dc_k, divided below
      }
      const double I = 0.5 * (hi - lo) * sum;
      if (!(I > 0.0)) bad = true;
      c[0] = 2.0 / (hi - lo); c[1] = (hi + lo) / (hi - lo); c[2] = 1.0 / I;
      for (int k = 0; k < np; ++k) c[3 + k] /= I;
      break;
    }
    case POISSON: {
      // I = sum_{k=lo}^{hi-1} pmf(k): from the mode outward by the ratio
      // recursion pmf(k+1) = pmf(k) lambda/(k+1), stopping once the terms
      // are below 1e-18 of the sum (the tails decrease geometrically).
      // dI/dlambda telescopes to pmf(lo-1) - pmf(hi-1).
      const double lam = param_of(q, 0, th);
      if (!(lam > 0.0)) { bad = true; break; }
      const double ll = log(lam);
      const double km = fmin(fmax(floor(lam), lo), hi - 1.0);
      const double pm = exp(km * ll - lam - lgamma(km + 1.0));
      double I = pm, p = pm;
      for (double k = km + 1.0; k < hi; k += 1.0) {
        p *= lam / k;
        I += p;
        if (p < 1e-18 * I) break;
      }
      p = pm;
      for (double k = km; k > lo; k -= 1.0) {
        p *= k / lam;
        I += p;
        if (p < 1e-18 * I) break;
      }
      const double pb = exp((hi - 1.0) * ll - lam - lgamma(hi));
      const double pa = lo > 0.0 ? exp((lo - 1.0) * ll - lam - lgamma(lo)) : 0.0;
      if (!(I > 0.0)) bad = true;
      c[0] = lam; c[1] = ll; c[2] = 1.0 / lam; c[3] = 1.0 / I; c[4] = (pa - pb) / I;
      break;
    }
    case POLY: {
      const int np = q.n_par;
      double I = hi - lo, ph = hi, pl = lo;
      for (int k = 1; k <= np; ++k) {
        ph *= hi; pl *= lo;
        const double ak = param_of(q, k - 1, th);
        const double Pk = (ph - pl) / (k + 1);
        I += ak * Pk;
        c[1 + np + k - 1] = ak;
        c[1 + k - 1] = Pk;
      }
      if (!(I > 0.0)) bad = true;
      c[0] = 1.0 / I;
      for (int k = 0; k < np; ++k) c[1 + k] /= I;
      break;
    }
    case EXPR:
      // computed by the whole block of the parameter-point kernel
      // (expr_consts_block); a single thread never takes this node
      bad = true;
      break;
    case SUM: {
      double fs = 0.0;
      for (int j = 0; j < q.n_par; ++j) {
        const double f = param_of(q, j, th);
        c[j] = f;
        fs += f;
      }
      c[q.n_par] = 1.0 - fs;
      break;
    }
    default: break;
  }
  return !bad;
}

// Extended likelihood: nu - N log nu for a set of N events and its
// derivative 1 - N/nu (the Poisson probability of N given nu, without the
// constant log N!).  nu <= 0 is flagged by the parameter-point kernel.
__device__ __forceinline__ void extended_term(const Program& P, const Pass& pass, int set, double N, double* t,
                                              double* dt) {
  const double nu = P.ext_free >= 0 ? pass.theta[(size_t)set * P.n_free + P.ext_free] : P.ext_fixed;
  *t = nu - (N > 0.0 ? N * log(nu) : 0.0);
  *dt = 1.0 - N / nu;
}

__device__ bool extended_bad(const Program& P, const Pass& pass, int s) {
  if (!P.ext) return false;
  const double nu = P.ext_free >= 0 ? pass.theta[(size_t)s * P.n_free + P.ext_free] : P.ext_fixed;
  return !(nu > 0.0);
}

// Finishes a set: domain flag, the float-float constants (unless ff_done),
// and the result of a set without events.
__device__ void finish_param_point(const Program& P, const Pass& pass, int s, bool bad, const double* C,
                                   bool ff_done = false) {
  bad = bad || extended_bad(P, pass, s);
  pass.flags[s] = bad ? kThetaBad : 0;
  if (!ff_done && !bad && pass.ff_shape != SHAPE_GENERIC && pass.ffc)
    prepare_ff(P, pass.ff_shape, C, pass.ffc + (size_t)s * kFFConst);
  if (pass.offsets[s + 1] == pass.offsets[s] && pass.pairs) {  // no events: empty pairs
    for (int k = 0; k < 2 * (1 + P.n_free); ++k) pass.pairs[(size_t)s * 2 * (1 + P.n_free) + k] = 0.0;
  } else if (pass.offsets[s + 1] == pass.offsets[s]) {  // no events: the empty sum (+ nu if extended)
    double* o = pass.out + (size_t)s * (1 + P.n_free);
    double ext = 0.0, dext = 0.0;
    if (P.ext && !bad) extended_term(P, pass, s, 0.0, &ext, &dext);
    o[0] = bad ? INFINITY : ext;
    if (pass.want_grad)
      for (int k = 0; k < P.n_free; ++k) o[1 + k] = k == P.ext_free ? dext : 0.0;
  }
}

// The decay shape's float-float K1 path (k1_ff.cuh) applies to its plain
// (not extended) form; the event kernel then reads the float-float block.
__device__ __forceinline__ bool decay_ff_eligible(const Program& P, const Pass& pass) {
  return pass.ff_shape == SHAPE_SUM_GAUSSEXP_CHEB2 && pass.ffc && !P.ext;
}

// One thread's float-float parameter point of a decay set: the CHEB2 and
// SUM constants in FP64, the decay node, its per-event constants and K in
// float-float.  False (nothing usable written): take the FP64 path.
__device__ bool decay_set_ff(const FFTables& T, const Program& P, const double* th, double* C, float* out) {
  const PNode &qg = P.node[0], &qc = P.node[1], &qs = P.node[2];
  if (!node_consts(qc, th, C + qc.cofs, nullptr) || !node_consts(qs, th, C + qs.cofs, nullptr)) return false;
  const DecayFF d = decay_setup(qg, param_of(qg, 0, th), param_of(qg, 1, th), param_of(qg, 2, th));
  if (!d.ok) return false;
  bool ok = true;
  EndFF A, B;
  decay_end_ff(T, d, d.al, A, ok);
  decay_end_ff(T, d, d.be, B, ok);
  ff ge[8];
  if (!ok || !decay_point_ff(T, d, A, B, C + qc.cofs, C + qs.cofs, ge, out)) return false;
  for (int k = 0; k < 8; ++k) C[qg.cofs + k] = ff_to_double(ge[k]);
  return true;
}

// K1, one thread per active set (many sets: toy fits).  Also resets the
// event kernel's work counter.
__global__ void param_point_kernel(const __grid_constant__ Program P, Pass pass) {
  __shared__ FFTables T;
  const int n_active = pass.dyn ? pass.dyn[0] : pass.n_active;
  if (n_active == 0) return;
  pdl_launch_dependents();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a == 0) {
    for (int i = 0; i < (pass.n_counters > 1 ? pass.n_counters : 1); ++i) pass.counter[i] = 0;
    if (pass.slow) *pass.slow = 0ull;
  }
  const bool try_ff = decay_ff_eligible(P, pass);
  if (try_ff) {
    ff_load_tables(T);
    __syncthreads();
  }
  if (a >= n_active) return;
  const int s = pass.sets[a];
  const double* th = pass.theta + (size_t)s * P.n_free;
  double* C = pass.consts + (size_t)s * P.n_const;
  if (try_ff && decay_set_ff(T, P, th, C, pass.ffc + (size_t)s * kFFConst)) {
    finish_param_point(P, pass, s, false, C, true);
    return;
  }
  bool bad = false;
  for (int n = 0; n < P.n_pdf; ++n) bad |= !node_consts(P.node[n], th, C + P.node[n].cofs, nullptr);
  finish_param_point(P, pass, s, bad, C);
}

// K1, one block per active set (few sets: one large fit).  Every FP64 warp
// instruction occupies a sub-partition's FP64 unit for many cycles, so a lone
// thread's chain of transcendentals is slow; here the work is cut into jobs
// on separate warps (the four sub-partitions' FP64 units run at once): per
// Gaussian node the mass term and density at each range end (2 jobs), per
// decay node also the convolution at each end (4 jobs); then every node's
// constants on its own warp; then the float-float constants.
constexpr int kK1Warps = 8;
static_assert(kK1Warps * 32 == kQuadPanels, "the EXPR quadrature takes one panel per thread of the block");
template <bool kExpr>
__global__ void __launch_bounds__(kK1Warps * 32) param_point_block_kernel(const __grid_constant__ Program P,
                                                                          Pass pass) {
  __shared__ EndVals ends[kMaxPdf][2];
  __shared__ double Ks[13 * 16];
  __shared__ double Cs[kMaxConst];  // the set's constant block, copied out at the end
  __shared__ int sbad;
  __shared__ FFTables T;
  __shared__ EndFF endff[2];
  __shared__ ff geff[8];
  __shared__ int ffok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if ((int)blockIdx.x >= (pass.dyn ? pass.dyn[0] : pass.n_active)) return;
  if (blockIdx.x == 0 && tid == 0) {
    for (int i = 0; i < (pass.n_counters > 1 ? pass.n_counters : 1); ++i) pass.counter[i] = 0;
    if (pass.slow) *pass.slow = 0ull;
  }
  // The event kernel may launch once this kernel has started (FP64 path) or
  // once the float-float chain is done: its waiting blocks would otherwise
  // share the issue slots that the chain's single warp depends on.
  const bool try_ff = decay_ff_eligible(P, pass);
  if (!try_ff) pdl_launch_dependents();
  if (tid == 0) {
    sbad = 0;
    ffok = 1;
  }
  if (try_ff) ff_load_tables(T);
  __syncthreads();
  const int s = pass.sets[blockIdx.x];
  const double* th = pass.theta + (size_t)s * P.n_free;
  double* C = pass.consts + (size_t)s * P.n_const;
  if (try_ff) {
    // float-float path (k1_ff.cuh): the two range ends of the decay node on
    // lanes 0 and 1 while warps 1 and 2 take the CHEB2 and SUM constants
    const PNode &qg = P.node[0], &qc = P.node[1], &qs = P.node[2];
    if (warp == 0 && lane < 2) {
      const DecayFF d = decay_setup(qg, param_of(qg, 0, th), param_of(qg, 1, th), param_of(qg, 2, th));
      bool ok = d.ok;
      if (ok) decay_end_ff(T, d, lane ? d.be : d.al, endff[lane], ok);
      if (!ok) atomicAnd(&ffok, 0);
    } else if ((warp == 1 || warp == 2) && lane == 0) {
      const PNode& q = warp == 1 ? qc : qs;
      if (!node_consts(q, th, Cs + q.cofs, nullptr)) atomicOr(&sbad, 1);
    }
    __syncthreads();
    if (ffok && !sbad && tid == 0) {
      const DecayFF d = decay_setup(qg, param_of(qg, 0, th), param_of(qg, 1, th), param_of(qg, 2, th));
      ff ge[8];
      if (decay_point_ff(T, d, endff[0], endff[1], Cs + qc.cofs, Cs + qs.cofs, ge,
                         pass.ffc + (size_t)s * kFFConst)) {
        for (int k = 0; k < 8; ++k) geff[k] = ge[k];
      } else {
        ffok = 0;
      }
    }
    __syncthreads();
    pdl_launch_dependents();
    if (ffok && !sbad) {
      if (tid < 8) Cs[qg.cofs + tid] = ff_to_double(geff[tid]);
      __syncthreads();
      for (int i = tid; i < P.n_const; i += blockDim.x) C[i] = Cs[i];
      if (tid == 0) finish_param_point(P, pass, s, false, Cs, true);
      return;
    }
    // otherwise the FP64 path below recomputes the set
    if (tid == 0) sbad = 0;
    __syncthreads();
  }
  // EXPR nodes: normalisation integral and its derivatives by the whole
  // block, constants [1/I, dlogI/dp_1..n, p_1..n]
  if constexpr (kExpr) {
    __shared__ QuadSmem quad[1];
    for (int n = 0; n < P.n_pdf; ++n) {
      const PNode& q = P.node[n];
      if (q.kind != EXPR) continue;
      double par[kMaxPar], I[1 + kMaxPar];
      for (int j = 0; j < q.n_par; ++j) par[j] = param_of(q, j, th);
      const bool ok = expr_integrate_block(P, q, par, quad[0], I);
      if (tid == 0) {
        if (!ok) {
          sbad = 1;
        } else {
          double* c = Cs + q.cofs;
          c[0] = 1.0 / I[0];
          for (int j = 0; j < q.n_par; ++j) {
            c[1 + j] = I[1 + j] / I[0];
            c[1 + q.n_par + j] = par[j];
          }
        }
      }
      __syncthreads();
    }
  }
  // jobs: (node, end, part), numbered in node order
  if (lane == 0) {
    int j = 0;
    for (int n = 0; n < P.n_pdf; ++n) {
      const PNode& q = P.node[n];
      if (q.kind != GAUSS && q.kind != GAUSSEXP) continue;
      const bool decay = q.kind == GAUSSEXP;
      const int parts = decay ? 2 : 1;
      for (int e = 0; e < 2; ++e)
        for (int part = 0; part < parts; ++part, ++j) {
          if (j % kK1Warps != warp) continue;
          const double tau = decay ? param_of(q, 0, th) : 1.0;
          const double mu = param_of(q, decay ? 1 : 0, th), sg = param_of(q, decay ? 2 : 1, th);
          if (!(sg > 0.0) || !(tau > 0.0)) continue;  // flagged when the node is finished
          const double isg = 1.0 / sg;
          const double al = (q.lo - mu) * isg, be = (q.hi - mu) * isg;
          end_part(mass_case(al, be), e ? be : al, decay, e ? q.hi : q.lo, tau, mu, sg, part, ends[n][e]);
        }
    }
  }
  __syncthreads();
  if (lane == 0) {
    bool bad = false;
    for (int n = warp; n < P.n_pdf; n += kK1Warps) {
      const PNode& q = P.node[n];
      if (q.kind == EXPR) continue;  // done above
      const bool split = q.kind == GAUSS || q.kind == GAUSSEXP;
      bad |= !node_consts(q, th, Cs + q.cofs, split ? ends[n] : nullptr);
    }
    if (bad) atomicOr(&sbad, 1);
  }
  __syncthreads();
  // the float-float constants: jobs on separate warps, then K converted by all threads
  const int shape = pass.ff_shape;
  const bool ff = shape != SHAPE_GENERIC && pass.ffc && sbad == 0 && !extended_bad(P, pass, s);
  if (ff) {
    float* out = pass.ffc + (size_t)s * kFFConst;
    for (int i = tid; i < ff_q(shape) * ff_nacc(shape); i += blockDim.x) Ks[i] = i == 0 ? 1.0 : 0.0;
    __syncthreads();
    if (lane == 0 && warp < ff_jobs(shape)) prepare_ff_job(P, shape, Cs, out, Ks, warp);
    __syncthreads();
    ff_convert_K(shape, Ks, out, tid, blockDim.x);
  }
  for (int i = tid; i < P.n_const; i += blockDim.x) C[i] = Cs[i];
  if (tid == 0) finish_param_point(P, pass, s, sbad != 0, Cs, true);
}

// ------------------------------------------------------------------- K2

__device__ __forceinline__ double load_col(const Columns& cols, int c, int64_t e) {
  return cols.is_f32[c] ? (double)__ldg((const float*)cols.ptr[c] + e) : __ldg((const double*)cols.ptr[c] + e);
}

// Exact two-sum merge of compensated pairs: (s, c) + (t, d).  Symmetric in its
// arguments (the two-sum error is exact), so butterfly lanes agree bitwise.
struct Pair {
  double s, c;
};
__device__ __forceinline__ Pair merge(Pair a, Pair b) {
  const double s = a.s + b.s;
  const double bb = s - a.s;
  const double e = (a.s - (s - bb)) + (b.s - bb);
  return {s, (a.c + b.c) + e};
}

// A lane's running product for sum_i log p_i = log(m) + e ln2: m multiplies
// the mantissas of the p_i (in [1, 2), split from the bits exactly), e sums
// their binary exponents.  One FP64 multiply per event instead of a log; a
// lane takes at most 64 factors per chunk, so m < 2^64.
struct LogProd64 {
  double m;
  int e;
};

__device__ __forceinline__ LogProd64 logprod64_init() { return {1.0, 0}; }

// p > 0 and finite
__device__ __forceinline__ void logprod64_mul(LogProd64& L, double p) {
  int hi = __double2hiint(p), sh = 0;
  if (hi < 0x00100000) {  // subnormal: scale by 2^64 (exact)
    p *= 18446744073709551616.0;
    hi = __double2hiint(p);
    sh = 64;
  }
  L.e += (hi >> 20) - 1023 - sh;
  L.m *= __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(p));
}

__device__ __forceinline__ double logprod64_log(const LogProd64& L) {
  return log(L.m) + (double)L.e * 0.69314718055994530942;
}

// Generic graph interpreter for one event.  kFull = false: the fast path,
// which returns false (and adds nothing) when some node needs its slow path.
// Multiplies p into the lane's running product L (the log p term) and adds
// the slot gradients to acc[1..]; counts events with p <= 0 or not finite in
// *bad instead.
// Nodes [n0, n1) with n1 - 1 as the root: the whole program by default, or
// one factor's sub-program (a PROD factor's nodes are contiguous in program
// order and refer only to each other), whose log p and slot gradients are
// then those of that factor alone.
template <bool kFull, bool kGrad, bool kExpr = false>
__device__ bool eval_generic(const Program& P, const double* __restrict__ C, const double* x, double* acc,
                             LogProd64& L, int* bad, int n0 = 0, int n1 = -1) {
  double v[kMaxPdf];
  const int N = n1 < 0 ? P.n_pdf : n1;
  for (int n = n0; n < N; ++n) {
    const PNode& q = P.node[n];
    const double* c = C + q.cofs;
    switch (q.kind) {
      case GAUSS: {
        const double u = (x[q.col] - c[0]) * c[1];
        v[n] = exp(-0.5 * u * u) * c[2];
        break;
      }
      case EXPO: v[n] = exp(c[0] * (x[q.col] - c[1])) * c[2]; break;
      case GAUSSEXP: {
        const double u = (x[q.col] - c[0]) * c[1], s = c[2];
        const double z = (s - u) * kSqrt1_2;
        double f;
        if (!kFull) {
          if (z >= kSlowZ) return false;
          f = exp(s * (0.5 * s - u));
        } else if (z > 0.0) {
          f = 0.5 * exp(-0.5 * u * u) * erfcx(z);
        } else {
          f = 0.5 * exp(s * (0.5 * s - u)) * erfc(z);
        }
        v[n] = f * c[4];
        break;
      }
      case CHEB: {
        const int np = q.n_par;
        const double xp = x[q.col] * c[0] - c[1];
        double t0 = 1.0, t1 = xp, sh = 1.0;
        for (int k = 1; k <= np; ++k) {
          sh += c[3 + np + k - 1] * t1;
          const double t2 = 2.0 * xp * t1 - t0;
          t0 = t1; t1 = t2;
        }
        v[n] = sh * c[2];
        break;
      }
      case POLY: {
        const int np = q.n_par;
        const double xv = x[q.col];
        double sh = 0.0;
        for (int k = np; k >= 1; --k) sh = (sh + c[1 + np + k - 1]) * xv;
        v[n] = (1.0 + sh) * c[0];
        break;
      }
      case POISSON: {
        const double k = fmin(floor(x[q.col]), q.hi - 1.0);
        v[n] = exp(k * c[1] - c[0] - lgamma(k + 1.0)) * c[3];
        break;
      }
      case EXPR: {
        double f;
        if constexpr (kExpr) v[n] = expr_eval(P, q, c + 1 + q.n_par, x[q.col], 0, &f, nullptr) ? f * c[0] : NAN;
        break;
      }
      case SUM: {
        double r = 0.0;
        for (int j = 0; j < q.n_child; ++j) r += c[j] * v[q.child[j]];
        v[n] = r;
        break;
      }
      case PROD: {
        double r = 1.0;
        for (int j = 0; j < q.n_child; ++j) r *= v[q.child[j]];
        v[n] = r;
        break;
      }
      default: v[n] = 0.0;
    }
  }
  const double p = v[N - 1];
  if (!(p > 0.0) || !isfinite(p)) {
    ++*bad;
    return true;
  }
  logprod64_mul(L, p);
  if constexpr (!kGrad) {
    return true;
  } else {
  double ad[kMaxPdf];
  for (int n = n0; n < N; ++n) ad[n] = 0.0;
  ad[N - 1] = 1.0 / p;
  double* g = acc + 1;
  for (int n = N - 1; n >= n0; --n) {
    const PNode& q = P.node[n];
    const double* c = C + q.cofs;
    const double a = ad[n];
    const int s0 = q.slot0;
    switch (q.kind) {
      case GAUSS: {
        const double w = a * v[n];
        const double u = (x[q.col] - c[0]) * c[1];
        g[s0] += w * (u * c[1] - c[3]);
        g[s0 + 1] += w * (u * u * c[1] - c[4]);
        break;
      }
      case EXPO: {
        g[s0] += a * v[n] * (x[q.col] - c[3]);
        break;
      }
      case POISSON: {
        const double k = fmin(floor(x[q.col]), q.hi - 1.0);
        g[s0] += a * v[n] * (k * c[2] - 1.0 - c[4]);
        break;
      }
      case EXPR: {  // dv/dp_j = (df/dp_j - f dlogI/dp_j) / I, with no division by f (which may underflow)
        if constexpr (kExpr) {
          double f, df[kMaxPar];
          expr_eval(P, q, c + 1 + q.n_par, x[q.col], q.n_par, &f, df);
          const double w = a * c[0];
          for (int j = 0; j < q.n_par; ++j) g[s0 + j] += w * (df[j] - f * c[1 + j]);
        }
        break;
      }
      case GAUSSEXP: {
        const double w = a * v[n];
        const double u = (x[q.col] - c[0]) * c[1], s = c[2], it = c[3];
        double dt = s * (u - s) * it, dm = it, ds = s * it;
        if (kFull) {
          const double z = (s - u) * kSqrt1_2;
          const double R = kTwoInvSqrtPi / erfcx(z);  // exp(-z^2)/erfc(z) * 2/sqrt(pi)
          dt -= R * (-s * it * kSqrt1_2);
          dm -= R * (c[1] * kSqrt1_2);
          ds -= R * ((it + u * c[1]) * kSqrt1_2);
        }
        g[s0] += w * (dt - c[5]);
        g[s0 + 1] += w * (dm - c[6]);
        g[s0 + 2] += w * (ds - c[7]);
        break;
      }
      case CHEB: {
        const int np = q.n_par;
        const double xp = x[q.col] * c[0] - c[1];
        const double sh = v[n] / c[2];
        const double ai = a * c[2];
        double t0 = 1.0, t1 = xp;
        for (int k = 1; k <= np; ++k) {
          g[s0 + k - 1] += ai * (t1 - sh * c[3 + k - 1]);
          const double t2 = 2.0 * xp * t1 - t0;
          t0 = t1; t1 = t2;
        }
        break;
      }
      case POLY: {
        const int np = q.n_par;
        const double xv = x[q.col];
        const double sh = v[n] / c[0];
        const double ai = a * c[0];
        double xk = 1.0;
        for (int k = 1; k <= np; ++k) {
          xk *= xv;
          g[s0 + k - 1] += ai * (xk - sh * c[1 + k - 1]);
        }
        break;
      }
      case SUM: {
        const int nc = q.n_child;
        const double vl = v[q.child[nc - 1]];
        for (int j = 0; j < nc; ++j) ad[q.child[j]] += a * c[j];
        for (int j = 0; j < nc - 1; ++j) g[s0 + j] += a * (v[q.child[j]] - vl);
        break;
      }
      case PROD: {
        const int nc = q.n_child;
        for (int j = 0; j < nc; ++j) {
          double o = a;
          for (int i = 0; i < nc; ++i)
            if (i != j) o *= v[q.child[i]];
          ad[q.child[j]] += o;
        }
        break;
      }
      default: break;
    }
  }
  return true;
  }
}

constexpr int kWarps = kLanes / 32;   // warps per chunk group
constexpr int kQMax = 1 + kMaxSlots;

template <class QT, int kQueue>
struct SmemT {
  double C[kMaxConst];
  double wsum[kWarps][kQMax];
  int wbad[kWarps];
  QT queue[kWarps][kQueue];
  int qn[kWarps];
  int item;
  int last;
};
using Smem = SmemT<int, kPerLane * 32>;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ Pair warp_merge(Pair p) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Pair q{__shfl_xor_sync(0xffffffffu, p.s, o), __shfl_xor_sync(0xffffffffu, p.c, o)};
    p = merge(p, q);
  }
  return p;
}

// Chunk partials climb the set's radix-32 tree: the block that completes the
// last child of a node (arrival ticket) reduces its <= 32 children with
// two-sum merges; the block that completes the root writes the set's result.
// The tree is fixed by the set's chunk count, so the result does not depend
// on which block ran which chunk, or in which order.
template <class S>
__device__ void climb_tree(const Program& P, const Pass& pass, S& sm, int set, int chunk, int64_t n_events) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Q = pass.Q;
  const int64_t base = pass.tree_base[set];
  int64_t n_l = (n_events + kChunk - 1) / kChunk;
  int64_t lvl = 0, idx = chunk;
  while (n_l > 1) {
    const int64_t parent = idx / kRadix, first = parent * kRadix;
    const int m = (int)min((int64_t)kRadix, n_l - first);
    const int64_t pnode = base + lvl + n_l + parent;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const int t = atomicAdd(&pass.tickets[pnode], 1);
      sm.last = (t == m - 1);
      if (sm.last) pass.tickets[pnode] = 0;
    }
    __syncthreads();
    if (!sm.last) return;
    __threadfence();
    const int64_t c0 = base + lvl + first;
    for (int q = warp; q < Q; q += kWarps) {
      Pair p{0.0, 0.0};
      if (lane < m) {
        p.s = __ldcg(pass.tree + (c0 + lane) * 2 * Q + q);
        p.c = __ldcg(pass.tree + (c0 + lane) * 2 * Q + Q + q);
      }
      p = warp_merge(p);
      if (lane == 0) {
        pass.tree[pnode * 2 * Q + q] = p.s;
        pass.tree[pnode * 2 * Q + Q + q] = p.c;
      }
    }
    if (warp == 0) {
      int b = lane < m ? __ldcg(pass.tree_bad + c0 + lane) : 0;
      b = warp_sum_int(b);
      if (lane == 0) pass.tree_bad[pnode] = b;
    }
    lvl += n_l;
    n_l = (n_l + kRadix - 1) / kRadix;
    idx = parent;
  }
  // Root: this block holds the set's sums.
  __threadfence();
  __syncthreads();
  const int64_t root = base + lvl;
  if (tid == 0 && pass.pairs) {
    pass.flags[set] += __ldcg(pass.tree_bad + root);
    double* pr = pass.pairs + (size_t)set * 2 * (1 + P.n_free);
    pr[0] = __ldcg(pass.tree + root * 2 * Q);
    pr[1] = __ldcg(pass.tree + root * 2 * Q + Q);
    for (int k = 0; k < P.n_free; ++k) {
      Pair g{0.0, 0.0};
      if (pass.want_grad)
        for (int sl = 0; sl < P.n_slots; ++sl)
          if (P.slot_free[sl] == k)
            g = merge(g, {__ldcg(pass.tree + root * 2 * Q + 1 + sl), __ldcg(pass.tree + root * 2 * Q + Q + 1 + sl)});
      pr[2 + 2 * k] = g.s;
      pr[3 + 2 * k] = g.c;
    }
  } else if (tid == 0) {
    const int flag = pass.flags[set] + __ldcg(pass.tree_bad + root);
    pass.flags[set] = flag;
    double* o = pass.out + (size_t)set * (1 + P.n_free);
    const double s0 = __ldcg(pass.tree + root * 2 * Q) + __ldcg(pass.tree + root * 2 * Q + Q);
    double ext = 0.0, dext = 0.0;
    if (P.ext) extended_term(P, pass, set, (double)n_events, &ext, &dext);
    o[0] = flag ? INFINITY : ext - s0;
    if (pass.want_grad) {
      for (int k = 0; k < P.n_free; ++k) {
        double gk = 0.0;
        for (int sl = 0; sl < P.n_slots; ++sl)
          if (P.slot_free[sl] == k)
            gk += __ldcg(pass.tree + root * 2 * Q + 1 + sl) + __ldcg(pass.tree + root * 2 * Q + Q + 1 + sl);
        o[1 + k] = (k == P.ext_free ? dext : 0.0) - gk;
      }
    }
  }
}

// Writes a chunk's totals (Q values in sm.wsum[0]) to its level-0 tree node
// and climbs the tree.
template <class S>
__device__ void write_chunk(const Program& P, const Pass& pass, S& sm, int bad, int set, int chunk,
                            int64_t n_events) {
  const int tid = threadIdx.x;
  const int Q = pass.Q;
  const int64_t node = pass.tree_base[set] + chunk;
  if (tid < Q) {
    pass.tree[node * 2 * Q + tid] = sm.wsum[0][tid];
    pass.tree[node * 2 * Q + Q + tid] = 0.0;
  }
  if (tid == 0) pass.tree_bad[node] = bad;
  climb_tree(P, pass, sm, set, chunk, n_events);
}

// Writes the chunk's partial (warp sums merged in a fixed order) to its
// level-0 tree node and climbs the tree.
__device__ void finish_chunk(const Program& P, const Pass& pass, Smem& sm, double* acc, int bad, int set,
                             int chunk, int64_t n_events) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Q = pass.Q;
  for (int q = 0; q < Q; ++q) {
    const double w = warp_sum(acc[q]);
    if (lane == 0) sm.wsum[warp][q] = w;
  }
  bad = warp_sum_int(bad);
  if (lane == 0) sm.wbad[warp] = bad;
  __syncthreads();
  const int64_t node = pass.tree_base[set] + chunk;
  if (tid < Q) {
    Pair a = merge({sm.wsum[0][tid], 0.0}, {sm.wsum[1][tid], 0.0});
    Pair b = merge({sm.wsum[2][tid], 0.0}, {sm.wsum[3][tid], 0.0});
    Pair r = merge(a, b);
    pass.tree[node * 2 * Q + tid] = r.s;
    pass.tree[node * 2 * Q + Q + tid] = r.c;
  }
  if (tid == 0) pass.tree_bad[node] = sm.wbad[0] + sm.wbad[1] + sm.wbad[2] + sm.wbad[3];
  climb_tree(P, pass, sm, set, chunk, n_events);
}

// Generic fused event kernel: persistent blocks of 128 threads take 4096-event
// chunks from the work counter; lane l evaluates events l, l+128, ... of the
// chunk in order.  Events that need a node's slow path are queued per warp
// (ballot order) and evaluated after the fast pass, so the warp stays
// converged; the lane order of additions is still fixed by the data alone.
template <bool kGrad, bool kExpr>
__global__ void __launch_bounds__(kLanes) events_generic(const __grid_constant__ Program P,
                                                         const __grid_constant__ Columns cols, Pass pass) {
  __shared__ Smem sm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Q = kGrad ? 1 + P.n_slots : 1;
  const int n_items = pass.dyn ? pass.dyn[1] : pass.n_items;
  if (n_items == 0) return;
  pdl_wait();
  while (true) {
    if (tid == 0) sm.item = atomicAdd(pass.counter, 1);
    __syncthreads();
    const int it = sm.item;
    if (it >= n_items) break;
    const int set = pass.items[it].x, chunk = pass.items[it].y;
    const int64_t s_begin = pass.offsets[set], s_end = pass.offsets[set + 1];
    const int64_t base = s_begin + (int64_t)chunk * kChunk;
    for (int i = tid; i < P.n_const; i += kLanes) sm.C[i] = pass.consts[(size_t)set * P.n_const + i];
    __syncthreads();
    double acc[kQMax];
    for (int q = 0; q < kQMax; ++q) acc[q] = 0.0;
    int bad = 0, qcnt = 0;
    LogProd64 L = logprod64_init();
    double x[kMaxObs];
    for (int k = 0; k < kPerLane; ++k) {
      const int64_t e = base + tid + (int64_t)k * kLanes;
      bool slow = false;
      if (e < s_end) {
        for (int c = 0; c < P.n_obs; ++c) x[c] = load_col(cols, c, e);
        slow = !eval_generic<false, kGrad, kExpr>(P, sm.C, x, acc, L, &bad);
      }
      if (P.has_slow) {
        const unsigned b = __ballot_sync(0xffffffffu, slow);
        if (slow) sm.queue[warp][qcnt + __popc(b & ((1u << lane) - 1u))] = (int)(e - base);
        qcnt += __popc(b);
      }
    }
    __syncwarp();
    if (P.has_slow && lane == 0 && qcnt > 0 && pass.slow) atomicAdd(pass.slow, (unsigned long long)qcnt);
    for (int j = lane; j < qcnt; j += 32) {
      const int64_t e = base + sm.queue[warp][j];
      for (int c = 0; c < P.n_obs; ++c) x[c] = load_col(cols, c, e);
      eval_generic<true, kGrad, kExpr>(P, sm.C, x, acc, L, &bad);
    }
    acc[0] += logprod64_log(L);
    (void)Q;
    finish_chunk(P, pass, sm, acc, bad, set, chunk, s_end - s_begin);
    __syncthreads();
  }
}

// Sums v[0..N) over the lanes of a warp with the xor butterfly (offsets 16,
// 8, 4, 2, 1).  At each of the first log2(N) levels a lane pair splits the
// values in two halves and each lane adds one half (reduce-scatter), so a
// lane adds N/2 + N/4 + ... values instead of 5 N; every value still gets the
// plain butterfly's pairwise tree (float-float addition is commutative and
// deterministic).  Afterwards v[0] of lane l holds the sum of value index
// ff_lane_index<N>(l), on every lane with that index.
template <int N>
__device__ __forceinline__ void warp_ff_reduce(ff* v, int lane) {
  static_assert(N == 1 || N == 2 || N == 4 || N == 8 || N == 16, "power of two up to 16");
  int h = N / 2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (h >= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int j = 0; j < N / 2; ++j) {
        if (j < h) {
          const ff send = up ? v[j] : v[j + h];
          const ff keep = up ? v[j + h] : v[j];
          const ff r = {__shfl_xor_sync(0xffffffffu, send.hi, o), __shfl_xor_sync(0xffffffffu, send.lo, o)};
          v[j] = ff_add(keep, r);
        }
      }
      h >>= 1;
    } else {
      const ff r = {__shfl_xor_sync(0xffffffffu, v[0].hi, o), __shfl_xor_sync(0xffffffffu, v[0].lo, o)};
      v[0] = ff_add(v[0], r);
    }
  }
}
template <int N>
__device__ __forceinline__ int ff_lane_index(int lane) {
  int idx = 0, h = N / 2;
#pragma unroll
  for (int o = 16; o > 0 && h >= 1; o >>= 1, h >>= 1) idx += (lane & o) ? h : 0;
  return idx;
}
// Lanes whose bits below the halving levels are zero (one writer per index).
template <int N>
__device__ __forceinline__ bool ff_lane_writes(int lane) {
  constexpr int levels = N >= 16 ? 4 : N >= 8 ? 3 : N >= 4 ? 2 : N >= 2 ? 1 : 0;
  return (lane & ((32 >> levels) - 1)) == 0;
}
__host__ __device__ constexpr int pow2_at_least(int n) { return n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : n <= 8 ? 8 : 16; }

// Float-float fused event kernel of a specialised shape.  Persistent blocks
// of 128 threads take work units from the counter: unit u is part u % 4 of
// work item u / 4 (a quarter of a 4096-event chunk, 8 events per lane), so
// the last round of units is short.  Per lane the shape's moments are summed
// in float-float; events in the decay resolution region are queued per warp
// (ballot order) and evaluated after the fast pass by all the block's
// threads; events outside the
// float-float range take the FP64 interpreter (FP64 sums).  At the end of a
// part the warps' moments are merged in fixed order and stored as the part's
// record; the block that completes the chunk's last part (arrival ticket)
// merges the four records in part order, maps the moments to (sum log p,
// slot gradients) with the set's matrix K and climbs the reduction tree.
// Every sum has a fixed order, so the result does not depend on the launch.
template <int kShape, bool kGrad, bool kF32>
__global__ void __launch_bounds__(kLanes, ff_min_blocks(kShape)) events_ff(const __grid_constant__ Program P,
                                                                  const __grid_constant__ Columns cols, Pass pass) {
  constexpr int NA = kGrad ? ff_nacc(kShape) : 1;
  constexpr int NP = pow2_at_least(NA);
  constexpr int NAK = ff_nacc(kShape);
  const int parts = pass.parts;
  const int kPartK = kPerLane / parts;
  __shared__ SmemT<short, kPerLane * 32> sm;
  __shared__ FFTables T;
  __shared__ float kc[kFFConst];
  __shared__ ff wacc[kWarps][16];
  __shared__ unsigned fbmask[kLanes];  // per lane: its events (bit k) that need the FP64 path
  // PROD3: events whose decay factor alone needs the FP64 path (their mass
  // and angle factors were summed in the fast pass)
  __shared__ unsigned fbmask_f[kShape == SHAPE_PROD3 ? kLanes : 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Q = pass.Q;
  const int n_items = pass.dyn ? pass.dyn[1] : pass.n_items;
  if (n_items == 0) return;
  ff_load_tables(T);
  int col[3];
  if (kShape == SHAPE_PROD3) {
    col[0] = P.node[0].col; col[1] = P.node[3].col; col[2] = P.node[6].col;
  } else {
    col[0] = col[1] = col[2] = P.node[0].col;
  }
  const int n_units = n_items * parts;
  int kc_set = -1, c_set = -1;  // sets whose constants the block holds (block-uniform)
  pdl_wait();  // K1 has reset the counter and written the constants
  // One unit of lookahead: thread 0 claims the next unit while the block
  // works on the current one, so the claim's round trip is hidden.
  int next_u = tid == 0 ? atomicAdd(pass.counter, 1) : 0;
  while (true) {
    if (tid == 0) sm.item = next_u;
    __syncthreads();
    const int u = sm.item;
    if (u >= n_units) break;
    if (tid == 0) next_u = atomicAdd(pass.counter, 1);
    const int it = u / parts, part = u % parts;
    const int set = pass.items[it].x, chunk = pass.items[it].y;
    const int64_t s_begin = pass.offsets[set], s_end = pass.offsets[set + 1];
    const int64_t base = s_begin + (int64_t)chunk * kChunk;
    if (set != kc_set) {
      for (int i = tid; i < kFFConst; i += kLanes) kc[i] = pass.ffc[(size_t)set * kFFConst + i];
      kc_set = set;
    }
    fbmask[tid] = 0u;
    if (kShape == SHAPE_PROD3) fbmask_f[tid] = 0u;
    __syncthreads();
    ff acc[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) acc[j] = {0.0f, 0.0f};
    LogProd lpd = logprod_init();
    unsigned myslow = 0u, myfb = 0u;  // the lane's events (bit k) for the slow pass / the FP64 path
    const int k0 = part * kPartK;
    // events of the chunk present (32-bit offsets within the chunk); the
    // next event's observables are loaded one iteration ahead
    const int rem = (int)(s_end - base < (int64_t)kChunk ? s_end - base : (int64_t)kChunk);
    int off = tid + k0 * kLanes;
    FFRaw<kShape> nxt;
    if (off < rem) nxt = ff_load_raw<kShape, kF32>(cols, col, base + off);
#pragma unroll 1
    for (int k = k0; k < k0 + kPartK; ++k, off += kLanes) {
      const FFIn<kShape> cur = ff_split_in<kShape, kF32>(cols, col, nxt);
      if (k + 1 < k0 + kPartK && off + kLanes < rem)
        nxt = ff_load_raw<kShape, kF32>(cols, col, base + off + kLanes);
      int st = 0;
      if (off < rem) st = ff_event<kShape, kGrad, false, kF32>(T, kc, cur, acc, lpd);
      myslow |= (st == 1 ? 1u : 0u) << k;
      myfb |= (st == 2 ? 1u : 0u) << k;
    }
    if constexpr (kShape == SHAPE_PROD3 && kGrad) {
      // moment 13: the lane's events summed in float-float (those present
      // in its part, less the ones the FP64 path takes whole)
      const int nv = min(max((rem - tid + kLanes - 1) / kLanes - k0, 0), kPartK);
      acc[13] = {(float)(nv - __popc(myfb)), 0.0f};
    }
    // The block's slow events form one queue, thread by thread and each
    // thread's in event order (an exclusive scan of the per-thread counts
    // places them), shared out over all its threads (entry j to thread j mod
    // 128), so only the last round of the queue leaves lanes idle.
    short* const queue = &sm.queue[0][0];
    const int ns = __popc(myslow);
    int incl = ns;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) sm.qn[warp] = incl;
    __syncthreads();
    int pos = incl - ns;
    for (int w = 0; w < warp; ++w) pos += sm.qn[w];
    const int qt = sm.qn[0] + sm.qn[1] + sm.qn[2] + sm.qn[3];
    for (unsigned mk = myslow; mk; mk &= mk - 1u) queue[pos++] = (short)(tid + (__ffs(mk) - 1) * kLanes);
    __syncthreads();
    if (tid == 0 && qt > 0 && pass.slow) atomicAdd(pass.slow, (unsigned long long)qt);
    for (int j = tid; j < qt; j += kLanes) {
      const int off = queue[j];
      if (ff_event<kShape, kGrad, true, kF32>(T, kc, ff_load<kShape, kF32>(cols, col, base + off), acc, lpd) == 2)
        atomicOr(kShape == SHAPE_PROD3 ? &fbmask_f[off % kLanes] : &fbmask[off % kLanes],
                 1u << (off / kLanes));  // owner lane, event bit
    }
    __syncthreads();
    myfb |= fbmask[tid];
    unsigned myfb_f = kShape == SHAPE_PROD3 ? fbmask_f[tid] : 0u;
    // FP64 fallback for events outside the float-float range: each lane
    // evaluates its own flagged events in event order.
    double acc64[kQMax];
    int bad = 0;
    const bool any_fb = __syncthreads_or((myfb | myfb_f) != 0u);
    if (any_fb) {
      if (set != c_set) {
        for (int i = tid; i < P.n_const; i += kLanes) sm.C[i] = pass.consts[(size_t)set * P.n_const + i];
        c_set = set;
      }
      __syncthreads();
      for (int q = 0; q < kQMax; ++q) acc64[q] = 0.0;
      double x[kMaxObs];
      LogProd64 L64 = logprod64_init();
      while (myfb) {
        const int k = __ffs(myfb) - 1;
        myfb &= myfb - 1u;
        const int64_t e = base + tid + (int64_t)k * kLanes;
        for (int c = 0; c < P.n_obs; ++c) x[c] = load_col(cols, c, e);
        eval_generic<true, kGrad>(P, sm.C, x, acc64, L64, &bad);
      }
      while (myfb_f) {  // PROD3: the decay factor's sub-program, program nodes 3..5
        const int k = __ffs(myfb_f) - 1;
        myfb_f &= myfb_f - 1u;
        const int64_t e = base + tid + (int64_t)k * kLanes;
        for (int c = 0; c < P.n_obs; ++c) x[c] = load_col(cols, c, e);
        eval_generic<true, kGrad>(P, sm.C, x, acc64, L64, &bad, 3, 6);
      }
      acc64[0] += logprod64_log(L64);
    }
    // sum log p of the lane's events from their product, then the part's
    // moments: reduce-scatter butterfly, then the warps in order
    {
      bool lok = true;
      acc[0] = logprod_log(T, lpd, lok);  // m in [1, 2): always in range
    }
    warp_ff_reduce<NP>(acc, lane);
    if (ff_lane_writes<NP>(lane)) wacc[warp][ff_lane_index<NP>(lane)] = acc[0];
    if (any_fb) {
      for (int q = 0; q < Q; ++q) {
        const double w = warp_sum(acc64[q]);
        if (lane == 0) sm.wsum[warp][q] = w;
      }
      bad = warp_sum_int(bad);
      if (lane == 0) sm.wbad[warp] = bad;
    }
    __syncthreads();
    const int64_t leaf = pass.tree_base[set] + chunk;
    const int64_t rec = leaf * parts + part;
    if (tid < NA) {
      const ff M = ff_add(ff_add(wacc[0][tid], wacc[1][tid]), ff_add(wacc[2][tid], wacc[3][tid]));
      pass.part_m[rec * kPartFloats + 2 * tid] = M.hi;
      pass.part_m[rec * kPartFloats + 2 * tid + 1] = M.lo;
    }
    if (any_fb && tid < Q) {
      const Pair a = merge({sm.wsum[0][tid], 0.0}, {sm.wsum[1][tid], 0.0});
      const Pair b = merge({sm.wsum[2][tid], 0.0}, {sm.wsum[3][tid], 0.0});
      const Pair r = merge(a, b);
      pass.part_fb[rec * Q + tid] = r.s + r.c;
    }
    if (tid == 0)
      pass.part_info[rec] = (any_fb ? 1 : 0) | ((any_fb ? sm.wbad[0] + sm.wbad[1] + sm.wbad[2] + sm.wbad[3] : 0) << 1);
    if (tid < 2 * 32) __threadfence();  // the record's writers (tid < NA, Q <= 33)
    __syncthreads();
    if (tid == 0) {
      const int t = atomicAdd(&pass.tickets[leaf], 1);
      sm.last = (t == parts - 1);
      if (sm.last) pass.tickets[leaf] = 0;
    }
    __syncthreads();
    if (!sm.last) continue;
    __threadfence();
    // The chunk: parts merged in part order, out_q = sum_j K[q][j] M_j.
    double v = 0.0;
    int info[kMaxParts];
#pragma unroll
    for (int p = 0; p < kMaxParts; ++p) info[p] = p < parts ? __ldcg(pass.part_info + leaf * parts + p) : 0;
    if (tid < Q) {
      const float* K = kc + ff_koff(kShape);
      const float* pm = pass.part_m + leaf * parts * kPartFloats;
      ff out = {0.0f, 0.0f};
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        ff Mj = {__ldcg(pm + 2 * j), __ldcg(pm + 2 * j + 1)};
        for (int p = 1; p < parts; ++p)
          Mj = ff_add(Mj, ff{__ldcg(pm + p * kPartFloats + 2 * j), __ldcg(pm + p * kPartFloats + 2 * j + 1)});
        out = ff_add(out, ff_mul(ff{K[2 * (tid * NAK + j)], K[2 * (tid * NAK + j) + 1]}, Mj));
      }
      v = ff_to_double(out);
#pragma unroll
      for (int p = 0; p < kMaxParts; ++p)
        if (info[p] & 1) v += __ldcg(pass.part_fb + (leaf * parts + p) * Q + tid);
    }
    int bad_all = 0;
#pragma unroll
    for (int p = 0; p < kMaxParts; ++p) bad_all += info[p] >> 1;
    __syncthreads();
    if (tid < Q) sm.wsum[0][tid] = v;
    __syncthreads();
    write_chunk(P, pass, sm, bad_all, set, chunk, s_end - s_begin);
    __syncthreads();
  }
}

}  // namespace

void launch_param_point(const Program& P, const Pass& pass, cudaStream_t st) {
  note_launches(1, st);
  if (pass.n_active > 0 && P.has_expr) {
    param_point_block_kernel<true><<<pass.n_active, kK1Warps * 32, 0, st>>>(P, pass);
    return;
  }
  // In the rounds of a device-resident fit (dyn counts) nothing runs beside
  // K1, and a block per set finishes sooner for any number of sets.
  if (pass.n_active > 0 && (pass.n_active <= kBlockK1MaxSets || pass.dyn)) {
    param_point_block_kernel<false><<<pass.n_active, kK1Warps * 32, 0, st>>>(P, pass);
    return;
  }
  // two-warp blocks: one fits in the registers that an SM full of event
  // kernel blocks leaves free, so the K1 of a pass on another stream runs
  // beside an event pass instead of waiting for its blocks to drain
  const int threads = 64;
  const int blocks = (pass.n_active + threads - 1) / threads;
  param_point_kernel<<<blocks > 0 ? blocks : 1, threads, 0, st>>>(P, pass);
}

bool launch_supports_threads(Shape shape, int threads) {
  (void)shape;
  return threads == kLanes;
}

template <int kShape>
const void* ff_kernel(bool grad) {
  return grad ? (const void*)events_ff<kShape, true, false> : (const void*)events_ff<kShape, false, false>;
}

const void* event_kernel(Shape shape, bool grad) {
  switch (shape) {
    case SHAPE_SUM_GAUSSEXP_CHEB2: return ff_kernel<SHAPE_SUM_GAUSSEXP_CHEB2>(grad);
    case SHAPE_SUM_GAUSS_POLY1: return ff_kernel<SHAPE_SUM_GAUSS_POLY1>(grad);
    case SHAPE_PROD3: return ff_kernel<SHAPE_PROD3>(grad);
    default: return grad ? (const void*)events_generic<true, false> : (const void*)events_generic<false, false>;
  }
}

bool launch_fits(Shape shape, int threads, int blocks_per_sm) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, event_kernel(shape, true), threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return blocks_per_sm <= 4;
  }
  return blocks_per_sm <= n;
}

// Launches an event kernel as a programmatic dependent of the stream's
// previous kernel (K1).
template <class... Args>
void launch_dependent(void (*kernel)(Args...), int grid, cudaStream_t st, const Program& P, const Columns& cols,
                      const Pass& pass) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kLanes);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, P, cols, pass);
}

// The float-float kernel of a shape, with or without the gradient, for
// datasets whose columns are all FP32 or not.
template <int kShape>
void launch_ff(bool grad, bool all_f32, int grid, cudaStream_t st, const Program& P, const Columns& cols,
               const Pass& pass) {
  if (grad && all_f32) launch_dependent(events_ff<kShape, true, true>, grid, st, P, cols, pass);
  else if (grad) launch_dependent(events_ff<kShape, true, false>, grid, st, P, cols, pass);
  else if (all_f32) launch_dependent(events_ff<kShape, false, true>, grid, st, P, cols, pass);
  else launch_dependent(events_ff<kShape, false, false>, grid, st, P, cols, pass);
}

void launch_events(const Program& P, Shape shape, const Columns& cols, const Pass& pass, int threads,
                   int blocks_per_sm, int n_sm, cudaStream_t st) {
  (void)threads;
  if (pass.n_items == 0) return;
  const int bps = blocks_per_sm > 0 ? blocks_per_sm : 8;
  int grid = n_sm * bps;
  const Shape sh = (pass.ff_shape != SHAPE_GENERIC && pass.ffc) ? shape : SHAPE_GENERIC;
  const int64_t units = sh == SHAPE_GENERIC ? (int64_t)pass.n_items : (int64_t)pass.n_items * pass.parts;
  if (grid > units) grid = (int)units;
  note_launches(1, st);
  timing_begin(st);
  bool all_f32 = true;
  for (int c = 0; c < P.n_obs; ++c) all_f32 = all_f32 && cols.is_f32[c];
  switch (sh) {
    case SHAPE_SUM_GAUSSEXP_CHEB2: launch_ff<SHAPE_SUM_GAUSSEXP_CHEB2>(pass.want_grad, all_f32, grid, st, P, cols, pass); break;
    case SHAPE_SUM_GAUSS_POLY1: launch_ff<SHAPE_SUM_GAUSS_POLY1>(pass.want_grad, all_f32, grid, st, P, cols, pass); break;
    case SHAPE_PROD3: launch_ff<SHAPE_PROD3>(pass.want_grad, all_f32, grid, st, P, cols, pass); break;
    default:
      if (P.has_expr && pass.want_grad) launch_dependent(events_generic<true, true>, grid, st, P, cols, pass);
      else if (P.has_expr) launch_dependent(events_generic<false, true>, grid, st, P, cols, pass);
      else if (pass.want_grad) launch_dependent(events_generic<true, false>, grid, st, P, cols, pass);
      else launch_dependent(events_generic<false, false>, grid, st, P, cols, pass);
  }
  timing_end(st);
}

}  // namespace rf
