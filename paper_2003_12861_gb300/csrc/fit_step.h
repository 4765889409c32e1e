// One set's quasi-Newton state machine, shared by the host fit driver
// (fit.cpp) and the device-resident step (fit_dev.cu, the batched fit's
// tail).  The paper does not describe its minimiser; this is BFGS (Nocedal &
// Wright, Numerical Optimization, 2nd ed., Alg. 6.1) with the strong-Wolfe
// line search of their Alg. 3.5 / 3.6 (cubic interpolation in the zoom, eq.
// 3.59), plus Hager & Zhang's approximate Wolfe conditions (SIAM J. Optim.
// 16, 2005) near a minimum.
//
// Both sides must produce the same trial points bit for bit: the code below
// uses only correctly rounded operations (+ - * / sqrt, fma, comparisons,
// rint) and its own sine and cosine, and both translation units that
// include it are compiled without floating-point contraction (host
// -ffp-contract=off, device --fmad=false), so every expression rounds the
// same way on the CPU and on the GPU; the fused multiply-adds are written
// out (fma), which halves the FP64 instructions of the sums on the device.
#pragma once

#include <math.h>
#include <stdint.h>

#include "rf.h"

#if defined(__CUDACC__)
#define RF_HD __host__ __device__ __forceinline__
#else
#define RF_HD inline
#endif

namespace rf {
namespace qn {

constexpr double kC1 = 1e-4, kC2 = 0.9;
// Near a minimum the decrease a step can make falls below the precision of
// the NLL itself (float-float event sums: ~1e-14 of sum |log p|), and the
// sufficient-decrease test turns into noise.  A step is then also accepted
// under the approximate Wolfe conditions: the curvature condition on the
// directional derivative, and a value no more than kEpsF |f| above the start.
constexpr double kEpsF = 1e-12;
constexpr int kMaxLineTrials = 25;

enum Phase : int32_t { INIT = 0, BRACKET = 1, ZOOM = 2, DONE = 3 };

// Scalar state of one set's fit.
struct State {
  int32_t phase, evals, status, first_step, reset_once, trials;
  double f, d0;                        // f(x), g.p
  double a_prev, f_prev, d_prev, a_cur;
  double a_lo, f_lo, d_lo, a_hi, f_hi, d_hi;
};

// Vectors of one set's fit (P each; H is P x P, row-major): the accepted
// point, its gradient, the inverse-Hessian estimate, the direction, the
// gradient at the zoom's low end, the point to evaluate next, and scratch.
struct Vecs {
  double *x, *g, *H, *p, *g_lo, *trial, *w_s, *w_y, *w_hy, *w_r;
};

RF_HD double inf_value() { return HUGE_VAL; }
RF_HD bool finite(double v) {
#if defined(__CUDA_ARCH__)
  return isfinite(v);
#else
  return std::isfinite(v);
#endif
}
RF_HD double dmin(double a, double b) { return b < a ? b : a; }
RF_HD double dmax(double a, double b) { return a < b ? b : a; }

RF_HD State initial_state() {
  State c{};
  c.phase = INIT;
  c.status = RF_E_NOT_CONVERGED;
  c.first_step = 1;
  c.f = inf_value();
  return c;
}

// The loops over vector and matrix elements take their indices from a
// policy: SeqLoop runs them in order (the host, or one device thread); the
// device step runs them across the lanes of a warp (each element computed
// by one lane with the same operations, between warp barriers).  Sums over
// elements are always taken in order, by every lane alike, so both give
// the same bits.
struct SeqLoop {
  RF_HD static int first() { return 0; }
  RF_HD static int step() { return 1; }
  RF_HD static void sync() {}
};

RF_HD double dot(const double* a, const double* b, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s = fma(a[i], b[i], s);
  return s;
}

// r = M v (M n x n row-major), each row summed in order.
template <class L>
RF_HD void mat_vec(const double* M, const double* v, double* r, int n) {
  L::sync();
  for (int i = L::first(); i < n; i += L::step()) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s = fma(M[i * n + j], v[j], s);
    r[i] = s;
  }
  L::sync();
}

// sin x and cos x: Cody & Waite's reduction by the nearest multiple k of
// pi/2 (pi/2 split into three parts, the first two with trailing zero bits
// so that k times them is exact for |k| < 2^20), then the Taylor series of
// sin and cos on |r| <= pi/4 to degree 19 and 20 (truncation below 1e-21)
// and the quadrant of k.  Accurate to a few units in the last place for
// |x| < 1e6; used for the bound transform on both host and device so that
// both compute the same bits.
RF_HD void sin_cos(double x, double* s_out, double* c_out) {
  // pi/2 = kPio2_1 + kPio2_2 + kPio2_3: the first two are pi/2 and its
  // remainder rounded to 33 significant bits, the third the rounded rest
  // (computed at 300 bits)
  const double kTwoOverPi = 0x1.45f306dc9c883p-1;
  const double kPio2_1 = 0x1.921fb544p+0;
  const double kPio2_2 = 0x1.0b4611a6p-34;
  const double kPio2_3 = 0x1.3198a2e037073p-69;
  const double k = rint(x * kTwoOverPi);
  const double r = ((x - k * kPio2_1) - k * kPio2_2) - k * kPio2_3;
  const double r2 = r * r;
  // 1/n! (correctly rounded) for the sine (odd n from 3) and cosine (even n
  // from 4)
  double ps = 0x1.2f49b46814157p-57;  // 1/19!
  ps = fma(ps, r2, -0x1.952c77030ad4ap-49);  // 1/17!
  ps = fma(ps, r2, 0x1.ae7f3e733b81fp-41);  // 1/15!
  ps = fma(ps, r2, -0x1.6124613a86d09p-33);  // 1/13!
  ps = fma(ps, r2, 0x1.ae64567f544e4p-26);  // 1/11!
  ps = fma(ps, r2, -0x1.71de3a556c734p-19);  // 1/9!
  ps = fma(ps, r2, 0x1.a01a01a01a01ap-13);  // 1/7!
  ps = fma(ps, r2, -0x1.1111111111111p-7);  // 1/5!
  ps = fma(ps, r2, 0x1.5555555555555p-3);  // 1/3!
  const double sn = fma(-(r * r2), ps, r);
  double pc = 0x1.e542ba4020225p-62;  // 1/20!
  pc = fma(pc, r2, -0x1.6827863b97d97p-53);  // 1/18!
  pc = fma(pc, r2, 0x1.ae7f3e733b81fp-45);  // 1/16!
  pc = fma(pc, r2, -0x1.93974a8c07c9dp-37);  // 1/14!
  pc = fma(pc, r2, 0x1.1eed8eff8d898p-29);  // 1/12!
  pc = fma(pc, r2, -0x1.27e4fb7789f5cp-22);  // 1/10!
  pc = fma(pc, r2, 0x1.a01a01a01a01ap-16);  // 1/8!
  pc = fma(pc, r2, -0x1.6c16c16c16c17p-10);  // 1/6!
  pc = fma(pc, r2, 0x1.5555555555555p-5);  // 1/4!
  const double cs = fma(r2 * r2, pc, fma(-0.5, r2, 1.0));
  const int q = (int)(long long)k & 3;
  double s = sn, c = cs;
  if (q == 1) {
    s = cs;
    c = -sn;
  } else if (q == 2) {
    s = -sn;
    c = -cs;
  } else if (q == 3) {
    s = -cs;
    c = sn;
  }
  *s_out = s;
  *c_out = c;
}

// theta and d theta / d x at the internal point x: a bounded parameter is
// theta = lo + (hi - lo)(sin x + 1)/2 (the transform MINUIT documents), an
// unbounded one is used as is.  th or jc may be null.
template <class L = SeqLoop>
RF_HD void to_theta_jac(int P, const double* lo, const double* hi, const char* bounded, const double* x,
                        double* th, double* jc) {
  L::sync();
  for (int k = L::first(); k < P; k += L::step()) {
    if (!bounded[k]) {
      if (th) th[k] = x[k];
      if (jc) jc[k] = 1.0;
      continue;
    }
    double sn, cs;
    sin_cos(x[k], &sn, &cs);
    if (th) th[k] = lo[k] + (hi[k] - lo[k]) * (sn + 1.0) * 0.5;
    if (jc) jc[k] = (hi[k] - lo[k]) * 0.5 * cs;
  }
  L::sync();
}

// Minimiser of the cubic through (a, fa, da), (b, fb, db) (N&W eq. 3.59),
// kept inside the middle 80 % of [a, b]; bisection when the data are unusable.
RF_HD double cubic_step(double a, double fa, double da, double b, double fb, double db) {
  const double lo = dmin(a, b), hi = dmax(a, b), w = hi - lo;
  const double mid = 0.5 * (a + b);
  if (!finite(fa) || !finite(fb) || !finite(da) || !finite(db)) return mid;
  const double d1 = da + db - 3.0 * (fa - fb) / (a - b);
  const double disc = d1 * d1 - da * db;
  if (disc < 0.0) return mid;
  const double d2 = copysign(sqrt(disc), b - a);
  const double den = db - da + 2.0 * d2;
  if (den == 0.0) return mid;
  const double t = b - (b - a) * (db + d2 - d1) / den;
  if (!finite(t)) return mid;
  return dmin(hi - 0.1 * w, dmax(lo + 0.1 * w, t));
}

template <class L>
RF_HD void copy_vec(double* dst, const double* src, int n) {
  L::sync();
  for (int k = L::first(); k < n; k += L::step()) dst[k] = src[k];
  L::sync();
}

template <class L>
RF_HD void set_trial(int P, State& c, const Vecs& v, double a) {
  c.a_cur = a;
  L::sync();
  for (int k = L::first(); k < P; k += L::step()) v.trial[k] = fma(a, v.p[k], v.x[k]);
  L::sync();
}

template <class L>
RF_HD void reset_hessian(int P, const Vecs& v) {
  L::sync();
  for (int e = L::first(); e < P * P; e += L::step()) v.H[e] = e / P == e % P ? 1.0 : 0.0;
  L::sync();
}

// New search direction p = -H g; resets H when it is not a descent direction.
template <class L>
RF_HD void new_direction(int P, State& c, const Vecs& v) {
  mat_vec<L>(v.H, v.g, v.w_r, P);
  L::sync();
  for (int k = L::first(); k < P; k += L::step()) v.p[k] = -v.w_r[k];
  L::sync();
  c.d0 = dot(v.g, v.p, P);
  if (!(c.d0 < 0.0)) {
    reset_hessian<L>(P, v);
    L::sync();
    for (int k = L::first(); k < P; k += L::step()) v.p[k] = -v.g[k];
    L::sync();
    c.first_step = 1;
    c.d0 = dot(v.g, v.p, P);
  }
  double a1 = 1.0;
  if (c.first_step) {  // keep the first step of a fresh H within 0.5 (internal units)
    double pm = 0.0;
    for (int k = 0; k < P; ++k) pm = dmax(pm, fabs(v.p[k]));
    if (pm > 0.0) a1 = dmin(1.0, 0.5 / pm);
  }
  c.a_prev = 0.0;
  c.f_prev = c.f;
  c.d_prev = c.d0;
  c.trials = 0;
  c.phase = BRACKET;
  set_trial<L>(P, c, v, a1);
}

// EDM = g^T H g / 2, from the rows of H g.
template <class L>
RF_HD double edm(int P, const Vecs& v) {
  mat_vec<L>(v.H, v.g, v.w_r, P);
  double e = 0.0;
  for (int i = 0; i < P; ++i) e = fma(0.5 * v.g[i], v.w_r[i], e);
  return e;
}

// Accept the step to alpha with value fa and gradient ga.
template <class L>
RF_HD void accept(int P, State& c, const Vecs& v, double a, double fa, const double* ga, double tol,
                  int max_evals) {
  double* s = v.w_s;
  double* y = v.w_y;
  L::sync();
  for (int k = L::first(); k < P; k += L::step()) {
    s[k] = a * v.p[k];
    y[k] = ga[k] - v.g[k];
  }
  L::sync();
  const double sy = dot(s, y, P);
  if (c.first_step && sy > 0.0) {  // N&W eq. 6.20
    const double sc = sy / dot(y, y, P);
    L::sync();
    for (int e = L::first(); e < P * P; e += L::step()) v.H[e] *= sc;
    L::sync();
  }
  c.first_step = 0;
  if (sy > 1e-300) {
    const double rho = 1.0 / sy;
    double* Hy = v.w_hy;
    mat_vec<L>(v.H, y, Hy, P);
    const double yHy = dot(y, Hy, P);
    const double b = rho * rho * yHy + rho;
    L::sync();
    for (int e = L::first(); e < P * P; e += L::step()) {
      const int i = e / P, j = e % P;
      const double u = fma(Hy[i], s[j], s[i] * Hy[j]);
      v.H[e] = fma(b * s[i], s[j], fma(-rho, u, v.H[e]));
    }
    L::sync();
  }
  L::sync();
  for (int k = L::first(); k < P; k += L::step()) {
    v.x[k] += s[k];
    v.g[k] = ga[k];
  }
  L::sync();
  c.f = fa;
  if (edm<L>(P, v) < tol) {
    c.status = RF_OK;
    c.phase = DONE;
    return;
  }
  if (c.evals >= max_evals) {
    c.phase = DONE;
    return;
  }
  new_direction<L>(P, c, v);
}

template <class L>
RF_HD void line_failed(int P, State& c, const Vecs& v, int max_evals) {
  if (!c.reset_once && c.evals < max_evals) {  // one restart from steepest descent
    c.reset_once = 1;
    reset_hessian<L>(P, v);
    c.first_step = 1;
    new_direction<L>(P, c, v);
    return;
  }
  c.phase = DONE;
}

// Hager-Zhang's approximate Wolfe conditions at a trial point (d0 < 0).
RF_HD bool approx_wolfe(const State& c, double fa, double da) {
  return finite(fa) && finite(da) && fa <= c.f + kEpsF * fabs(c.f) && da >= kC2 * c.d0 &&
         da <= (2.0 * kC1 - 1.0) * c.d0;
}

// With H = I the EDM is |g|^2/2: a start at the minimum is already done.
RF_HD bool edm_identity_small(int P, State& c, const Vecs& v, double tol) {
  if (0.5 * dot(v.g, v.g, P) < tol * 1e-6) {
    c.status = RF_OK;
    c.phase = DONE;
    return true;
  }
  return false;
}

// Deliver f and the gradient (internal coordinates) at the last trial point;
// leaves the next trial point in v.trial unless the fit is done.  ga may be
// any buffer but v's own vectors.
template <class L = SeqLoop>
RF_HD void deliver(int P, State& c, const Vecs& v, double fa, const double* ga, double tol, int max_evals) {
  ++c.evals;
  if (c.phase == INIT) {
    copy_vec<L>(v.x, v.trial, P);
    if (!finite(fa)) {
      c.status = RF_E_DOMAIN;
      c.phase = DONE;
      return;
    }
    c.f = fa;
    copy_vec<L>(v.g, ga, P);
    if (edm_identity_small(P, c, v, tol)) return;
    new_direction<L>(P, c, v);
    return;
  }
  const double a = c.a_cur;
  const double da = finite(fa) ? dot(ga, v.p, P) : (double)NAN;
  ++c.trials;
  const bool too_many = c.trials >= kMaxLineTrials || c.evals >= max_evals;
  if (approx_wolfe(c, fa, da)) {
    accept<L>(P, c, v, a, fa, ga, tol, max_evals);
    return;
  }
  if (c.phase == BRACKET) {
    if (!(fa <= c.f + kC1 * a * c.d0) || (c.trials > 1 && fa >= c.f_prev)) {
      c.a_lo = c.a_prev; c.f_lo = c.f_prev; c.d_lo = c.d_prev;
      if (c.a_prev == 0.0) copy_vec<L>(v.g_lo, v.g, P);
      c.a_hi = a; c.f_hi = fa; c.d_hi = da;
      c.phase = ZOOM;
    } else if (fabs(da) <= -kC2 * c.d0) {
      accept<L>(P, c, v, a, fa, ga, tol, max_evals);
      return;
    } else if (da >= 0.0) {
      c.a_lo = a; c.f_lo = fa; c.d_lo = da;
      copy_vec<L>(v.g_lo, ga, P);
      c.a_hi = c.a_prev; c.f_hi = c.f_prev; c.d_hi = c.d_prev;
      c.phase = ZOOM;
    } else {
      c.a_prev = a; c.f_prev = fa; c.d_prev = da;
      copy_vec<L>(v.g_lo, ga, P);
      if (too_many) {
        accept<L>(P, c, v, a, fa, ga, tol, max_evals);  // sufficient decrease holds here
        return;
      }
      set_trial<L>(P, c, v, 2.0 * a);  // expand the bracket
      return;
    }
  } else {  // ZOOM
    if (!(fa <= c.f + kC1 * a * c.d0) || fa >= c.f_lo) {
      c.a_hi = a; c.f_hi = fa; c.d_hi = da;
    } else {
      if (fabs(da) <= -kC2 * c.d0) {
        accept<L>(P, c, v, a, fa, ga, tol, max_evals);
        return;
      }
      if (da * (c.a_hi - c.a_lo) >= 0.0) {
        c.a_hi = c.a_lo; c.f_hi = c.f_lo; c.d_hi = c.d_lo;
      }
      c.a_lo = a; c.f_lo = fa; c.d_lo = da;
      copy_vec<L>(v.g_lo, ga, P);
    }
  }
  if (too_many) {
    if (c.a_lo > 0.0) accept<L>(P, c, v, c.a_lo, c.f_lo, v.g_lo, tol, max_evals);
    else line_failed<L>(P, c, v, max_evals);
    return;
  }
  set_trial<L>(P, c, v, finite(c.f_hi) ? cubic_step(c.a_lo, c.f_lo, c.d_lo, c.a_hi, c.f_hi, c.d_hi)
                                       : 0.5 * (c.a_lo + c.a_hi));
}

// A set's record in the device-resident rounds: its State, then x, g, p,
// g_lo, trial, the Jacobian of the transform at trial (P each), then H.
constexpr int kTailMaxP = 16;
constexpr int kStateWords = (int)((sizeof(State) + sizeof(double) - 1) / sizeof(double));
RF_HD int tail_record_words(int P) { return kStateWords + 6 * P + P * P; }
struct TailView {
  State* c;
  double *x, *g, *p, *g_lo, *trial, *jc, *H;
};
RF_HD TailView tail_view(double* rec, int P) {
  TailView t;
  t.c = reinterpret_cast<State*>(rec);
  double* v = rec + kStateWords;
  t.x = v;
  t.g = v + P;
  t.p = v + 2 * P;
  t.g_lo = v + 3 * P;
  t.trial = v + 4 * P;
  t.jc = v + 5 * P;
  t.H = v + 6 * P;
  return t;
}

}  // namespace qn
}  // namespace rf
