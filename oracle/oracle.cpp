// Oracle for the batched unbinned-likelihood hot path of "Making RooFit Ready
// for Run 3" (Hageboeck & Moneta, ACAT 2019, arXiv:2003.12861).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded CPU
// restatement of what the GPU path computes.  Only the tests, the package's
// smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
// no code, header, table or helper with the CUDA library and includes none of
// its files.
//
// What it computes (Sec. 1 and Sec. 4 of the paper): a computation graph of
// observables, parameters and PDFs; for each event the probability of the top
// PDF; the negative log-likelihood NLL = -sum_i log p_i over the events; and
// its gradient in the free parameters.  Batching in the paper (Sec. 4.1) only
// reorders this work, so the oracle evaluates the plain per-event definition,
// one event at a time, with forward-mode derivatives (value + gradient vector
// carried through every node).  Sums over events are sequential Neumaier sums.
//
// Every pdf is normalised by its analytic integral over the observable range
// (Sec. 4, "additional calls for the normalisation of PDFs").  Node formulas:
//   GAUSS    exp(-u^2/2), u=(x-mu)/sigma
//   EXP      exp(c x)
//   GAUSSEXP decay exp(-t/tau) (t>=0) convolved with a unit Gaussian(mu,sigma):
//            f(t) = 1/2 exp(s^2/2 - u s) erfc((s-u)/sqrt2), s=sigma/tau
//            (Fig. 1: signal = a convolution of PDFs)
//   CHEB     1 + sum_k c_k T_k(x'), x' mapped from [a,b] to [-1,1]
//   POLY     1 + sum_k a_k x^k      (Fig. 1: polynomial background)
//   SUM      sum_j f_j p_j, last fraction 1 - sum f_j, each p_j normalised
//   PROD     product of factors over disjoint observables
//   POISSON  lambda^k exp(-lambda) / k!, k = floor(x) (at most b-1), on an
//            observable range [a, b] with integer bounds 0 <= a < b: the
//            count k as a step density of unit-width steps; its integral is
//            the Poisson mass of k = a .. b-1 (Sec. 4.1 lists the batched
//            Poisson PDF)
//   EXPR     a density written as a short postfix program over the
//            observable, the node's parameters and constants (+ - * /,
//            neg, exp, log, pow), normalised by adaptive Gauss-Legendre
//            quadrature of the program and of its parameter derivatives
//            (Sec. 5: a fall-back evaluation for PDFs without specialised
//            batch code)
//   EXTEND   root only: the pdf below it, and the NLL gains the extended
//            term nu - N log nu for N events and expected count nu (the
//            Poisson probability of observing N, up to the constant log N!)
//
// Also here: a BFGS fitter (Sec. 1: "compute likelihoods and perform fits"),
// the Philox4x32-10 counter-based generator (Salmon et al., SC'11), Poisson
// sampling (inversion; PTRS of Hoermann 1993), accept-reject toy generation
// (Sec. 1: RooStats toy Monte Carlo) and a 64-bin histogram of a toy.
//
// Compiled with -ffp-contract=off so no multiply-add is fused behind the
// reader's back (this matters on aarch64 hosts).
//
// Parity status: every function here is pinned by the not-gpu tests (closed
// forms, quadrature, finite differences, brute force in mpmath, published
// Philox known-answer vectors, Poisson moments); see the test files.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

namespace {

constexpr int kMaxFree = 32;
constexpr double kInf = std::numeric_limits<double>::infinity();
constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kSqrtPi = 1.77245385090551602730;
constexpr double kSqrt2Pi = 2.50662827463100050242;

enum Kind { OBS = 0, PARAM = 1, GAUSS = 2, EXPO = 3, GAUSSEXP = 4, CHEB = 5, POLY = 6, SUM = 7, PROD = 8,
            POISSON = 9, EXTEND = 10, EXPR = 11 };

// EXPR programs: one int per operation, code | (argument << 8).
enum ExprCode { EX_X = 0, EX_PAR = 1, EX_CONST = 2, EX_ADD = 3, EX_SUB = 4, EX_MUL = 5, EX_DIV = 6, EX_NEG = 7,
                EX_EXP = 8, EX_LOG = 9, EX_POW = 10 };
constexpr int kExprMaxOps = 64, kExprMaxStack = 16, kExprMaxConsts = 16;

struct Node {
  int kind = 0;
  std::vector<int> in;
  double value = 0, lo = 0, hi = 0;
  bool is_free = false;
  int free_index = -1;  // PARAM: index into theta, or -1 if fixed
  int column = -1;      // OBS: column index (order of OBS nodes)
  std::vector<int> obs; // PDFs: sorted observable columns this node depends on
  std::vector<int> prog;       // EXPR: the program
  std::vector<double> consts;  // EXPR: its constants
};

struct Model {
  std::vector<Node> nodes;
  int root = -1;
  int n_free = 0;
  int n_obs = 0;
  std::vector<int> order;      // PDF nodes in dependency order (children first)
  std::vector<int> obs_node;   // column -> OBS node index
};

thread_local std::string g_err;

bool is_leaf_pdf(int k) {
  return k == GAUSS || k == EXPO || k == GAUSSEXP || k == CHEB || k == POLY || k == POISSON || k == EXPR;
}
bool is_pdf(int k) { return is_leaf_pdf(k) || k == SUM || k == PROD || k == EXTEND; }

// A dual number: value and derivatives in the n free parameters.
struct Dual {
  double v = 0;
  double d[kMaxFree] = {0};
};

// ---------------------------------------------------------------- numerics

// Sequential Neumaier (improved Kahan) summation.
struct Neumaier {
  double s = 0, c = 0;
  void add(double x) {
    double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// Phi(beta) - Phi(alpha) for the standard normal CDF, written with erfc on the
// side of the tail so that far-tail differences keep their precision.
double normal_mass(double alpha, double beta) {
  if (alpha >= 0) return 0.5 * (std::erfc(alpha / kSqrt2) - std::erfc(beta / kSqrt2));
  if (beta <= 0) return 0.5 * (std::erfc(-beta / kSqrt2) - std::erfc(-alpha / kSqrt2));
  return 0.5 * (std::erf(beta / kSqrt2) - std::erf(alpha / kSqrt2));
}

double phi_pdf(double x) { return std::exp(-0.5 * x * x) / kSqrt2Pi; }

// erfcx(z) = exp(z^2) erfc(z).  For z < 5 directly from libm; for z >= 5 from
// the classical continued fraction of erfc (Abramowitz & Stegun 7.1.14),
// evaluated bottom-up at a fixed, generous depth.
double erfcx(double z) {
  if (z < 5.0) return std::exp(z * z) * std::erfc(z);
  // erfc(z) = exp(-z^2)/sqrt(pi) * 1/(z + (1/2)/(z + 1/(z + (3/2)/(z + 2/(z + ...)))))
  double t = z;
  for (int k = 400; k >= 1; --k) t = z + (0.5 * k) / t;
  return 1.0 / (kSqrtPi * t);
}

// ------------------------------------------------------------- the model

double param_value(const Model& m, int node, const double* theta) {
  const Node& p = m.nodes[node];
  return p.free_index >= 0 ? theta[p.free_index] : p.value;
}
int param_index(const Model& m, int node) { return m.nodes[node].free_index; }

// Chebychev polynomials T_0..T_n at x by the three-term recurrence.
void cheb_T(double x, int n, double* T) {
  T[0] = 1.0;
  if (n >= 1) T[1] = x;
  for (int k = 2; k <= n; ++k) T[k] = 2.0 * x * T[k - 1] - T[k - 2];
}

// Mean of the density exp(y w) on w in [0,1]: 1/(1-exp(-y)) - 1/y, with the
// series 1/2 + y/12 - y^3/720 near y = 0 (from coth's Laurent series).
double trunc_exp_mean01(double y) {
  if (std::fabs(y) < 1e-3) return 0.5 + y / 12.0 - y * y * y / 720.0;
  return 1.0 / (-std::expm1(-y)) - 1.0 / y;
}

// GAUSSEXP shape and its partial derivatives in (tau, mu, sigma) at one point t.
// f = 1/2 exp(A) erfc(z), A = s^2/2 - u s, z = (s-u)/sqrt2, u=(t-mu)/sigma, s=sigma/tau.
// Uses A - z^2 = -u^2/2, so df/dtheta = f dA/dtheta - exp(-u^2/2)/sqrt(pi) dz/dtheta.
void gaussexp_shape(double t, double tau, double mu, double sigma, double* f, double df[3]) {
  const double u = (t - mu) / sigma;
  const double s = sigma / tau;
  const double A = 0.5 * s * s - u * s;
  const double z = (s - u) / kSqrt2;
  const double g = std::exp(-0.5 * u * u);
  double val;
  if (z < 5.0) val = 0.5 * std::exp(A) * std::erfc(z);
  else val = 0.5 * g * erfcx(z);
  const double dA[3] = {-sigma * sigma / (tau * tau * tau) + (t - mu) / (tau * tau), 1.0 / tau, sigma / (tau * tau)};
  const double dz[3] = {-sigma / (kSqrt2 * tau * tau), 1.0 / (kSqrt2 * sigma),
                        (1.0 / tau + (t - mu) / (sigma * sigma)) / kSqrt2};
  *f = val;
  for (int k = 0; k < 3; ++k) df[k] = val * dA[k] - g / kSqrtPi * dz[k];
}

// ------------------------------------------------------------ EXPR leaves

// The program's value at x with its derivatives in the node's np local
// parameters q (forward mode: every stack entry carries its np tangents).
// False when an operation leaves its domain (log or pow of a value <= 0,
// division by 0) or the result is not finite.
bool expr_eval(const Node& n, const double* q, int np, double x, double* f, double* df) {
  struct T {
    double v, d[8];
  };
  T st[kExprMaxStack];
  int sp = 0;
  if (n.prog.empty()) return false;  // no program attached (orc_model_set_expr)
  for (int op : n.prog) {
    const int code = op & 0xff, arg = op >> 8;
    if (code <= EX_CONST) {
      T& t = st[sp++];
      t.v = code == EX_X ? x : code == EX_PAR ? q[arg] : n.consts[arg];
      for (int k = 0; k < np; ++k) t.d[k] = (code == EX_PAR && k == arg) ? 1.0 : 0.0;
      continue;
    }
    if (code == EX_NEG || code == EX_EXP || code == EX_LOG) {
      T& a = st[sp - 1];
      if (code == EX_NEG) {
        a.v = -a.v;
        for (int k = 0; k < np; ++k) a.d[k] = -a.d[k];
      } else if (code == EX_EXP) {
        a.v = std::exp(a.v);
        for (int k = 0; k < np; ++k) a.d[k] *= a.v;
      } else {
        if (!(a.v > 0)) return false;
        for (int k = 0; k < np; ++k) a.d[k] /= a.v;
        a.v = std::log(a.v);
      }
      continue;
    }
    const T b = st[--sp];
    T& a = st[sp - 1];
    switch (code) {
      case EX_ADD:
        a.v += b.v;
        for (int k = 0; k < np; ++k) a.d[k] += b.d[k];
        break;
      case EX_SUB:
        a.v -= b.v;
        for (int k = 0; k < np; ++k) a.d[k] -= b.d[k];
        break;
      case EX_MUL:
        for (int k = 0; k < np; ++k) a.d[k] = a.d[k] * b.v + a.v * b.d[k];
        a.v *= b.v;
        break;
      case EX_DIV: {
        if (b.v == 0.0) return false;
        const double v = a.v / b.v;
        for (int k = 0; k < np; ++k) a.d[k] = (a.d[k] - v * b.d[k]) / b.v;
        a.v = v;
        break;
      }
      case EX_POW: {  // a^b = exp(b log a), a > 0
        if (!(a.v > 0)) return false;
        const double la = std::log(a.v), v = std::exp(b.v * la);
        for (int k = 0; k < np; ++k) a.d[k] = v * (b.d[k] * la + b.v * a.d[k] / a.v);
        a.v = v;
        break;
      }
    }
  }
  *f = st[0].v;
  for (int k = 0; k < np; ++k) df[k] = st[0].d[k];
  if (!std::isfinite(*f)) return false;
  for (int k = 0; k < np; ++k)
    if (!std::isfinite(df[k])) return false;
  return true;
}

// Gauss-Legendre rule of order n on [-1, 1]: the nodes are the roots of the
// Legendre polynomial P_n, found by Newton's method from the estimates
// cos(pi (i + 3/4) / (n + 1/2)), with P_n and P_n' from the three-term
// recurrence; the weights are 2 / ((1 - x^2) P_n'(x)^2).
struct GLRule {
  std::vector<double> x, w;
  explicit GLRule(int n) : x(n), w(n) {
    for (int i = 0; i < n; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-17) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};
const GLRule& gl20() {
  static const GLRule r(20);
  return r;
}

// The 20-point rule on [a, b] for the program and its np derivatives
// (out[0] = value, out[1 + k] = derivative k).
bool gl_panel(const Node& n, const double* q, int np, double a, double b, double* out) {
  const GLRule& r = gl20();
  const double h = 0.5 * (b - a), c = 0.5 * (a + b);
  for (int k = 0; k <= np; ++k) out[k] = 0.0;
  for (size_t i = 0; i < r.x.size(); ++i) {
    double f, df[8];
    if (!expr_eval(n, q, np, c + h * r.x[i], &f, df)) return false;
    out[0] += r.w[i] * f;
    for (int k = 0; k < np; ++k) out[1 + k] += r.w[i] * df[k];
  }
  for (int k = 0; k <= np; ++k) out[k] *= h;
  return true;
}

// Adaptive bisection: a panel is split until its two halves agree with it
// within tol (absolute, halved per split, so the panels' errors add up to
// at most the first panel's tol) or its depth reaches 30; the halves' sums
// are returned.  tol is kept well above the panels' rounding (1e-14 of the
// integral), so the recursion ends.
bool gl_adapt(const Node& n, const double* q, int np, double a, double b, const double* whole, double tol,
              int depth, double* out) {
  double L[9], R[9];
  const double m = 0.5 * (a + b);
  if (!gl_panel(n, q, np, a, m, L) || !gl_panel(n, q, np, m, b, R)) return false;
  if (std::fabs(L[0] + R[0] - whole[0]) <= tol || depth >= 30) {
    for (int k = 0; k <= np; ++k) out[k] += L[k] + R[k];
    return true;
  }
  return gl_adapt(n, q, np, a, m, L, 0.5 * tol, depth + 1, out) &&
         gl_adapt(n, q, np, m, b, R, 0.5 * tol, depth + 1, out);
}

// Integral of an EXPR leaf over [a, b] to ~1e-14 of itself, with its
// derivatives; false outside the program's domain or for I <= 0.
bool expr_norm(const Node& n, const double* q, int np, double a, double b, double* I, double* dI) {
  // a first estimate from 16 panels sets the absolute tolerance
  double est = 0.0, P[9];
  for (int j = 0; j < 16; ++j) {
    if (!gl_panel(n, q, np, a + (b - a) * j / 16.0, a + (b - a) * (j + 1) / 16.0, P)) return false;
    est += std::fabs(P[0]);
  }
  double out[9] = {0};
  const double tol = 1e-14 * est / 16.0;
  for (int j = 0; j < 16; ++j) {
    const double pa = a + (b - a) * j / 16.0, pb = a + (b - a) * (j + 1) / 16.0;
    if (!gl_panel(n, q, np, pa, pb, P) || !gl_adapt(n, q, np, pa, pb, P, tol, 0, out)) return false;
  }
  *I = out[0];
  for (int k = 0; k < np; ++k) dI[k] = out[1 + k];
  return *I > 0.0 && std::isfinite(*I);
}

// Normalisation integral of a leaf pdf over its observable range, with its
// derivatives in the leaf's parameters (local order = the leaf's inputs 1..n).
// Returns false on a parameter outside the pdf's domain.
bool leaf_norm(const Model& m, const Node& n, const double* theta, double* I, double* dI) {
  const Node& ob = m.nodes[n.in[0]];
  const double a = ob.lo, b = ob.hi;
  const int np = (int)n.in.size() - 1;
  std::vector<double> q(np);
  for (int k = 0; k < np; ++k) q[k] = param_value(m, n.in[k + 1], theta);
  for (int k = 0; k < np; ++k) dI[k] = 0;
  switch (n.kind) {
    case GAUSS: {
      const double mu = q[0], sigma = q[1];
      if (!(sigma > 0)) return false;
      const double al = (a - mu) / sigma, be = (b - mu) / sigma;
      // I = sigma sqrt(2 pi) [Phi(be) - Phi(al)]
      *I = sigma * kSqrt2Pi * normal_mass(al, be);
      dI[0] = std::exp(-0.5 * al * al) - std::exp(-0.5 * be * be);
      dI[1] = *I / sigma - (be * std::exp(-0.5 * be * be) - al * std::exp(-0.5 * al * al));
      return true;
    }
    case EXPO: {
      const double c = q[0];
      const double L = b - a;
      // I = int_a^b exp(c x) dx; dI/dc = I * E[x]
      if (c == 0.0) *I = L;
      else *I = std::exp(c * a) * std::expm1(c * L) / c;
      dI[0] = *I * (a + L * trunc_exp_mean01(c * L));
      return true;
    }
    case GAUSSEXP: {
      const double tau = q[0], mu = q[1], sigma = q[2];
      if (!(tau > 0) || !(sigma > 0)) return false;
      // I = tau [Phi(be) - Phi(al) - f(b) + f(a)], from f' = G(t-mu) - f/tau.
      const double al = (a - mu) / sigma, be = (b - mu) / sigma;
      double fa, fb, dfa[3], dfb[3];
      gaussexp_shape(a, tau, mu, sigma, &fa, dfa);
      gaussexp_shape(b, tau, mu, sigma, &fb, dfb);
      const double D = normal_mass(al, be);
      const double br = D - fb + fa;
      *I = tau * br;
      const double dD[3] = {0.0, -(phi_pdf(be) - phi_pdf(al)) / sigma, -(be * phi_pdf(be) - al * phi_pdf(al)) / sigma};
      for (int k = 0; k < 3; ++k) dI[k] = (k == 0 ? br : 0.0) + tau * (dD[k] - dfb[k] + dfa[k]);
      return true;
    }
    case CHEB: {
      // x' = (2x - a - b)/(b - a); int_{-1}^{1} T_k = 2/(1-k^2) for even k, 0 for odd k.
      double s = 2.0;
      for (int k = 1; k <= np; ++k) {
        const double Tk = (k % 2 == 0) ? 2.0 / (1.0 - (double)k * k) : 0.0;
        s += q[k - 1] * Tk;
        dI[k - 1] = 0.5 * (b - a) * Tk;
      }
      *I = 0.5 * (b - a) * s;
      return true;
    }
    case POLY: {
      double s = b - a;
      for (int k = 1; k <= np; ++k) {
        const double Pk = (std::pow(b, k + 1) - std::pow(a, k + 1)) / (k + 1);
        s += q[k - 1] * Pk;
        dI[k - 1] = Pk;
      }
      *I = s;
      return true;
    }
    case EXPR:
      return expr_norm(n, q.data(), np, a, b, I, dI);
    case POISSON: {
      // I = sum_{k=a}^{b-1} P(k), dI/dlambda = sum P(k) (k/lambda - 1), summed term by term.
      const double lam = q[0];
      if (!(lam > 0)) return false;
      Neumaier s, ds;
      for (double k = a; k < b; k += 1.0) {
        const double pk = std::exp(k * std::log(lam) - lam - std::lgamma(k + 1.0));
        s.add(pk);
        ds.add(pk * (k / lam - 1.0));
      }
      *I = s.value();
      dI[0] = ds.value();
      return true;
    }
  }
  return false;
}

// Unnormalised shape of a leaf at x with derivatives in its local parameters.
void leaf_shape(const Model& m, const Node& n, const double* theta, double x, double* f, double* df) {
  const Node& ob = m.nodes[n.in[0]];
  const double a = ob.lo, b = ob.hi;
  const int np = (int)n.in.size() - 1;
  double q[8];
  for (int k = 0; k < np; ++k) q[k] = param_value(m, n.in[k + 1], theta);
  switch (n.kind) {
    case GAUSS: {
      const double u = (x - q[0]) / q[1];
      *f = std::exp(-0.5 * u * u);
      df[0] = *f * u / q[1];
      df[1] = *f * u * u / q[1];
      return;
    }
    case EXPO: {
      *f = std::exp(q[0] * x);
      df[0] = x * *f;
      return;
    }
    case GAUSSEXP: {
      gaussexp_shape(x, q[0], q[1], q[2], f, df);
      return;
    }
    case CHEB: {
      double T[9];
      const double xp = (2.0 * x - a - b) / (b - a);
      cheb_T(xp, np, T);
      double s = 1.0;
      for (int k = 1; k <= np; ++k) { s += q[k - 1] * T[k]; df[k - 1] = T[k]; }
      *f = s;
      return;
    }
    case POLY: {
      double s = 1.0, xk = 1.0;
      for (int k = 1; k <= np; ++k) { xk *= x; s += q[k - 1] * xk; df[k - 1] = xk; }
      *f = s;
      return;
    }
    case EXPR: {
      if (!expr_eval(n, q, np, x, f, df)) {
        *f = std::numeric_limits<double>::quiet_NaN();
        for (int k = 0; k < np; ++k) df[k] = 0.0;
      }
      return;
    }
    case POISSON: {
      const double k = std::min(std::floor(x), b - 1.0);
      *f = std::exp(k * std::log(q[0]) - q[0] - std::lgamma(k + 1.0));
      df[0] = *f * (k / q[0] - 1.0);
      return;
    }
  }
}

// Per parameter point: every leaf's integral and its derivatives.
struct Norms {
  std::vector<double> I;               // per node (leaves only)
  std::vector<std::vector<double>> dI; // per node, local parameter order
};

bool compute_norms(const Model& m, const double* theta, Norms* out) {
  out->I.assign(m.nodes.size(), 0.0);
  out->dI.assign(m.nodes.size(), {});
  for (int idx : m.order) {
    const Node& n = m.nodes[idx];
    if (!is_leaf_pdf(n.kind)) continue;
    out->dI[idx].assign(n.in.size() - 1, 0.0);
    if (!leaf_norm(m, n, theta, &out->I[idx], out->dI[idx].data())) return false;
  }
  return true;
}

// One event: normalised probability of every PDF node, in dependency order,
// with forward-mode derivatives.  Returns the root's dual number.
Dual eval_event(const Model& m, const Norms& nm, const double* theta, const double* x, std::vector<Dual>& val) {
  const int P = m.n_free;
  for (int idx : m.order) {
    const Node& n = m.nodes[idx];
    Dual& r = val[idx];
    for (int k = 0; k < P; ++k) r.d[k] = 0.0;
    if (is_leaf_pdf(n.kind)) {
      const double xv = x[m.nodes[n.in[0]].column];
      double f, df[8];
      leaf_shape(m, n, theta, xv, &f, df);
      const double I = nm.I[idx];
      r.v = f / I;
      // d(f/I) = (df I - f dI)/I^2
      for (size_t k = 1; k < n.in.size(); ++k) {
        const int fi = param_index(m, n.in[k]);
        if (fi < 0) continue;
        r.d[fi] += (df[k - 1] * I - f * nm.dI[idx][k - 1]) / (I * I);
      }
    } else if (n.kind == SUM) {
      const int nc = ((int)n.in.size() + 1) / 2;  // components; fractions = nc-1
      double frac_sum = 0.0;
      r.v = 0.0;
      for (int j = 0; j < nc - 1; ++j) {
        const double fj = param_value(m, n.in[nc + j], theta);
        frac_sum += fj;
        const Dual& c = val[n.in[j]];
        r.v += fj * c.v;
        for (int k = 0; k < P; ++k) r.d[k] += fj * c.d[k];
      }
      const Dual& last = val[n.in[nc - 1]];
      const double fl = 1.0 - frac_sum;
      r.v += fl * last.v;
      for (int k = 0; k < P; ++k) r.d[k] += fl * last.d[k];
      for (int j = 0; j < nc - 1; ++j) {
        const int fi = param_index(m, n.in[nc + j]);
        if (fi >= 0) r.d[fi] += val[n.in[j]].v - last.v;
      }
    } else if (n.kind == EXTEND) {
      r = val[n.in[0]];  // per event the pdf below; the extended term is per dataset
    } else if (n.kind == PROD) {
      // Product rule over the factors.
      r.v = 1.0;
      for (int c : n.in) r.v *= val[c].v;
      for (size_t j = 0; j < n.in.size(); ++j) {
        double others = 1.0;
        for (size_t i = 0; i < n.in.size(); ++i)
          if (i != j) others *= val[n.in[i]].v;
        for (int k = 0; k < P; ++k) r.d[k] += others * val[n.in[j]].d[k];
      }
    }
  }
  return val[m.root];
}

bool collect_obs(Model& m, int idx, std::string* why) {
  Node& n = m.nodes[idx];
  if (!n.obs.empty() || n.kind == OBS || n.kind == PARAM) return true;
  if (is_leaf_pdf(n.kind)) {
    n.obs = {m.nodes[n.in[0]].column};
    return true;
  }
  if (n.kind == SUM) {
    const int nc = ((int)n.in.size() + 1) / 2;
    for (int j = 0; j < nc; ++j) {
      const std::vector<int>& o = m.nodes[n.in[j]].obs;
      if (j == 0) n.obs = o;
      else if (o != n.obs) { *why = "SUM components depend on different observables"; return false; }
    }
    return true;
  }
  if (n.kind == EXTEND) {
    n.obs = m.nodes[n.in[0]].obs;
    return true;
  }
  if (n.kind == PROD) {
    for (int c : n.in) {
      for (int o : m.nodes[c].obs) {
        if (std::find(n.obs.begin(), n.obs.end(), o) != n.obs.end()) {
          *why = "PROD factors share an observable";
          return false;
        }
        n.obs.push_back(o);
      }
    }
    std::sort(n.obs.begin(), n.obs.end());
    return true;
  }
  return true;
}

// Depth-first topological order of the PDF nodes under the root.
bool topo(Model& m, int idx, std::vector<int>& state, std::string* why) {
  if (state[idx] == 2) return true;
  if (state[idx] == 1) { *why = "cycle in the graph"; return false; }
  state[idx] = 1;
  const Node& n = m.nodes[idx];
  if (n.kind == EXTEND) {
    if (!topo(m, n.in[0], state, why)) return false;
  } else if (n.kind == SUM || n.kind == PROD) {
    const int nc = n.kind == SUM ? ((int)n.in.size() + 1) / 2 : (int)n.in.size();
    for (int j = 0; j < nc; ++j)
      if (!topo(m, n.in[j], state, why)) return false;
  }
  state[idx] = 2;
  if (is_pdf(n.kind)) m.order.push_back(idx);
  return true;
}

// --------------------------------------------------------------- Philox

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications, the key
// bumped by the Weyl constants between rounds.
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c[0] = hi1 ^ c[1] ^ k0;
    c[1] = lo1;
    c[2] = hi0 ^ c[3] ^ k1;
    c[3] = lo0;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Uniform double from two 32-bit words: the top 53 bits as an integer times 2^-53.
double u53(uint32_t hi, uint32_t lo) { return (double)(((uint64_t)hi << 21) | (lo >> 11)) * 0x1.0p-53; }
// The same, shifted by half a step so it never is 0 or 1.
double u53_open(uint32_t hi, uint32_t lo) {
  return ((double)(((uint64_t)hi << 21) | (lo >> 11)) + 0.5) * 0x1.0p-53;
}

// Stream layout shared by definition with any other implementation of this
// generator: key = (seed low word, seed high word); counter = (i, attempt, set, tag).
void draw(uint64_t seed, uint32_t i, uint32_t attempt, uint32_t set, uint32_t tag, uint32_t out[4]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t ctr[4] = {i, attempt, set, tag};
  philox4x32_10(ctr, key, out);
}

constexpr uint32_t kPoissonTag = 0xFFFFFFFFu;

// Poisson(mu): inversion by sequential search for mu < 10; otherwise PTRS, the
// transformed rejection with squeeze of W. Hoermann, "The transformed rejection
// method for generating Poisson random variables", Insurance: Mathematics and
// Economics 12 (1993).  Iteration j uses counter (j, 0, set, kPoissonTag).
int64_t poisson(uint64_t seed, uint32_t set, double mu) {
  if (!(mu > 0)) return 0;
  uint32_t r[4];
  if (mu < 10.0) {
    draw(seed, 0, 0, set, kPoissonTag, r);
    const double u = u53(r[0], r[1]);
    double p = std::exp(-mu), F = p;
    int64_t k = 0;
    while (u > F && k < 1000) { ++k; p *= mu / (double)k; F += p; }
    return k;
  }
  const double smu = std::sqrt(mu);
  const double b = 0.931 + 2.53 * smu;
  const double a = -0.059 + 0.02483 * b;
  const double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
  const double vr = 0.9277 - 3.6224 / (b - 2.0);
  const double log_mu = std::log(mu);
  for (uint32_t j = 0; j < 100000u; ++j) {
    draw(seed, j, 0, set, kPoissonTag, r);
    const double U = u53_open(r[0], r[1]) - 0.5;
    const double V = u53_open(r[2], r[3]);
    const double us = 0.5 - std::fabs(U);
    const double kd = std::floor((2.0 * a / us + b) * U + mu + 0.43);
    if (us >= 0.07 && V <= vr) return (int64_t)kd;
    if (kd < 0.0 || (us < 0.013 && V > us)) continue;
    const double lhs = std::log(V) + std::log(inv_alpha) - std::log(a / (us * us) + b);
    const double rhs = -mu + kd * log_mu - std::lgamma(kd + 1.0);
    if (lhs <= rhs) return (int64_t)kd;
  }
  return -1;
}

// Factors that are generated independently: the root, or the leaves of a
// (nested) PROD at the root.
void gen_factors(const Model& m, int idx, std::vector<int>* out) {
  const Node& n = m.nodes[idx];
  if (n.kind == EXTEND) {
    gen_factors(m, n.in[0], out);
  } else if (n.kind == PROD) {
    for (int c : n.in) gen_factors(m, c, out);
  } else {
    out->push_back(idx);
  }
}

// Probability of one factor (a sub-graph) at a value of its single observable.
double factor_density(const Model& m, const Norms& nm, const double* theta, int factor, double xv,
                      std::vector<Dual>& val) {
  std::vector<double> x(m.n_obs, 0.0);
  x[m.nodes[factor].obs[0]] = xv;
  // Evaluate the whole graph and read the factor's node value.
  eval_event(m, nm, theta, x.data(), val);
  return val[factor].v;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

struct orc_model;  // opaque

const char* orc_last_error() { return g_err.c_str(); }

// Build a model from flat arrays.  kinds[i] uses this file's Kind numbering;
// ins is n x 8 (unused slots ignored).  Returns NULL on an invalid graph.
orc_model* orc_model_new(int n, const int* kinds, const int* n_in, const int* ins, const double* values,
                         const double* los, const double* his, const int* is_free, int root) {
  Model* m = new Model();
  m->nodes.resize(n);
  std::string why;
  int col = 0, fi = 0;
  for (int i = 0; i < n; ++i) {
    Node& nd = m->nodes[i];
    nd.kind = kinds[i];
    nd.in.assign(ins + 8 * i, ins + 8 * i + n_in[i]);
    nd.value = values[i];
    nd.lo = los[i];
    nd.hi = his[i];
    nd.is_free = is_free[i] != 0;
    if (nd.kind == OBS) { nd.column = col++; m->obs_node.push_back(i); }
    if (nd.kind == PARAM && nd.is_free) nd.free_index = fi++;
  }
  m->n_free = fi;
  m->n_obs = col;
  m->root = root;
  bool ok = root >= 0 && root < n && is_pdf(m->nodes[root].kind) && fi <= kMaxFree;
  if (!ok) why = "root is not a pdf node, or too many free parameters";
  for (int i = 0; ok && i < n; ++i) {
    const Node& nd = m->nodes[i];
    for (int c : nd.in)
      if (c < 0 || c >= n) { ok = false; why = "input index out of range"; }
    if (!ok) break;
    if (is_leaf_pdf(nd.kind)) {
      int want = nd.kind == GAUSS ? 3 : nd.kind == EXPO ? 2 : nd.kind == GAUSSEXP ? 4 : nd.kind == POISSON ? 2 : -1;
      if ((want > 0 && (int)nd.in.size() != want) || nd.in.size() < 1 || nd.in.size() > 8) { ok = false; why = "leaf arity"; }
      else if (m->nodes[nd.in[0]].kind != OBS) { ok = false; why = "leaf input 0 must be an observable"; }
      else
        for (size_t k = 1; k < nd.in.size(); ++k)
          if (m->nodes[nd.in[k]].kind != PARAM) { ok = false; why = "leaf parameter input is not a PARAM"; }
    } else if (nd.kind == SUM) {
      if (nd.in.size() < 3 || nd.in.size() % 2 == 0) { ok = false; why = "SUM arity"; }
      const int nc = ((int)nd.in.size() + 1) / 2;
      for (int j = 0; ok && j < (int)nd.in.size(); ++j) {
        const int k = m->nodes[nd.in[j]].kind;
        if (j < nc ? !is_pdf(k) : k != PARAM) { ok = false; why = "SUM inputs"; }
      }
    } else if (nd.kind == PROD) {
      if (nd.in.empty()) { ok = false; why = "PROD arity"; }
      for (int c : nd.in)
        if (!is_pdf(m->nodes[c].kind) || m->nodes[c].kind == EXTEND) { ok = false; why = "PROD inputs"; }
    } else if (nd.kind == EXTEND) {
      if (nd.in.size() != 2 || !is_pdf(m->nodes[nd.in[0]].kind) || m->nodes[nd.in[0]].kind == EXTEND ||
          m->nodes[nd.in[1]].kind != PARAM) { ok = false; why = "EXTEND inputs: [pdf, expected count]"; }
      else if (i != root) { ok = false; why = "EXTEND must be the root"; }
    }
    if (ok && nd.kind == POISSON) {
      const Node& ob = m->nodes[nd.in[0]];
      if (!(ob.lo >= 0) || ob.lo != std::floor(ob.lo) || ob.hi != std::floor(ob.hi) || !(ob.hi > ob.lo) ||
          ob.hi - ob.lo > 100000) { ok = false; why = "POISSON range must have integer bounds 0 <= a < b <= a + 1e5"; }
    }
    if (ok && nd.kind == SUM) {
      const int nc = ((int)nd.in.size() + 1) / 2;
      for (int j = 0; j < nc; ++j)
        if (m->nodes[nd.in[j]].kind == EXTEND) { ok = false; why = "EXTEND must be the root"; }
    }
  }
  if (ok) {
    std::vector<int> state(n, 0);
    ok = topo(*m, root, state, &why);
  }
  for (size_t j = 0; ok && j < m->order.size(); ++j) ok = collect_obs(*m, m->order[j], &why);
  if (!ok) {
    g_err = why;
    delete m;
    return nullptr;
  }
  return reinterpret_cast<orc_model*>(m);
}

void orc_model_free(orc_model* h) { delete reinterpret_cast<Model*>(h); }

// Attach the program of EXPR node `node` (ops: n_ops codes, code | arg << 8;
// consts: n_consts values).  The program is checked as a whole: every
// argument in range, the stack never underflows nor exceeds its depth, and
// exactly one value is left.  Returns 0, or -1 with the reason in
// orc_last_error.
int orc_model_set_expr(orc_model* h, int node, int n_ops, const int* ops, int n_consts, const double* consts) {
  Model& m = *reinterpret_cast<Model*>(h);
  auto fail = [](const char* why) {
    g_err = why;
    return -1;
  };
  if (node < 0 || node >= (int)m.nodes.size() || m.nodes[node].kind != EXPR) return fail("not an EXPR node");
  if (n_ops < 1 || n_ops > kExprMaxOps) return fail("program length must be 1..64");
  if (n_consts < 0 || n_consts > kExprMaxConsts) return fail("at most 16 constants");
  Node& nd = m.nodes[node];
  const int np = (int)nd.in.size() - 1;
  int depth = 0;
  for (int i = 0; i < n_ops; ++i) {
    const int code = ops[i] & 0xff, arg = ops[i] >> 8;
    if (code < EX_X || code > EX_POW) return fail("unknown operation");
    if (code == EX_PAR && (arg < 0 || arg >= np)) return fail("parameter index out of range");
    if (code == EX_CONST && (arg < 0 || arg >= n_consts)) return fail("constant index out of range");
    if (code > EX_CONST && arg != 0) return fail("operation with an argument");
    if (code <= EX_CONST) ++depth;
    else if (code == EX_NEG || code == EX_EXP || code == EX_LOG) { if (depth < 1) return fail("stack underflow"); }
    else { if (depth < 2) return fail("stack underflow"); --depth; }
    if (depth > kExprMaxStack) return fail("stack deeper than 16");
  }
  if (depth != 1) return fail("the program must leave exactly one value");
  nd.prog.assign(ops, ops + n_ops);
  nd.consts.assign(consts, consts + n_consts);
  return 0;
}
int orc_n_free(const orc_model* h) { return reinterpret_cast<const Model*>(h)->n_free; }
int orc_n_obs(const orc_model* h) { return reinterpret_cast<const Model*>(h)->n_obs; }

// Normalisation integral of leaf `node` and its derivatives in the free
// parameters (dI, length n_free).  Returns 0 on success.
int orc_leaf_norm(const orc_model* h, int node, const double* theta, double* I, double* dI_free) {
  const Model& m = *reinterpret_cast<const Model*>(h);
  const Node& n = m.nodes[node];
  if (!is_leaf_pdf(n.kind)) return -1;
  double dI[8];
  if (!leaf_norm(m, n, theta, I, dI)) return -2;
  for (int k = 0; k < m.n_free; ++k) dI_free[k] = 0;
  for (size_t k = 1; k < n.in.size(); ++k) {
    const int fi = param_index(m, n.in[k]);
    if (fi >= 0) dI_free[fi] += dI[k - 1];
  }
  return 0;
}

// Unnormalised shape of leaf `node` at x.
double orc_leaf_shape(const orc_model* h, int node, const double* theta, double x) {
  const Model& m = *reinterpret_cast<const Model*>(h);
  double f, df[8];
  leaf_shape(m, m.nodes[node], theta, x, &f, df);
  return f;
}

// Normalised probability of `node` (any PDF node) for each of N events, and
// optionally its gradient (N x n_free, row-major).  cols: n_obs pointers.
int orc_pdf(const orc_model* h, int node, const double* theta, const double* const* cols, int64_t N, double* p,
            double* grad) {
  const Model& m = *reinterpret_cast<const Model*>(h);
  Norms nm;
  if (!compute_norms(m, theta, &nm)) return -2;
  std::vector<Dual> val(m.nodes.size());
  std::vector<double> x(m.n_obs);
  for (int64_t i = 0; i < N; ++i) {
    for (int c = 0; c < m.n_obs; ++c) x[c] = cols[c][i];
    eval_event(m, nm, theta, x.data(), val);
    p[i] = val[node].v;
    if (grad)
      for (int k = 0; k < m.n_free; ++k) grad[i * m.n_free + k] = val[node].d[k];
  }
  return 0;
}

// NLL = -sum_i log p_i and its gradient -sum_i dlog p_i/dtheta over N events,
// Neumaier-summed in event order.  abs_logp = sum_i |log p_i| and
// abs_grad[k] = sum_i |dlog p_i/dtheta_k| are the scales against which
// tolerances are stated.  Returns 0, -2 (parameter outside the domain) or
// -3 (some p_i <= 0 or not finite; nll = +inf).
int orc_nll(const orc_model* h, const double* theta, const double* const* cols, int64_t N, double* nll,
            double* grad, double* abs_logp, double* abs_grad) {
  const Model& m = *reinterpret_cast<const Model*>(h);
  const int P = m.n_free;
  Norms nm;
  if (!compute_norms(m, theta, &nm)) {
    *nll = kInf;
    return -2;
  }
  std::vector<Dual> val(m.nodes.size());
  std::vector<double> x(m.n_obs);
  Neumaier s0, sa;
  std::vector<Neumaier> sg(P), sga(P);
  bool bad = false;
  for (int64_t i = 0; i < N; ++i) {
    for (int c = 0; c < m.n_obs; ++c) x[c] = cols[c][i];
    const Dual r = eval_event(m, nm, theta, x.data(), val);
    if (!(r.v > 0) || !std::isfinite(r.v)) { bad = true; continue; }
    const double lp = std::log(r.v);
    s0.add(lp);
    sa.add(std::fabs(lp));
    for (int k = 0; k < P; ++k) {
      const double g = r.d[k] / r.v;
      sg[k].add(g);
      sga[k].add(std::fabs(g));
    }
  }
  // Extended likelihood: + nu - N log nu (the Poisson probability of N
  // events given nu, without the constant log N!), d/dnu = 1 - N/nu.
  double ext = 0.0, ext_abs = 0.0;
  const Node& top = m.nodes[m.root];
  if (top.kind == EXTEND) {
    const double nu = param_value(m, top.in[1], theta);
    if (!(nu > 0)) {
      *nll = kInf;
      return -2;
    }
    ext = nu - (double)N * std::log(nu);
    ext_abs = nu + std::fabs((double)N * std::log(nu));
    const int fi = param_index(m, top.in[1]);
    if (fi >= 0) {
      sg[fi].add(-(1.0 - (double)N / nu));
      sga[fi].add(1.0 + (double)N / nu);
    }
  }
  *nll = bad ? kInf : ext - s0.value();
  if (abs_logp) *abs_logp = sa.value() + ext_abs;
  for (int k = 0; k < P; ++k) {
    if (grad) grad[k] = -sg[k].value();
    if (abs_grad) abs_grad[k] = sga[k].value();
  }
  return bad ? -3 : 0;
}

// Raw Philox4x32-10 block, for known-answer tests.
void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

// Poisson(mu) draw for set `set` under `seed`.
int64_t orc_poisson(uint64_t seed, uint32_t set, double mu) { return poisson(seed, set, mu); }

// Accept-reject bound of every generation factor: 1.2 x the maximum of the
// factor's density over the 4096 midpoints of its observable range.
// Writes n_factors bounds; returns the number of factors, or -1.
int orc_gen_bounds(const orc_model* h, const double* theta, double* bounds, int max_factors) {
  const Model& m = *reinterpret_cast<const Model*>(h);
  std::vector<int> fac;
  gen_factors(m, m.root, &fac);
  if ((int)fac.size() > max_factors) return -1;
  Norms nm;
  if (!compute_norms(m, theta, &nm)) return -1;
  std::vector<Dual> val(m.nodes.size());
  for (size_t j = 0; j < fac.size(); ++j) {
    if (m.nodes[fac[j]].obs.size() != 1) return -1;
    const Node& ob = m.nodes[m.obs_node[m.nodes[fac[j]].obs[0]]];
    double mx = 0;
    for (int g = 0; g < 4096; ++g) {
      const double xv = ob.lo + (ob.hi - ob.lo) * ((g + 0.5) / 4096.0);
      mx = std::max(mx, factor_density(m, nm, theta, fac[j], xv, val));
    }
    bounds[j] = 1.2 * mx;
  }
  return (int)fac.size();
}

// Events [i0, i1) of set `set`, generated by accept-reject: for factor j and
// event i, attempt a draws one Philox block at counter (i, a, set, j):
// x = lo + (hi-lo) u53(r0,r1), y = bound_j u53(r2,r3), accepted if y < density(x).
// cols[c] receives column c (length i1-i0).  Returns 0, or -1 when an event
// needs more than 100000 attempts.
int orc_generate(const orc_model* h, const double* theta, const double* bounds, uint64_t seed, uint32_t set,
                 int64_t i0, int64_t i1, double* const* cols) {
  const Model& m = *reinterpret_cast<const Model*>(h);
  std::vector<int> fac;
  gen_factors(m, m.root, &fac);
  Norms nm;
  if (!compute_norms(m, theta, &nm)) return -1;
  std::vector<Dual> val(m.nodes.size());
  for (size_t j = 0; j < fac.size(); ++j) {
    const int col = m.nodes[fac[j]].obs[0];
    const Node& ob = m.nodes[m.obs_node[col]];
    const double width = ob.hi - ob.lo;
    for (int64_t i = i0; i < i1; ++i) {
      bool done = false;
      for (uint32_t a = 0; a < 100000u && !done; ++a) {
        uint32_t r[4];
        draw(seed, (uint32_t)i, a, set, (uint32_t)j, r);
        const double xv = ob.lo + width * u53(r[0], r[1]);
        const double y = bounds[j] * u53(r[2], r[3]);
        if (y < factor_density(m, nm, theta, fac[j], xv, val)) {
          cols[col][i - i0] = xv;
          done = true;
        }
      }
      if (!done) return -1;
    }
  }
  return 0;
}

// 64-bin histogram of column values on [lo, hi], normalised by the number of
// events: bin = floor((x - lo) * (64 / (hi - lo))), clamped to [0, 63].
void orc_hist64(const double* x, int64_t N, double lo, double hi, float* out) {
  int64_t cnt[64] = {0};
  const double scale = 64.0 / (hi - lo);
  for (int64_t i = 0; i < N; ++i) {
    double t = (x[i] - lo) * scale;
    int b = (int)std::floor(t);
    b = std::min(63, std::max(0, b));
    cnt[b]++;
  }
  for (int b = 0; b < 64; ++b) out[b] = N > 0 ? (float)((double)cnt[b] / (double)N) : 0.0f;
}

}  // extern "C"

// ------------------------------------------------------------------ fitter
//
// Minimise the NLL over the free parameters (Sec. 1: "perform fits to data").
// The paper does not name its minimiser; this is BFGS (Nocedal & Wright,
// Numerical Optimization, 2nd ed., Alg. 6.1) with the strong-Wolfe line search
// of their Alg. 3.5/3.6, run in internal coordinates: a bounded parameter is
// theta = lo + (hi-lo)(sin(phi)+1)/2 (the transform MINUIT documents), an
// unbounded one is used as is.  Stop when EDM = g^T H g / 2 < tol.  The
// covariance is the inverse of the NLL's Hessian in theta, taken by central
// differences of the analytic gradient (an NLL has "up" = 1/2, so cov = H^-1).

namespace {

struct Problem {
  const Model* m;
  const double* const* cols;
  int64_t N;
  int P;
  std::vector<double> lo, hi;
  std::vector<bool> bounded;
  int evals = 0;

  void to_theta(const double* x, double* th) const {
    for (int k = 0; k < P; ++k)
      th[k] = bounded[k] ? lo[k] + (hi[k] - lo[k]) * (std::sin(x[k]) + 1.0) * 0.5 : x[k];
  }
  void to_internal(const double* th, double* x) const {
    for (int k = 0; k < P; ++k) {
      if (!bounded[k]) { x[k] = th[k]; continue; }
      double r = 2.0 * (th[k] - lo[k]) / (hi[k] - lo[k]) - 1.0;
      r = std::min(1.0, std::max(-1.0, r));
      x[k] = std::asin(r);
    }
  }
  // f and gradient in internal coordinates; f = +inf outside the domain.
  double f(const double* x, double* g) {
    ++evals;
    std::vector<double> th(P), gt(P);
    to_theta(x, th.data());
    double nll;
    const int rc = orc_nll_impl(th.data(), &nll, gt.data());
    if (rc != 0 || !std::isfinite(nll)) {
      for (int k = 0; k < P; ++k) g[k] = 0;
      return kInf;
    }
    for (int k = 0; k < P; ++k)
      g[k] = bounded[k] ? gt[k] * (hi[k] - lo[k]) * 0.5 * std::cos(x[k]) : gt[k];
    return nll;
  }
  int orc_nll_impl(const double* th, double* nll, double* g);
};

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// Strong-Wolfe line search along p from x (Nocedal & Wright Alg. 3.5 with the
// zoom of Alg. 3.6, bisection as the interpolation), first trial step a1.
// Returns the accepted step, or 0 when none is found.
// A trial point is also accepted under the approximate Wolfe conditions of
// Hager & Zhang (SIAM J. Optim. 16, 2005): phi'(a) within [c2, 2 c1 - 1]
// times phi'(0) and phi(a) <= phi(0) + 1e-12 |phi(0)|, which still hold when
// the decrease near a minimum is below the NLL's rounding.
double line_search(Problem& pr, const std::vector<double>& x, double f0, const std::vector<double>& g0,
                   const std::vector<double>& p, double* f_out, std::vector<double>* g_out, int max_evals,
                   double a1) {
  const double c1 = 1e-4, c2 = 0.9, eps_f = 1e-12;
  const int P = pr.P;
  const double d0 = dot(g0, p);
  std::vector<double> xt(P), gt(P);
  auto phi = [&](double a, double* d) {
    for (int k = 0; k < P; ++k) xt[k] = x[k] + a * p[k];
    const double v = pr.f(xt.data(), gt.data());
    *d = dot(gt, p);
    return v;
  };
  auto approx_wolfe = [&](double fa, double d) {
    return std::isfinite(fa) && fa <= f0 + eps_f * std::fabs(f0) && d >= c2 * d0 && d <= (2.0 * c1 - 1.0) * d0;
  };
  auto zoom = [&](double alo, double flo, double ahi) -> double {
    for (int it = 0; it < max_evals; ++it) {
      const double a = 0.5 * (alo + ahi);
      double d;
      const double fa = phi(a, &d);
      if (approx_wolfe(fa, d)) { *f_out = fa; *g_out = gt; return a; }
      if (fa > f0 + c1 * a * d0 || fa >= flo) {
        ahi = a;
      } else {
        if (std::fabs(d) <= -c2 * d0) { *f_out = fa; *g_out = gt; return a; }
        if (d * (ahi - alo) >= 0) ahi = alo;
        alo = a;
        flo = fa;
      }
    }
    if (alo > 0) {  // settle for the best sufficient-decrease point seen
      double d;
      *f_out = phi(alo, &d);
      *g_out = gt;
      return alo;
    }
    return 0.0;
  };
  double a_prev = 0.0, f_prev = f0, a = a1;
  for (int it = 0; it < max_evals; ++it) {
    double d;
    const double fa = phi(a, &d);
    if (approx_wolfe(fa, d)) { *f_out = fa; *g_out = gt; return a; }
    if (fa > f0 + c1 * a * d0 || (it > 0 && fa >= f_prev)) return zoom(a_prev, f_prev, a);
    if (std::fabs(d) <= -c2 * d0) { *f_out = fa; *g_out = gt; return a; }
    if (d >= 0) return zoom(a, fa, a_prev);
    a_prev = a;
    f_prev = fa;
    a *= 2.0;
  }
  return 0.0;
}

// Gauss-Jordan inverse with partial pivoting; false if singular.
bool invert(std::vector<double> A, int n, std::vector<double>* inv) {
  inv->assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) (*inv)[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    for (int k = 0; k < n; ++k) {
      std::swap(A[c * n + k], A[piv * n + k]);
      std::swap((*inv)[c * n + k], (*inv)[piv * n + k]);
    }
    const double d = A[c * n + c];
    for (int k = 0; k < n; ++k) { A[c * n + k] /= d; (*inv)[c * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; (*inv)[r * n + k] -= f * (*inv)[c * n + k]; }
    }
  }
  return true;
}

}  // namespace

int Problem::orc_nll_impl(const double* th, double* nll, double* g) {
  return orc_nll(reinterpret_cast<const orc_model*>(m), th, cols, N, nll, g, nullptr, nullptr);
}

extern "C" {

// Fit: theta0 (n_free; NULL = the PARAM nodes' values) -> theta_hat, nll_min,
// cov (n_free^2 or NULL), *n_evals.  Returns 0 converged, 1 not converged
// within max_evals, 2 line search failed, -2 start outside the domain.
int orc_fit(const orc_model* h, const double* const* cols, int64_t N, const double* theta0, double tol_edm,
            int max_evals, double* theta_hat, double* nll_min, double* cov, int* n_evals) {
  const Model& m = *reinterpret_cast<const Model*>(h);
  Problem pr;
  pr.m = &m;
  pr.cols = cols;
  pr.N = N;
  pr.P = m.n_free;
  const int P = pr.P;
  std::vector<double> th0(P);
  for (size_t i = 0; i < m.nodes.size(); ++i) {
    const Node& n = m.nodes[i];
    if (n.free_index < 0) continue;
    pr.lo.push_back(n.lo);
    pr.hi.push_back(n.hi);
    pr.bounded.push_back(n.lo < n.hi && std::isfinite(n.lo) && std::isfinite(n.hi));
    th0[n.free_index] = theta0 ? theta0[n.free_index] : n.value;
  }
  std::vector<double> x(P), g(P), H(P * P, 0.0);
  pr.to_internal(th0.data(), x.data());
  double f = pr.f(x.data(), g.data());
  if (!std::isfinite(f)) { *n_evals = pr.evals; return -2; }
  for (int k = 0; k < P; ++k) H[k * P + k] = 1.0;
  int status = 1;
  bool first = true;
  while (pr.evals < max_evals) {
    double edm = 0;
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) edm += 0.5 * g[i] * H[i * P + j] * g[j];
    if (edm < tol_edm) { status = 0; break; }
    std::vector<double> p(P, 0.0);
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) p[i] -= H[i * P + j] * g[j];
    if (dot(p, g) >= 0) {  // not a descent direction: restart from steepest descent
      std::fill(H.begin(), H.end(), 0.0);
      for (int k = 0; k < P; ++k) { H[k * P + k] = 1.0; p[k] = -g[k]; }
      first = true;
    }
    // N&W Sec. 3.5 leave the first trial step to the implementation; with a
    // fresh (identity) H the step -g carries the gradient's units, so its
    // first trial is limited to 0.5 in every internal coordinate (the sin
    // transform makes a bounded coordinate periodic: a longer step can land
    // anywhere in the parameter's range).  Later steps try 1 first (Alg. 6.1).
    double a1 = 1.0;
    if (first) {
      double pm = 0.0;
      for (int k = 0; k < P; ++k) pm = std::max(pm, std::fabs(p[k]));
      if (pm > 0.0) a1 = std::min(1.0, 0.5 / pm);
    }
    double fn;
    std::vector<double> gn(P);
    const double a = line_search(pr, x, f, g, p, &fn, &gn, 30, a1);
    if (a == 0.0) { status = 2; break; }
    std::vector<double> s(P), y(P);
    for (int k = 0; k < P; ++k) { s[k] = a * p[k]; y[k] = gn[k] - g[k]; }
    const double sy = dot(s, y);
    if (first && sy > 0) {  // N&W eq. 6.20: scale the initial inverse Hessian
      const double sc = sy / dot(y, y);
      for (int k = 0; k < P * P; ++k) H[k] *= sc;
    }
    first = false;
    if (sy > 1e-300) {
      // H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T
      const double rho = 1.0 / sy;
      std::vector<double> Hy(P, 0.0);
      for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j) Hy[i] += H[i * P + j] * y[j];
      const double yHy = dot(y, Hy);
      for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j)
          H[i * P + j] += -rho * (Hy[i] * s[j] + s[i] * Hy[j]) + (rho * rho * yHy + rho) * s[i] * s[j];
    }
    for (int k = 0; k < P; ++k) x[k] += s[k];
    f = fn;
    g = gn;
  }
  pr.to_theta(x.data(), theta_hat);
  *nll_min = f;
  if (cov) {
    // Hessian in theta by central differences of the analytic gradient.
    std::vector<double> Hs(P * P), tp(P), gp(P), gm(P);
    for (int k = 0; k < P; ++k) {
      const double hstep = 1e-5 * std::max(std::fabs(theta_hat[k]), 1e-2);
      for (int j = 0; j < P; ++j) tp[j] = theta_hat[j];
      double dummy;
      tp[k] = theta_hat[k] + hstep;
      pr.orc_nll_impl(tp.data(), &dummy, gp.data());
      tp[k] = theta_hat[k] - hstep;
      pr.orc_nll_impl(tp.data(), &dummy, gm.data());
      for (int j = 0; j < P; ++j) Hs[j * P + k] = (gp[j] - gm[j]) / (2.0 * hstep);
    }
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < i; ++j) Hs[i * P + j] = Hs[j * P + i] = 0.5 * (Hs[i * P + j] + Hs[j * P + i]);
    std::vector<double> C;
    if (invert(Hs, P, &C)) std::copy(C.begin(), C.end(), cov);
    else std::fill(cov, cov + P * P, std::numeric_limits<double>::quiet_NaN());
  }
  *n_evals = pr.evals;
  return status;
}

}  // extern "C"
