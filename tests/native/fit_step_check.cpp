// Host checks of the fit's shared quasi-Newton code (fit_step.h): its sine
// and cosine against the C library, and whole fits of functions whose
// minimum is known in closed form.  Prints one "name value" line per result.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "fit_step.h"

using namespace rf;

namespace {

// Drives one fit to the end: f_and_g(theta, grad_theta) -> f.
template <class F>
qn::State fit(int P, const std::vector<double>& lo, const std::vector<double>& hi, std::vector<double> theta0,
              double tol, int max_evals, F f_and_g, std::vector<double>* theta_out) {
  std::vector<char> bounded(P);
  for (int k = 0; k < P; ++k) bounded[k] = lo[k] < hi[k];
  std::vector<double> x(P), g(P), H(P * P), p(P), g_lo(P), trial(P), ws(P), wy(P), why(P), wr(P);
  for (int k = 0; k < P; ++k) H[k * P + k] = 1.0;
  for (int k = 0; k < P; ++k)
    trial[k] = bounded[k] ? std::asin(2.0 * (theta0[k] - lo[k]) / (hi[k] - lo[k]) - 1.0) : theta0[k];
  qn::State c = qn::initial_state();
  const qn::Vecs v{x.data(), g.data(), H.data(), p.data(), g_lo.data(), trial.data(),
                   ws.data(), wy.data(), why.data(), wr.data()};
  std::vector<double> th(P), jc(P), gt(P), ga(P);
  while (c.phase != qn::DONE) {
    qn::to_theta_jac(P, lo.data(), hi.data(), bounded.data(), trial.data(), th.data(), jc.data());
    const double fv = f_and_g(th, gt);
    for (int k = 0; k < P; ++k) ga[k] = gt[k] * jc[k];
    qn::deliver(P, c, v, fv, ga.data(), tol, max_evals);
  }
  theta_out->assign(P, 0.0);
  qn::to_theta_jac(P, lo.data(), hi.data(), bounded.data(), x.data(), theta_out->data(), nullptr);
  return c;
}

}  // namespace

int main() {
  // sine and cosine
  double es = 0.0, ec = 0.0, es_small = 0.0;
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> U(-60.0, 60.0);
  for (int i = 0; i < 200000; ++i) {
    const double x = i < 100000 ? U(rng) : std::ldexp(U(rng), -(i % 40));
    double s, c;
    qn::sin_cos(x, &s, &c);
    es = std::fmax(es, std::fabs(s - std::sin(x)));
    ec = std::fmax(ec, std::fabs(c - std::cos(x)));
    if (std::fabs(x) < 1.0 && x != 0.0) es_small = std::fmax(es_small, std::fabs(s - std::sin(x)) / std::fabs(std::sin(x)));
  }
  std::printf("sin_abs_err %.3e\ncos_abs_err %.3e\nsin_rel_err_small %.3e\n", es, ec, es_small);
  double s0, c0;
  qn::sin_cos(0.0, &s0, &c0);
  std::printf("sin0 %.17g\ncos0 %.17g\n", s0, c0);

  // a convex quadratic in 6 unbounded parameters: minimum at a
  {
    const int P = 6;
    std::vector<double> a = {1.0, -2.0, 0.5, 3.0, -1.5, 0.25}, A(P * P);
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) A[i * P + j] = (i == j ? 2.0 + i : 0.0) + 0.3 / (1.0 + i + j);
    std::vector<double> lo(P, 0.0), hi(P, 0.0), th;
    auto f = [&](const std::vector<double>& t, std::vector<double>& g) {
      double v = 0.0;
      for (int i = 0; i < P; ++i) {
        g[i] = 0.0;
        for (int j = 0; j < P; ++j) g[i] += A[i * P + j] * (t[j] - a[j]);
        v += 0.5 * (t[i] - a[i]) * g[i];
      }
      return v;
    };
    qn::State c = fit(P, lo, hi, std::vector<double>(P, 0.0), 1e-14, 1000, f, &th);
    double e = 0.0;
    for (int k = 0; k < P; ++k) e = std::fmax(e, std::fabs(th[k] - a[k]));
    std::printf("quad_status %d\nquad_err %.3e\nquad_evals %d\n", c.status, e, c.evals);
  }
  // Rosenbrock in two bounded parameters: minimum at (1, 1)
  {
    const int P = 2;
    std::vector<double> lo = {-2.0, -1.0}, hi = {2.0, 3.0}, th;
    auto f = [&](const std::vector<double>& t, std::vector<double>& g) {
      const double u = t[1] - t[0] * t[0], w = 1.0 - t[0];
      g[0] = -400.0 * t[0] * u - 2.0 * w;
      g[1] = 200.0 * u;
      return 100.0 * u * u + w * w;
    };
    qn::State c = fit(P, lo, hi, {-1.2, 1.0}, 1e-16, 2000, f, &th);
    std::printf("rosen_status %d\nrosen_err %.3e\nrosen_evals %d\n", c.status, std::fmax(std::fabs(th[0] - 1.0), std::fabs(th[1] - 1.0)), c.evals);
  }
  // the minimum of (theta - 5)^2 outside [0, 2]: the fit ends at the bound
  {
    std::vector<double> lo = {0.0}, hi = {2.0}, th;
    auto f = [&](const std::vector<double>& t, std::vector<double>& g) {
      g[0] = 2.0 * (t[0] - 5.0);
      return (t[0] - 5.0) * (t[0] - 5.0);
    };
    qn::State c = fit(1, lo, hi, {1.0}, 1e-10, 1000, f, &th);
    std::printf("bound_status %d\nbound_theta %.12f\n", c.status, th[0]);
  }
  // a start outside the domain (f not finite): RF_E_DOMAIN after one evaluation
  {
    std::vector<double> lo = {0.0}, hi = {0.0}, th;
    auto f = [&](const std::vector<double>&, std::vector<double>& g) {
      g[0] = 0.0;
      return HUGE_VAL;
    };
    qn::State c = fit(1, lo, hi, {1.0}, 1e-10, 1000, f, &th);
    std::printf("domain_status %d\ndomain_evals %d\n", c.status, c.evals);
  }
  // max_evals ends a fit that cannot converge in time
  {
    const int P = 2;
    std::vector<double> lo = {0.0, 0.0}, hi = {0.0, 0.0}, th;
    auto f = [&](const std::vector<double>& t, std::vector<double>& g) {
      const double u = t[1] - t[0] * t[0], w = 1.0 - t[0];
      g[0] = -400.0 * t[0] * u - 2.0 * w;
      g[1] = 200.0 * u;
      return 100.0 * u * u + w * w;
    };
    qn::State c = fit(P, lo, hi, {-1.2, 1.0}, 1e-16, 7, f, &th);
    std::printf("cap_status %d\ncap_evals %d\n", c.status, c.evals);
  }
  return 0;
}
