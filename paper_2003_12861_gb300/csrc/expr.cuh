// RF_EXPR leaves on the device: a density given as a short postfix program
// over the observable x, the node's parameters and constants, for PDFs that
// have no built-in kind (Sec. 5: a fall-back implementation for PDFs that
// have not been given batch code).  The generic graph interpreter evaluates
// it per event; its normalisation integral and the integral's parameter
// derivatives are computed per parameter point by adaptive Gauss-Kronrod
// quadrature, cooperatively by the parameter-point kernel's block.
#pragma once

#include <cuda_runtime.h>

#include "rf_internal.h"

namespace rf {

// The program's value at x and, for nd > 0, its derivatives in the node's
// first nd parameters (forward mode: each stack entry carries nd tangents).
// par: the node's n_par parameter values.  False outside the program's
// domain (log or pow of a value <= 0, division by 0) or for a result that
// is not finite.
__device__ inline bool expr_eval(const Program& P, const PNode& q, const double* par, double x, int nd, double* f,
                                 double* df) {
  double v[kExprStack], d[kExprStack][kMaxPar];
  int sp = 0;
  const int32_t* ops = P.ex_ops + q.ex_op0;
  const double* cs = P.ex_consts + q.ex_c0;
  for (int i = 0; i < q.ex_nops; ++i) {
    const int code = ops[i] & 0xff, arg = ops[i] >> 8;
    if (code <= RF_EX_CONST) {
      v[sp] = code == RF_EX_X ? x : code == RF_EX_PAR ? par[arg] : cs[arg];
      for (int k = 0; k < nd; ++k) d[sp][k] = (code == RF_EX_PAR && k == arg) ? 1.0 : 0.0;
      ++sp;
      continue;
    }
    const int a = sp - (code >= RF_EX_NEG && code <= RF_EX_LOG ? 1 : 2), b = a + 1;
    switch (code) {
      case RF_EX_NEG:
        v[a] = -v[a];
        for (int k = 0; k < nd; ++k) d[a][k] = -d[a][k];
        break;
      case RF_EX_EXP:
        v[a] = exp(v[a]);
        for (int k = 0; k < nd; ++k) d[a][k] *= v[a];
        break;
      case RF_EX_LOG:
        if (!(v[a] > 0.0)) return false;
        for (int k = 0; k < nd; ++k) d[a][k] /= v[a];
        v[a] = log(v[a]);
        break;
      case RF_EX_ADD:
        v[a] += v[b];
        for (int k = 0; k < nd; ++k) d[a][k] += d[b][k];
        break;
      case RF_EX_SUB:
        v[a] -= v[b];
        for (int k = 0; k < nd; ++k) d[a][k] -= d[b][k];
        break;
      case RF_EX_MUL:
        for (int k = 0; k < nd; ++k) d[a][k] = d[a][k] * v[b] + v[a] * d[b][k];
        v[a] *= v[b];
        break;
      case RF_EX_DIV: {
        if (v[b] == 0.0) return false;
        const double r = v[a] / v[b];
        for (int k = 0; k < nd; ++k) d[a][k] = (d[a][k] - r * d[b][k]) / v[b];
        v[a] = r;
        break;
      }
      default: {  // RF_EX_POW: a^b = exp(b log a), a > 0
        if (!(v[a] > 0.0)) return false;
        const double la = log(v[a]), r = exp(v[b] * la);
        for (int k = 0; k < nd; ++k) d[a][k] = r * (d[b][k] * la + v[b] * d[a][k] / v[a]);
        v[a] = r;
      }
    }
    sp = a + 1;
  }
  *f = v[0];
  bool ok = isfinite(v[0]);
  for (int k = 0; k < nd; ++k) {
    df[k] = d[0][k];
    ok = ok && isfinite(d[0][k]);
  }
  return ok;
}

// 15-point Gauss-Kronrod rule and its embedded 7-point Gauss rule on
// [-1, 1] (Kronrod 1965; the abscissae and weights as tabulated with
// QUADPACK's qk15): nodes +-kGK15x[i] with Kronrod weights kGK15w[i], the
// Gauss nodes being kGK15x[1], kGK15x[3], kGK15x[5] and 0 with weights kG7w.
__device__ __constant__ const double kGK15x[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851, 0.864864423359769072789712788640926,
    0.741531185599394439863864773280788, 0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.0};
__device__ __constant__ const double kGK15w[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204, 0.104790010322250183839876322541518,
    0.140653259715525918745189590510238, 0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
__device__ __constant__ const double kG7w[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

constexpr int kQuadPanels = 256;   // panels per refinement level (one per thread of the block)
constexpr int kQuadLevels = 16;    // refinement levels at most
constexpr double kQuadRel = 1e-14; // target error, relative to the integral

// Shared-memory workspace of the block-cooperative quadrature.
struct QuadSmem {
  double a[2][kQuadPanels], b[2][kQuadPanels];
  double red[kQuadPanels / 32][1 + kMaxPar];
  int scan[kQuadPanels];
  int bad;
};

// Sum of val[0..nv) over the block in a fixed order (lanes by butterfly,
// then warps in order): the same bits for the same inputs.  Block-wide,
// every thread gets the result.
__device__ inline void quad_block_sum(QuadSmem& s, double* val, int nv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < nv; ++k) {
    double x = val[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s.red[warp][k] = x;
  }
  __syncthreads();
  for (int k = 0; k < nv; ++k) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += s.red[w][k];
    val[k] = x;
  }
  __syncthreads();
}

// Integral of node q's program over [q.lo, q.hi] (out[0]) and its
// derivatives in the node's parameters (out[1..n_par]), by the whole block
// (blockDim.x == kQuadPanels).  Start: 16 equal panels.  At each level every
// thread takes one panel, the 15-point Kronrod sum and the embedded 7-point
// Gauss sum of the program; a panel whose two sums differ by at most
// kQuadRel |I| times its share of the range is accepted (its Kronrod sums are
// added), the others are halved for the next level, in order; when the next
// level would exceed kQuadPanels panels, or at the last level, all are
// accepted.  |I| is first estimated by the 16 panels' Kronrod sum.  Every
// sum has a fixed order, so the result depends only on the parameters.
// Returns false (on every thread) outside the program's domain or for I <= 0.
__device__ inline bool expr_integrate_block(const Program& P, const PNode& q, const double* par, QuadSmem& s,
                                            double* out) {
  const int t = threadIdx.x, np = q.n_par;
  const double lo = q.lo, hi = q.hi, span = hi - lo;
  if (t == 0) s.bad = 0;
  for (int k = 0; k <= np; ++k) out[k] = 0.0;
  int cur = 0, n_pan = 16;
  if (t < n_pan) {
    s.a[0][t] = lo + span * t / 16.0;
    s.b[0][t] = t == 15 ? hi : lo + span * (t + 1) / 16.0;
  }
  __syncthreads();
  double tol = 0.0;
  for (int level = 0; level < kQuadLevels && n_pan > 0; ++level) {
    double kr[1 + kMaxPar], g7 = 0.0;
    for (int k = 0; k <= np; ++k) kr[k] = 0.0;
    double width = 0.0;
    if (t < n_pan) {
      const double a = s.a[cur][t], b = s.b[cur][t];
      const double c = 0.5 * (a + b), h = 0.5 * (b - a);
      width = b - a;
      for (int i = 0; i < 15; ++i) {
        const int j = i < 7 ? i : i < 14 ? i - 7 : 7;
        const double x = i < 7 ? c - h * kGK15x[j] : i < 14 ? c + h * kGK15x[j] : c;
        double f, df[kMaxPar];
        if (!expr_eval(P, q, par, x, np, &f, df)) {
          atomicOr(&s.bad, 1);
          break;
        }
        const double w = kGK15w[j];
        kr[0] += w * f;
        for (int k = 0; k < np; ++k) kr[1 + k] += w * df[k];
        if (j & 1) g7 += kG7w[j >> 1] * f;
        else if (j == 7) g7 += kG7w[3] * f;
      }
      for (int k = 0; k <= np; ++k) kr[k] *= h;
      g7 *= h;
    }
    __syncthreads();
    if (s.bad) return false;
    if (level == 0) {  // the tolerance from the first estimate of |I|
      double e = fabs(kr[0]);
      quad_block_sum(s, &e, 1);
      tol = kQuadRel * e;
    }
    int split = (t < n_pan && fabs(kr[0] - g7) > tol * (width / span)) ? 1 : 0;
    // exclusive prefix sum of the split flags (a Hillis-Steele scan)
    s.scan[t] = split;
    __syncthreads();
    for (int o = 1; o < kQuadPanels; o <<= 1) {
      const int v = t >= o ? s.scan[t - o] : 0;
      __syncthreads();
      s.scan[t] += v;
      __syncthreads();
    }
    const int n_split = s.scan[kQuadPanels - 1];
    const int pref = s.scan[t] - split;
    __syncthreads();
    if (2 * n_split > kQuadPanels || level == kQuadLevels - 1) split = 0;  // accept all
    double contrib[1 + kMaxPar];
    for (int k = 0; k <= np; ++k) contrib[k] = (t < n_pan && !split) ? kr[k] : 0.0;
    quad_block_sum(s, contrib, 1 + np);
    for (int k = 0; k <= np; ++k) out[k] += contrib[k];
    if (2 * n_split > kQuadPanels || level == kQuadLevels - 1) break;
    if (split) {
      const double a = s.a[cur][t], b = s.b[cur][t], m = 0.5 * (a + b);
      s.a[cur ^ 1][2 * pref] = a;
      s.b[cur ^ 1][2 * pref] = m;
      s.a[cur ^ 1][2 * pref + 1] = m;
      s.b[cur ^ 1][2 * pref + 1] = b;
    }
    __syncthreads();
    cur ^= 1;
    n_pan = 2 * n_split;
  }
  return out[0] > 0.0 && isfinite(out[0]);
}

}  // namespace rf
