// Toy datasets on the device (Sec. 1: RooStats toy Monte Carlo) and their
// 64-bin histograms.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), a
// counter-based generator, so every event of every set is addressable on its
// own: key = (seed, seed >> 32), counter = (event, attempt, set, factor); the
// size draw uses counter (iteration, 0, set, 0xFFFFFFFF).  Uniforms take the
// top 53 bits of two words.  Set sizes: Poisson by inversion below mean 10,
// else by PTRS (W. Hoermann, "The transformed rejection method for generating
// Poisson random variables", 1993).  Events: accept-reject, independently for
// each factor of a product at the root, against 1.2 x the largest density on
// 4096 midpoints of the factor's range.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "expr.cuh"
#include "nll_kernels.cuh"

namespace rf {

namespace {

constexpr int kMaxFactors = 8;
constexpr uint32_t kMaxAttempts = 100000u;

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
  return (double)(((uint64_t)hi << 21) | (lo >> 11)) * 0x1.0p-53;
}
__device__ __forceinline__ double u53_open(uint32_t hi, uint32_t lo) {
  return __dmul_rn(__dadd_rn((double)(((uint64_t)hi << 21) | (lo >> 11)), 0.5), 0x1.0p-53);
}

// Forward values of every PDF node at one point (the full-precision formulas
// of the event kernel, without the adjoint).
__device__ void node_values(const Program& P, const double* __restrict__ C, const double* x, double* v) {
  for (int n = 0; n < P.n_pdf; ++n) {
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
        const double z = (s - u) * 0.70710678118654752440;
        const double f = z > 0.0 ? 0.5 * exp(-0.5 * u * u) * erfcx(z) : 0.5 * exp(s * (0.5 * s - u)) * erfc(z);
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
          t0 = t1;
          t1 = t2;
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
        v[n] = expr_eval(P, q, c + 1 + q.n_par, x[q.col], 0, &f, nullptr) ? f * c[0] : NAN;
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
}

struct GenArgs {
  int32_t n_factors;
  int32_t factor[kMaxFactors];  // program index of each factor
  int32_t fcol[kMaxFactors];    // its observable column
  double lo[kMaxFactors], hi[kMaxFactors];
};

// Accept-reject bound of (set, factor): one block per pair, 4096 midpoints.
__global__ void bounds_kernel(const __grid_constant__ Program P, const __grid_constant__ GenArgs g,
                              const double* __restrict__ consts, const int32_t* __restrict__ sets, double* bounds) {
  const int s = sets[blockIdx.x / g.n_factors], j = blockIdx.x % g.n_factors;
  const double* C = consts + (size_t)s * P.n_const;
  __shared__ double red[256];
  double mx = 0.0;
  double x[kMaxObs], v[kMaxPdf];
  for (int c = 0; c < kMaxObs; ++c) x[c] = 0.0;
  const double width = g.hi[j] - g.lo[j];
  for (int p = threadIdx.x; p < 4096; p += blockDim.x) {
    x[g.fcol[j]] = __dadd_rn(g.lo[j], __dmul_rn(width, (p + 0.5) / 4096.0));
    node_values(P, C, x, v);
    const double d = v[g.factor[j]];
    if (d > mx) mx = d;
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) bounds[(size_t)s * kMaxFactors + j] = 1.2 * red[0];
}

// Set sizes: Poisson(mean) (or round(mean) when poisson == 0), one thread per set.
__global__ void sizes_kernel(const double* __restrict__ mean_n, int n_sets, int poisson, uint32_t k0, uint32_t k1,
                             int64_t* __restrict__ sizes) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_sets) return;
  const double mu = mean_n[s];
  if (!poisson) {
    sizes[s] = (mu > 0.0) ? (int64_t)llrint(mu) : 0;
    return;
  }
  if (!(mu > 0.0)) {
    sizes[s] = 0;
    return;
  }
  uint32_t r[4];
  if (mu < 10.0) {
    philox4x32_10(0u, 0u, (uint32_t)s, 0xFFFFFFFFu, k0, k1, r);
    const double u = u53(r[0], r[1]);
    double p = exp(-mu), F = p;
    int64_t k = 0;
    while (u > F && k < 1000) {
      ++k;
      p = __dmul_rn(p, __ddiv_rn(mu, (double)k));
      F = __dadd_rn(F, p);
    }
    sizes[s] = k;
    return;
  }
  const double smu = sqrt(mu);
  const double b = __dadd_rn(0.931, __dmul_rn(2.53, smu));
  const double a = __dadd_rn(-0.059, __dmul_rn(0.02483, b));
  const double inv_alpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dsub_rn(b, 3.4)));
  const double vr = __dsub_rn(0.9277, __ddiv_rn(3.6224, __dsub_rn(b, 2.0)));
  const double log_mu = log(mu);
  for (uint32_t j = 0; j < 100000u; ++j) {
    philox4x32_10(j, 0u, (uint32_t)s, 0xFFFFFFFFu, k0, k1, r);
    const double U = __dsub_rn(u53_open(r[0], r[1]), 0.5);
    const double V = u53_open(r[2], r[3]);
    const double us = __dsub_rn(0.5, fabs(U));
    const double kd =
        floor(__dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, a), us), b), U), mu), 0.43));
    if (us >= 0.07 && V <= vr) {
      sizes[s] = (int64_t)kd;
      return;
    }
    if (kd < 0.0 || (us < 0.013 && V > us)) continue;
    const double lhs = __dsub_rn(__dadd_rn(log(V), log(inv_alpha)), log(__dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b)));
    const double rhs = __dsub_rn(__dadd_rn(-mu, __dmul_rn(kd, log_mu)), lgamma(__dadd_rn(kd, 1.0)));
    if (lhs <= rhs) {
      sizes[s] = (int64_t)kd;
      return;
    }
  }
  sizes[s] = -1;
}

// Events: one thread per event; the set comes from a binary search of the
// offsets.  Each factor's observable is drawn by accept-reject.
__global__ void events_kernel(const __grid_constant__ Program P, const __grid_constant__ GenArgs g,
                              const double* __restrict__ consts, const double* __restrict__ bounds,
                              const int64_t* __restrict__ offsets, int n_sets, int64_t n_events, uint32_t k0,
                              uint32_t k1, const __grid_constant__ Columns out, int32_t* __restrict__ error) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_events) return;
  int lo = 0, hi = n_sets - 1;  // last set with offsets[set] <= e
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  const int s = lo;
  const uint32_t i = (uint32_t)(e - offsets[s]);
  const double* C = consts + (size_t)s * P.n_const;
  double x[kMaxObs], v[kMaxPdf];
  for (int c = 0; c < kMaxObs; ++c) x[c] = 0.0;
  for (int j = 0; j < g.n_factors; ++j) {
    const int col = g.fcol[j];
    const double width = __dsub_rn(g.hi[j], g.lo[j]);
    const double M = bounds[(size_t)s * kMaxFactors + j];
    bool done = false;
    for (uint32_t a = 0; a < kMaxAttempts && !done; ++a) {
      uint32_t r[4];
      philox4x32_10(i, a, (uint32_t)s, (uint32_t)j, k0, k1, r);
      const double xv = __dadd_rn(g.lo[j], __dmul_rn(width, u53(r[0], r[1])));
      const double y = __dmul_rn(M, u53(r[2], r[3]));
      x[col] = xv;
      node_values(P, C, x, v);
      if (y < v[g.factor[j]]) {
        if (out.is_f32[col]) ((float*)out.ptr[col])[e] = (float)xv;
        else ((double*)out.ptr[col])[e] = xv;
        done = true;
      }
    }
    x[col] = 0.0;
    if (!done) atomicExch(error, 1);
  }
}

// Per-set 64-bin histogram, one block per set.
__global__ void hist64_kernel(const __grid_constant__ Columns cols, int col, const int64_t* __restrict__ offsets,
                              double lo, double scale, float* __restrict__ out) {
  __shared__ int bins[64];
  const int s = blockIdx.x;
  if (threadIdx.x < 64) bins[threadIdx.x] = 0;
  __syncthreads();
  const int64_t b0 = offsets[s], b1 = offsets[s + 1];
  for (int64_t e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
    const double xv = cols.is_f32[col] ? (double)((const float*)cols.ptr[col])[e] : ((const double*)cols.ptr[col])[e];
    int b = (int)floor(__dmul_rn(__dsub_rn(xv, lo), scale));
    b = min(63, max(0, b));
    atomicAdd(&bins[b], 1);
  }
  __syncthreads();
  if (threadIdx.x < 64) {
    const int64_t n = b1 - b0;
    out[(size_t)s * 64 + threadIdx.x] = n > 0 ? (float)((double)bins[threadIdx.x] / (double)n) : 0.0f;
  }
}

}  // namespace

}  // namespace rf

using namespace rf;

extern "C" {

rf_status rf_generate_toys(const rf_model* m, const double* theta, int32_t theta_per_set, uint64_t seed,
                           int32_t n_sets, const double* mean_n, int32_t poisson, const int32_t* dtype,
                           rf_data** out) {
  if (!m || !out || n_sets < 1 || !mean_n) {
    set_error("rf_generate_toys: bad argument");
    return RF_E_INVALID;
  }
  *out = nullptr;
  const Model& mm = m->m;
  const Program& P = mm.prog;
  if (mm.gen_factors.empty() || (int)mm.gen_factors.size() > kMaxFactors) {
    set_error("rf_generate_toys: the model must be a product of 1-D factors (or one 1-D pdf)");
    return RF_E_INVALID;
  }
  for (int s = 0; s < n_sets; ++s)
    if (!(mean_n[s] >= 0.0) || mean_n[s] > 2e9) {
      set_error("rf_generate_toys: mean sizes must be in [0, 2e9]");
      return RF_E_INVALID;
    }
  const int nf = P.n_free;
  std::vector<double> th((size_t)n_sets * nf);
  for (int s = 0; s < n_sets; ++s)
    for (int k = 0; k < nf; ++k)
      th[(size_t)s * nf + k] = theta ? theta[(theta_per_set ? (size_t)s * nf : 0) + k] : mm.theta_default[k];

  GenArgs g{};
  g.n_factors = (int)mm.gen_factors.size();
  for (int j = 0; j < g.n_factors; ++j) {
    const PNode& q = P.node[mm.gen_factors[j]];
    g.factor[j] = mm.gen_factors[j];
    // the factor's observable: the column of its first leaf
    int n = mm.gen_factors[j];
    while (P.node[n].kind == SUM || P.node[n].kind == PROD) n = P.node[n].child[0];
    g.fcol[j] = P.node[n].col;
    g.lo[j] = mm.obs_lo[g.fcol[j]];
    g.hi[j] = mm.obs_hi[g.fcol[j]];
    (void)q;
  }
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);

  // Constants of the generating parameters (the parameter-point kernel).
  DevBuf d_theta, d_consts, d_sets, d_flags, d_out, d_counter, d_bounds, d_mean, d_sizes, d_err;
  std::vector<int32_t> sets(n_sets);
  for (int s = 0; s < n_sets; ++s) sets[s] = s;
  if (!d_theta.ensure(sizeof(double) * std::max<size_t>(1, th.size())) ||
      !d_consts.ensure(sizeof(double) * n_sets * std::max(1, P.n_const)) || !d_sets.ensure(sizeof(int32_t) * n_sets) ||
      !d_flags.ensure(sizeof(int32_t) * n_sets) || !d_out.ensure(sizeof(double) * n_sets * (1 + nf)) ||
      !d_counter.ensure(sizeof(int32_t)) || !d_bounds.ensure(sizeof(double) * n_sets * kMaxFactors) ||
      !d_mean.ensure(sizeof(double) * n_sets) || !d_sizes.ensure(sizeof(int64_t) * n_sets) || !d_err.ensure(sizeof(int32_t)))
    return RF_E_OOM;
  std::vector<int64_t> zero_off(n_sets + 1, 1);  // every set "non-empty" for the parameter-point pass
  DevBuf d_zoff;
  for (int s = 0; s <= n_sets; ++s) zero_off[s] = s;
  if (!d_zoff.ensure(sizeof(int64_t) * (n_sets + 1))) return RF_E_OOM;
  bool ok = cuda_ok(cudaMemcpy(d_theta.p, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice), "theta") &&
            cuda_ok(cudaMemcpy(d_sets.p, sets.data(), sizeof(int32_t) * n_sets, cudaMemcpyHostToDevice), "sets") &&
            cuda_ok(cudaMemcpy(d_mean.p, mean_n, sizeof(double) * n_sets, cudaMemcpyHostToDevice), "mean") &&
            cuda_ok(cudaMemcpy(d_zoff.p, zero_off.data(), sizeof(int64_t) * (n_sets + 1), cudaMemcpyHostToDevice), "off") &&
            cuda_ok(cudaMemset(d_err.p, 0, sizeof(int32_t)), "memset");
  if (!ok) return RF_E_CUDA;
  Pass pass{};
  pass.offsets = (const int64_t*)d_zoff.p;
  pass.sets = (const int32_t*)d_sets.p;
  pass.n_active = n_sets;
  pass.theta = (const double*)d_theta.p;
  pass.consts = (double*)d_consts.p;
  pass.counter = (int32_t*)d_counter.p;
  pass.out = (double*)d_out.p;
  pass.flags = (int32_t*)d_flags.p;
  pass.Q = 1;
  launch_param_point(P, pass, 0);
  std::vector<int32_t> flags(n_sets);
  if (!cuda_ok(cudaMemcpy(flags.data(), d_flags.p, sizeof(int32_t) * n_sets, cudaMemcpyDeviceToHost), "flags"))
    return RF_E_CUDA;
  for (int s = 0; s < n_sets; ++s)
    if (flags[s]) {
      set_error("rf_generate_toys: generating parameters outside the pdf's domain");
      return RF_E_DOMAIN;
    }
  note_launches(1, nullptr);
  bounds_kernel<<<n_sets * g.n_factors, 256>>>(P, g, (const double*)d_consts.p, (const int32_t*)d_sets.p,
                                               (double*)d_bounds.p);
  note_launches(1, nullptr);
  sizes_kernel<<<(n_sets + 127) / 128, 128>>>((const double*)d_mean.p, n_sets, poisson, k0, k1,
                                              (int64_t*)d_sizes.p);
  std::vector<int64_t> sizes(n_sets);
  if (!cuda_ok(cudaGetLastError(), "launch") ||
      !cuda_ok(cudaMemcpy(sizes.data(), d_sizes.p, sizeof(int64_t) * n_sets, cudaMemcpyDeviceToHost), "sizes"))
    return RF_E_CUDA;
  std::vector<int64_t> off(n_sets + 1, 0);
  for (int s = 0; s < n_sets; ++s) {
    if (sizes[s] < 0) {
      set_error("rf_generate_toys: Poisson draw did not terminate");
      return RF_E_TIMEOUT;
    }
    off[s + 1] = off[s] + sizes[s];
  }
  rf_data* d = new (std::nothrow) rf_data();
  if (!d) return RF_E_OOM;
  d->n_obs = P.n_obs;
  d->n_sets = n_sets;
  d->n_events = off[n_sets];
  d->offsets = off;
  d->owns_cols = true;
  Columns outc{};
  for (int c = 0; c < P.n_obs; ++c) {
    d->dtype[c] = dtype ? dtype[c] : RF_F64;
    if (d->dtype[c] != RF_F64 && d->dtype[c] != RF_F32) {
      delete d;
      set_error("rf_generate_toys: dtype must be RF_F64 or RF_F32");
      return RF_E_INVALID;
    }
    if (!d->col_bufs[c].ensure((size_t)std::max<int64_t>(1, d->n_events) * (d->dtype[c] == RF_F32 ? 4 : 8))) {
      delete d;
      return RF_E_OOM;
    }
    d->cols[c] = d->col_bufs[c].p;
    outc.ptr[c] = d->cols[c];
    outc.is_f32[c] = d->dtype[c] == RF_F32;
  }
  rf_status st = finish_data(d);
  if (st != RF_OK) {
    delete d;
    return st;
  }
  if (d->n_events > 0) {
    const int64_t blocks = (d->n_events + 127) / 128;
    note_launches(1, nullptr);
    events_kernel<<<(unsigned)blocks, 128>>>(P, g, (const double*)d_consts.p, (const double*)d_bounds.p,
                                             (const int64_t*)d->offsets_dev.p, n_sets, d->n_events, k0, k1, outc,
                                             (int32_t*)d_err.p);
  }
  int32_t err = 0;
  if (!cuda_ok(cudaGetLastError(), "launch") ||
      !cuda_ok(cudaMemcpy(&err, d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost), "generation")) {
    delete d;
    return RF_E_CUDA;
  }
  if (err) {
    delete d;
    set_error("rf_generate_toys: an event needed more than 100000 accept-reject attempts");
    return RF_E_TIMEOUT;
  }
  *out = d;
  return RF_OK;
}

rf_status rf_hist64(const rf_model* m, const rf_data* d, int32_t col, float* d_out, void* stream) {
  if (!m || !d || !d_out || col < 0 || col >= d->n_obs || d->n_obs != m->m.prog.n_obs) {
    set_error("rf_hist64: bad argument");
    return RF_E_INVALID;
  }
  Columns c{};
  for (int i = 0; i < d->n_obs; ++i) {
    c.ptr[i] = d->cols[i];
    c.is_f32[i] = d->dtype[i] == RF_F32;
  }
  const double lo = m->m.obs_lo[col], hi = m->m.obs_hi[col];
  note_launches(1, (cudaStream_t)stream);
  hist64_kernel<<<d->n_sets, 256, 0, (cudaStream_t)stream>>>(c, col, (const int64_t*)d->offsets_dev.p, lo,
                                                            64.0 / (hi - lo), d_out);
  return cuda_ok(cudaGetLastError(), "rf_hist64 launch") ? RF_OK : RF_E_CUDA;
}

}  // extern "C"
