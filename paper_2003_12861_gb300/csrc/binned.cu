// Binned (HistFactory-style) likelihood: NLL and gradient of many datasets
// of bin counts at once (paper Sec. 3: models built from histograms --
// channels of samples with +-1 sigma systematic variations).
//
// nu_s[i] = prod(normfactors) prod(normsys eta) (h_s[i] + sum histosys
// delta), eta = exp(a alpha + b g(alpha)) with a, b = (log k_hi -+ log
// k_lo)/2, delta_i = a_i alpha + b_i g(alpha) with a_i = (h_hi - h_lo)/2,
// b_i = (h_hi + h_lo)/2 - h, g = alpha^2 inside +-1 and 2|alpha| - 1
// beyond (quadratic interpolation, linear extrapolation: continuous with a
// continuous derivative, so quasi-Newton fits see no kink); nu_b = sum over
// the samples on bin b; NLL = sum_b (nu_b - n_b log nu_b) + sum over
// constrained parameters theta^2/2.  d NLL / d theta_k = sum_b w_b d nu_b /
// d theta_k + [constrained] theta_k, w_b = 1 - n_b / nu_b; per modifier of
// parameter k: a normfactor or normsys on sample s contributes dlog(factor)
// / dtheta_k sum_i w nu_s[i], a histosys F_s sum_i w (a_i + b_i g').
//
// One block per dataset (persistent over datasets), every sum in a fixed
// order (each thread's bins / samples / modifiers in index order, a fixed
// tree across threads), so results do not depend on the launch.  The two
// loops that carry nearly all the multiply-adds -- the entries' histosys
// sums and the histosys modifiers' weighted coefficient sums -- and the
// samples' weighted sums run in float-float on the FP32 pipe (ff.cuh: FP64
// issues at 1/58 of the FP32 rate); the sample factors, the bins' Poisson
// terms and weights, the gradient's assembly and the expected counts stay
// in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "ff.cuh"

namespace rf {

namespace {

constexpr int kBinnedThreads = 256;
constexpr int kMaxBinnedBins = 8192, kMaxBinnedSamples = 2048;

// Dynamic shared memory of the kernels (8-byte slots): theta, F and Ssum per
// sample, W per bin (a float pair), one partial sum per thread, g and g' per
// parameter, then theta, g and F as float pairs.
size_t binned_smem(int n_params, int n_samples, int n_bins) {
  return sizeof(double) * (5 * (size_t)n_params + 3 * (size_t)n_samples + (size_t)n_bins + kBinnedThreads);
}

enum ModKind : int32_t { MOD_NORMFACTOR = 0, MOD_NORMSYS = 1, MOD_HISTOSYS = 2 };

struct BinnedDev {
  int32_t n_bins, n_samples, n_params, n_mods, n_entries, n_hs;
  const int32_t* bin0;        // per sample: first bin
  const int32_t* nb;          // per sample: bins
  const int32_t* eofs;        // per sample: its first (sample, bin) entry; entries run sample by sample
  const int32_t* esample;     // per entry: its sample
  const double* nominal;      // per entry
  const int32_t* smod_start;  // per sample: its normfactor / normsys modifiers (CSR, modifier order)
  const int32_t* smod;
  const int32_t* shs_start;   // per sample: its histosys modifiers (CSR, modifier order), as indices
  const int32_t* shs;         //   into the histosys arrays below
  const int32_t* kind;        // per modifier
  const int32_t* param;
  const int32_t* msample;
  const int32_t* mhs;         // per modifier: its histosys index, or -1
  const double* ns_a;         // normsys: a, b of log eta = a alpha + b g(alpha)
  const double* ns_b;
  const int32_t* hs_param;    // per histosys: parameter, sample
  const int32_t* hs_sample;
  const int64_t* hs_ofs;      // per histosys: a_i then b_i, nb each, in `coef`
  const double* coef;
  // The same coefficients transposed per sample for the weighted sums:
  // sample s's histosys j (its j-th in shs order) at local bin i sits at
  // tbase[s] + i * (histosys of s) + j, in coef_a and coef_b.
  const int64_t* tbase;
  const int32_t* g_sample;    // per position in shs: its sample
  const double* coef_a;
  const double* coef_b;
  // The nominal rates and the histosys coefficients again as float pairs
  // (same indexing), for the float-float loops.
  const float2* nominal_f;
  const float2* coef_f;
  const int32_t* shs_k;       // per position in shs: the histosys's parameter and
  const int64_t* shs_ofs;     //   coefficient offset (one load level instead of two)
  const float2* coef_af;
  const float2* coef_bf;
  const int32_t* bin_start;   // per bin: its entries (CSR, sample order)
  const int32_t* bin_entry;
  const int32_t* pmod_start;  // per parameter: its modifiers (CSR, modifier order)
  const int32_t* pmod;
  const int32_t* constrained;
};

// theta, g(theta) and g'(theta) into smem (once per parameter and dataset:
// an FP64 comparison per term would occupy the FP64 unit as long as the
// multiply-add itself), then the sample factors F: the normfactors times
// one exponential of the normsys exponents' sum.
__device__ __forceinline__ void sample_factors(const BinnedDev& m, const double* th_g, double* th, double* gk,
                                               double* dgk, double* F) {
  for (int k = threadIdx.x; k < m.n_params; k += kBinnedThreads) {
    const double a = th_g[k];
    th[k] = a;
    const bool in = fabs(a) <= 1.0;
    gk[k] = in ? a * a : 2.0 * fabs(a) - 1.0;
    dgk[k] = in ? 2.0 * a : (a > 0.0 ? 2.0 : -2.0);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < m.n_samples; s += kBinnedThreads) {
    double f = 1.0, le = 0.0;
    for (int j = m.smod_start[s]; j < m.smod_start[s + 1]; ++j) {
      const int md = m.smod[j], k = m.param[md];
      if (m.kind[md] == MOD_NORMFACTOR) f *= th[k];
      else le = fma(m.ns_b[md], gk[k], fma(m.ns_a[md], th[k], le));
    }
    F[s] = le != 0.0 ? f * exp(le) : f;
  }
  __syncthreads();
}

// nu of every (sample, bin) entry: consecutive threads take consecutive
// bins of a sample, so its histosys coefficients are read coalesced.
__device__ __forceinline__ void entry_rates(const BinnedDev& m, const double* th, const double* gk, const double* F,
                                            double* nu_e) {
  for (int e = threadIdx.x; e < m.n_entries; e += kBinnedThreads) {
    const int s = m.esample[e], i = e - m.eofs[s], n = m.nb[s];
    double shape = m.nominal[e];
    for (int j = m.shs_start[s]; j < m.shs_start[s + 1]; ++j) {
      const int h = m.shs[j], k = m.hs_param[h];
      const double* c = m.coef + m.hs_ofs[h] + i;
      shape = fma(c[n], gk[k], fma(c[0], th[k], shape));
    }
    nu_e[e] = F[s] * shape;
  }
}

__device__ __forceinline__ ff ld_pair(const float2* p) {
  const float2 v = __ldg(p);
  return {v.x, v.y};
}
__device__ __forceinline__ ff as_ff(double v) { return ff_from_double(v); }

// The same rates in float-float from the pairs' copies of the constants:
// thf, gkf, Ff = theta, g, F as pairs.
__device__ __forceinline__ void entry_rates_ff(const BinnedDev& m, const ff* thf, const ff* gkf, const ff* Ff,
                                               ff* nu_e) {
  for (int e = threadIdx.x; e < m.n_entries; e += kBinnedThreads) {
    const int s = m.esample[e], i = e - m.eofs[s], n = m.nb[s];
    ff shape = ld_pair(m.nominal_f + e);
    const int j1 = m.shs_start[s + 1];
#pragma unroll 4
    for (int j = m.shs_start[s]; j < j1; ++j) {
      const int k = __ldg(m.shs_k + j);
      const float2* c = m.coef_f + __ldg(m.shs_ofs + j) + i;
      shape = ff_fma(ld_pair(c + n), gkf[k], ff_fma(ld_pair(c), thf[k], shape));
    }
    nu_e[e] = ff_mul(Ff[s], shape);
  }
}

// out[set]: NLL then gradient (1 + n_params); flags[set]: 1 if some bin has
// nu <= 0 (NLL +inf).  scratch: per block n_entries (entry rates) +
// n_hs (histosys sums) doubles.
// sets: null, or the dataset (row of counts) of each of the n_sets points.
__global__ void __launch_bounds__(kBinnedThreads) binned_kernel(const BinnedDev m, int n_sets, const int32_t* sets,
                                                                 const double* counts, const double* theta,
                                                                 double* out, int32_t* flags, double* scratch) {
  extern __shared__ double smem[];
  double* th = smem;
  double* F = th + m.n_params;
  double* Ssum = F + m.n_samples;
  ff* W = reinterpret_cast<ff*>(Ssum + m.n_samples);
  double* part = reinterpret_cast<double*>(W + m.n_bins);
  double* gk = part + kBinnedThreads;
  double* dgk = gk + m.n_params;
  ff* thf = reinterpret_cast<ff*>(dgk + m.n_params);
  ff* gkf = thf + m.n_params;
  ff* Ff = gkf + m.n_params;
  __shared__ int bad;
  const int tid = threadIdx.x;
  ff* nu_e = reinterpret_cast<ff*>(scratch + (size_t)blockIdx.x * (m.n_entries + m.n_hs));
  double* T = reinterpret_cast<double*>(nu_e + m.n_entries);
  for (int set = blockIdx.x; set < n_sets; set += gridDim.x) {
    const double* n = counts + (size_t)(sets ? sets[set] : set) * m.n_bins;
    if (tid == 0) bad = 0;
    sample_factors(m, theta + (size_t)set * m.n_params, th, gk, dgk, F);
    for (int k = tid; k < m.n_params; k += kBinnedThreads) {
      thf[k] = as_ff(th[k]);
      gkf[k] = as_ff(gk[k]);
    }
    for (int s = tid; s < m.n_samples; s += kBinnedThreads) Ff[s] = as_ff(F[s]);
    __syncthreads();
    entry_rates_ff(m, thf, gkf, Ff, nu_e);
    __syncthreads();
    // bins: expected count, weight 1 - n/nu, the Poisson term
    double acc = 0.0;
    for (int b = tid; b < m.n_bins; b += kBinnedThreads) {
      ff nf = {0.0f, 0.0f};
      const int j1 = m.bin_start[b + 1];
#pragma unroll 4
      for (int j = m.bin_start[b]; j < j1; ++j) nf = ff_add(nf, nu_e[__ldg(m.bin_entry + j)]);
      const double nu = ff_to_double(nf);
      if (!(nu > 0.0) || !isfinite(nu)) {
        bad = 1;
        W[b] = {0.0f, 0.0f};
        continue;
      }
      W[b] = as_ff(1.0 - n[b] / nu);
      acc += nu - (n[b] != 0.0 ? n[b] * log(nu) : 0.0);
    }
    part[tid] = acc;
    __syncthreads();
    // per sample sum_i w nu_s[i]; per histosys sum_i w (a_i + b_i g')
    for (int s = tid; s < m.n_samples; s += kBinnedThreads) {
      ff a = {0.0f, 0.0f};
      const int nbs = m.nb[s], b0 = m.bin0[s], e0 = m.eofs[s];
#pragma unroll 4
      for (int i = 0; i < nbs; ++i) ff_acc_mul(a, W[b0 + i], nu_e[e0 + i]);
      Ssum[s] = ff_to_double(a);
    }
    // (a thread each, bins in order; consecutive threads read consecutive
    // coefficients of the transposed layout)
    for (int g = tid; g < m.n_hs; g += kBinnedThreads) {
      const int s = m.g_sample[g], h = m.shs[g];
      const int nh = m.shs_start[s + 1] - m.shs_start[s], j = g - m.shs_start[s];
      const float2* ca = m.coef_af + m.tbase[s] + j;
      const float2* cb = m.coef_bf + m.tbase[s] + j;
      const ff* w = W + m.bin0[s];
      ff ta = {0.0f, 0.0f}, tb = {0.0f, 0.0f};
      const int nbs = m.nb[s];
#pragma unroll 4
      for (int i = 0; i < nbs; ++i) {
        ff_acc_mul(ta, w[i], ld_pair(ca + (size_t)i * nh));
        ff_acc_mul(tb, w[i], ld_pair(cb + (size_t)i * nh));
      }
      T[h] = fma(dgk[m.hs_param[h]], ff_to_double(tb), ff_to_double(ta));
    }
    // NLL: the threads' partial sums by a fixed tree
    for (int o = kBinnedThreads / 2; o > 0; o >>= 1) {
      __syncthreads();
      if (tid < o) part[tid] += part[tid + o];
    }
    __syncthreads();
    double* o = out + (size_t)set * (1 + m.n_params);
    // gradient: each parameter's modifiers in order, then its constraint
    for (int k = tid; k < m.n_params; k += kBinnedThreads) {
      double g = 0.0;
      const double a = th[k];
      for (int j = m.pmod_start[k]; j < m.pmod_start[k + 1]; ++j) {
        const int md = m.pmod[j], s = m.msample[md];
        if (m.kind[md] == MOD_NORMFACTOR) g += Ssum[s] / a;
        else if (m.kind[md] == MOD_NORMSYS) g += Ssum[s] * fma(m.ns_b[md], dgk[k], m.ns_a[md]);
        else g += F[s] * T[m.mhs[md]];
      }
      if (m.constrained[k]) g += a;
      o[1 + k] = g;
    }
    if (tid == 0) {
      double c = 0.0;
      for (int k = 0; k < m.n_params; ++k)
        if (m.constrained[k]) c += 0.5 * th[k] * th[k];
      o[0] = bad ? INFINITY : part[0] + c;
      flags[set] = bad;
    }
    __syncthreads();
  }
}

// Expected counts nu_b per dataset (for generating toys).
__global__ void __launch_bounds__(kBinnedThreads) binned_expected_kernel(const BinnedDev m, int n_sets,
                                                                          const double* theta, double* nu_out,
                                                                          double* scratch) {
  extern __shared__ double smem[];
  double* th = smem;
  double* F = th + m.n_params;
  double* gk = F + m.n_samples;
  double* dgk = gk + m.n_params;
  double* nu_e = scratch + (size_t)blockIdx.x * (m.n_entries + m.n_hs);
  for (int set = blockIdx.x; set < n_sets; set += gridDim.x) {
    sample_factors(m, theta + (size_t)set * m.n_params, th, gk, dgk, F);
    entry_rates(m, th, gk, F, nu_e);
    __syncthreads();
    for (int b = threadIdx.x; b < m.n_bins; b += kBinnedThreads) {
      double nu = 0.0;
      for (int j = m.bin_start[b]; j < m.bin_start[b + 1]; ++j) nu += nu_e[m.bin_entry[j]];
      nu_out[(size_t)set * m.n_bins + b] = nu;
    }
    __syncthreads();
  }
}

}  // namespace

}  // namespace rf

// ---------------------------------------------------------------- handle

struct rf_binned {
  int32_t n_bins = 0, n_samples = 0, n_params = 0, n_mods = 0, n_entries = 0, n_hs = 0;
  rf::DevBuf bin0, nb, eofs, esample, nominal, smod_start, smod, shs_start, shs, kind, param, msample, mhs, ns_a,
      ns_b, hs_param, hs_sample, hs_ofs, coef, tbase, g_sample, coef_a, coef_b, bin_start, bin_entry, pmod_start, pmod,
      constrained, nominal_f, coef_f, coef_af, coef_bf, shs_k, shs_ofs;
  rf::DevBuf scratch, counts, theta, out, flags, sets;
  rf::HostBuf h_out, h_flags, h_theta, h_sets;
  rf::BinnedDev dev{};
  int grid = 0;
  size_t smem = 0;
};

using namespace rf;

namespace {

template <class T>
bool upload(DevBuf& b, const std::vector<T>& v) {
  if (!b.ensure(sizeof(T) * std::max<size_t>(1, v.size()))) return false;
  return v.empty() || cuda_ok(cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice), "binned upload");
}

rf_status launch_binned(rf_binned* m, int32_t n_sets, const double* d_counts, const double* d_theta, double* d_out,
                        int32_t* d_flags, cudaStream_t st, const int32_t* d_sets = nullptr) {
  if (n_sets == 0) return RF_OK;
  const int grid = std::min(n_sets, m->grid);
  note_launches(1, st);
  binned_kernel<<<grid, kBinnedThreads, m->smem, st>>>(m->dev, n_sets, d_sets, d_counts, d_theta, d_out, d_flags,
                                                        (double*)m->scratch.p);
  return cuda_ok(cudaGetLastError(), "binned launch") ? RF_OK : RF_E_CUDA;
}

}  // namespace

extern "C" {

rf_status rf_binned_create(int32_t n_bins, int32_t n_samples, const int32_t* bin0, const int32_t* nbins,
                           const double* nominal, int32_t n_params, const int32_t* constrained, int32_t n_mods,
                           const rf_modifier* mods, const double* hist_data, rf_binned** out) {
  if (!out || n_bins < 1 || n_bins > kMaxBinnedBins || n_samples < 1 || n_samples > kMaxBinnedSamples ||
      n_params < 0 || n_mods < 0 || !bin0 || !nbins || !nominal || (n_params > 0 && !constrained) ||
      (n_mods > 0 && !mods)) {
    set_error("rf_binned_create: bad argument (1 <= bins <= 8192, 1 <= samples <= 2048)");
    return RF_E_INVALID;
  }
  *out = nullptr;
  std::vector<int32_t> eofs(n_samples), esample;
  int64_t total = 0;
  for (int s = 0; s < n_samples; ++s) {
    if (nbins[s] < 1 || bin0[s] < 0 || bin0[s] + nbins[s] > n_bins) {
      set_error("rf_binned_create: a sample's bins lie outside the model's bins");
      return RF_E_INVALID;
    }
    eofs[s] = (int32_t)total;
    total += nbins[s];
    for (int i = 0; i < nbins[s]; ++i) esample.push_back(s);
  }
  if (total > (int64_t)1 << 30) {
    set_error("rf_binned_create: too many (sample, bin) entries");
    return RF_E_INVALID;
  }
  std::vector<int32_t> kind(n_mods), param(n_mods), msample(n_mods), mhs(n_mods, -1);
  std::vector<double> ns_a(n_mods, 0.0), ns_b(n_mods, 0.0);
  std::vector<int32_t> hs_param, hs_sample;
  std::vector<int64_t> hs_ofs;
  std::vector<double> coef;
  int64_t hd = 0;
  for (int j = 0; j < n_mods; ++j) {
    const rf_modifier& md = mods[j];
    if (md.sample < 0 || md.sample >= n_samples || md.param < 0 || md.param >= n_params || md.kind < 0 ||
        md.kind > 2) {
      set_error("rf_binned_create: bad modifier");
      return RF_E_INVALID;
    }
    if (md.kind == RF_MOD_NORMSYS && !(md.k_lo > 0.0 && md.k_hi > 0.0)) {
      set_error("rf_binned_create: normsys factors must be positive");
      return RF_E_INVALID;
    }
    kind[j] = md.kind;
    param[j] = md.param;
    msample[j] = md.sample;
    if (md.kind == RF_MOD_NORMSYS) {
      ns_a[j] = 0.5 * (std::log(md.k_hi) - std::log(md.k_lo));
      ns_b[j] = 0.5 * (std::log(md.k_hi) + std::log(md.k_lo));
    }
    if (md.kind == RF_MOD_HISTOSYS) {
      if (!hist_data) {
        set_error("rf_binned_create: histosys modifiers need hist_data");
        return RF_E_INVALID;
      }
      const int n = nbins[md.sample];
      const double* h = nominal + eofs[md.sample];
      const double *lo = hist_data + hd, *hi = hist_data + hd + n;
      mhs[j] = (int32_t)hs_param.size();
      hs_param.push_back(md.param);
      hs_sample.push_back(md.sample);
      hs_ofs.push_back((int64_t)coef.size());
      for (int i = 0; i < n; ++i) coef.push_back(0.5 * (hi[i] - lo[i]));
      for (int i = 0; i < n; ++i) coef.push_back(0.5 * (hi[i] + lo[i]) - h[i]);
      hd += 2 * (int64_t)n;
    }
  }
  const int n_hs = (int)hs_param.size();
  // CSR lists: factor modifiers and histosys per sample, modifiers per
  // parameter (modifier order), the entries of each bin (sample order).
  std::vector<int32_t> smod_start(n_samples + 1, 0), shs_start(n_samples + 1, 0), pmod_start(n_params + 1, 0);
  for (int j = 0; j < n_mods; ++j) {
    (kind[j] == RF_MOD_HISTOSYS ? shs_start : smod_start)[msample[j] + 1]++;
    pmod_start[param[j] + 1]++;
  }
  for (int s = 0; s < n_samples; ++s) {
    smod_start[s + 1] += smod_start[s];
    shs_start[s + 1] += shs_start[s];
  }
  for (int k = 0; k < n_params; ++k) pmod_start[k + 1] += pmod_start[k];
  std::vector<int32_t> smod(smod_start[n_samples]), shs(shs_start[n_samples]), pmod(n_mods);
  std::vector<int32_t> sfill(smod_start.begin(), smod_start.end() - 1), hfill(shs_start.begin(), shs_start.end() - 1),
      pfill(pmod_start.begin(), pmod_start.end() - 1);
  for (int j = 0; j < n_mods; ++j) {
    if (kind[j] == RF_MOD_HISTOSYS) shs[hfill[msample[j]]++] = mhs[j];
    else smod[sfill[msample[j]]++] = j;
    pmod[pfill[param[j]]++] = j;
  }
  // transposed coefficients per sample
  std::vector<int64_t> tbase(n_samples);
  std::vector<int32_t> g_sample(shs.size());
  std::vector<double> coef_a, coef_b;
  for (int s = 0; s < n_samples; ++s) {
    const int nh = shs_start[s + 1] - shs_start[s], n = nbins[s];
    tbase[s] = (int64_t)coef_a.size();
    for (int g = shs_start[s]; g < shs_start[s + 1]; ++g) g_sample[g] = s;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < nh; ++j) {
        const int h = shs[shs_start[s] + j];
        coef_a.push_back(coef[hs_ofs[h] + i]);
        coef_b.push_back(coef[hs_ofs[h] + n + i]);
      }
  }
  std::vector<int32_t> bin_start(n_bins + 1, 0);
  for (int s = 0; s < n_samples; ++s)
    for (int i = 0; i < nbins[s]; ++i) bin_start[bin0[s] + i + 1]++;
  for (int b = 0; b < n_bins; ++b) bin_start[b + 1] += bin_start[b];
  std::vector<int32_t> bin_entry(bin_start[n_bins]);
  std::vector<int32_t> bfill(bin_start.begin(), bin_start.end() - 1);
  for (int s = 0; s < n_samples; ++s)
    for (int i = 0; i < nbins[s]; ++i) bin_entry[bfill[bin0[s] + i]++] = eofs[s] + i;

  rf_binned* m = new (std::nothrow) rf_binned();
  if (!m) return RF_E_OOM;
  m->n_bins = n_bins;
  m->n_samples = n_samples;
  m->n_params = n_params;
  m->n_mods = n_mods;
  m->n_entries = (int32_t)total;
  m->n_hs = n_hs;
  const std::vector<int32_t> vb0(bin0, bin0 + n_samples), vnb(nbins, nbins + n_samples);
  const std::vector<double> vnom(nominal, nominal + total);
  std::vector<int32_t> vcon(n_params);
  for (int k = 0; k < n_params; ++k) vcon[k] = constrained[k] ? 1 : 0;
  std::vector<int32_t> shs_k(shs.size());
  std::vector<int64_t> shs_ofs(shs.size());
  for (size_t j = 0; j < shs.size(); ++j) {
    shs_k[j] = hs_param[shs[j]];
    shs_ofs[j] = hs_ofs[shs[j]];
  }
  // float-pair copies: hi = the float nearest v, lo = the float nearest v - hi
  auto pairs = [](const std::vector<double>& v) {
    std::vector<float2> f(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float h = (float)v[i];
      f[i] = make_float2(h, (float)(v[i] - (double)h));
    }
    return f;
  };
  const bool ok = upload(m->shs_k, shs_k) && upload(m->shs_ofs, shs_ofs) &&
                  upload(m->nominal_f, pairs(vnom)) && upload(m->coef_f, pairs(coef)) &&
                  upload(m->coef_af, pairs(coef_a)) && upload(m->coef_bf, pairs(coef_b)) &&
                  upload(m->bin0, vb0) && upload(m->nb, vnb) && upload(m->eofs, eofs) && upload(m->esample, esample) &&
                  upload(m->nominal, vnom) && upload(m->smod_start, smod_start) && upload(m->smod, smod) &&
                  upload(m->shs_start, shs_start) && upload(m->shs, shs) && upload(m->kind, kind) &&
                  upload(m->param, param) && upload(m->msample, msample) && upload(m->mhs, mhs) &&
                  upload(m->ns_a, ns_a) && upload(m->ns_b, ns_b) && upload(m->hs_param, hs_param) &&
                  upload(m->hs_sample, hs_sample) && upload(m->hs_ofs, hs_ofs) && upload(m->coef, coef) &&
                  upload(m->tbase, tbase) && upload(m->g_sample, g_sample) && upload(m->coef_a, coef_a) &&
                  upload(m->coef_b, coef_b) &&
                  upload(m->bin_start, bin_start) && upload(m->bin_entry, bin_entry) &&
                  upload(m->pmod_start, pmod_start) && upload(m->pmod, pmod) && upload(m->constrained, vcon);
  m->smem = binned_smem(n_params, n_samples, n_bins);
  int dev_id = 0, max_optin = 0;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev_id);
  if (m->smem > (size_t)max_optin ||
      !cuda_ok(cudaFuncSetAttribute(binned_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m->smem),
               "binned smem") ||
      !cuda_ok(cudaFuncSetAttribute(binned_expected_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)m->smem),
               "binned smem")) {
    delete m;
    set_error("rf_binned_create: the model needs more shared memory than a block has");
    return RF_E_INVALID;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, binned_kernel, kBinnedThreads, m->smem);
  m->grid = sm_count() * std::max(1, per_sm);
  if (!ok || !m->scratch.ensure(sizeof(double) * (size_t)m->grid * (size_t)(m->n_entries + std::max(1, n_hs)))) {
    delete m;
    return RF_E_OOM;
  }
  BinnedDev& D = m->dev;
  D.n_bins = n_bins;
  D.n_samples = n_samples;
  D.n_params = n_params;
  D.n_mods = n_mods;
  D.n_entries = m->n_entries;
  D.n_hs = n_hs;
  D.bin0 = (const int32_t*)m->bin0.p;
  D.nb = (const int32_t*)m->nb.p;
  D.eofs = (const int32_t*)m->eofs.p;
  D.esample = (const int32_t*)m->esample.p;
  D.nominal = (const double*)m->nominal.p;
  D.smod_start = (const int32_t*)m->smod_start.p;
  D.smod = (const int32_t*)m->smod.p;
  D.shs_start = (const int32_t*)m->shs_start.p;
  D.shs = (const int32_t*)m->shs.p;
  D.kind = (const int32_t*)m->kind.p;
  D.param = (const int32_t*)m->param.p;
  D.msample = (const int32_t*)m->msample.p;
  D.mhs = (const int32_t*)m->mhs.p;
  D.ns_a = (const double*)m->ns_a.p;
  D.ns_b = (const double*)m->ns_b.p;
  D.hs_param = (const int32_t*)m->hs_param.p;
  D.hs_sample = (const int32_t*)m->hs_sample.p;
  D.hs_ofs = (const int64_t*)m->hs_ofs.p;
  D.coef = (const double*)m->coef.p;
  D.tbase = (const int64_t*)m->tbase.p;
  D.g_sample = (const int32_t*)m->g_sample.p;
  D.coef_a = (const double*)m->coef_a.p;
  D.coef_b = (const double*)m->coef_b.p;
  D.nominal_f = (const float2*)m->nominal_f.p;
  D.shs_k = (const int32_t*)m->shs_k.p;
  D.shs_ofs = (const int64_t*)m->shs_ofs.p;
  D.coef_f = (const float2*)m->coef_f.p;
  D.coef_af = (const float2*)m->coef_af.p;
  D.coef_bf = (const float2*)m->coef_bf.p;
  D.bin_start = (const int32_t*)m->bin_start.p;
  D.bin_entry = (const int32_t*)m->bin_entry.p;
  D.pmod_start = (const int32_t*)m->pmod_start.p;
  D.pmod = (const int32_t*)m->pmod.p;
  D.constrained = (const int32_t*)m->constrained.p;
  *out = m;
  return RF_OK;
}

void rf_binned_destroy(rf_binned* m) { delete m; }

int32_t rf_binned_n_params(const rf_binned* m) { return m ? m->n_params : 0; }

rf_status rf_binned_nll_grad_async(rf_binned* m, int32_t n_sets, const double* d_counts, const double* d_theta,
                                   double* d_out, int32_t* d_flags, void* stream) {
  if (!m || n_sets < 0 || (n_sets > 0 && (!d_counts || !d_theta || !d_out || !d_flags))) {
    set_error("rf_binned_nll_grad_async: bad argument");
    return RF_E_INVALID;
  }
  return launch_binned(m, n_sets, d_counts, d_theta, d_out, d_flags, (cudaStream_t)stream);
}

rf_status rf_binned_nll_grad(rf_binned* m, int32_t n_sets, const double* counts, const double* theta, double* nll,
                             double* grad) {
  if (!m || n_sets < 0 || (n_sets > 0 && (!counts || !theta || !nll || !grad))) {
    set_error("rf_binned_nll_grad: bad argument");
    return RF_E_INVALID;
  }
  if (n_sets == 0) return RF_OK;
  const int P = m->n_params, B = m->n_bins;
  if (!m->counts.ensure(sizeof(double) * (size_t)n_sets * B) ||
      !m->theta.ensure(sizeof(double) * (size_t)n_sets * std::max(P, 1)) ||
      !m->out.ensure(sizeof(double) * (size_t)n_sets * (1 + P)) || !m->flags.ensure(sizeof(int32_t) * n_sets) ||
      !m->h_out.ensure(sizeof(double) * (size_t)n_sets * (1 + P)) || !m->h_flags.ensure(sizeof(int32_t) * n_sets))
    return RF_E_OOM;
  if (!cuda_ok(cudaMemcpy(m->counts.p, counts, sizeof(double) * (size_t)n_sets * B, cudaMemcpyHostToDevice), "binned") ||
      (P > 0 && !cuda_ok(cudaMemcpy(m->theta.p, theta, sizeof(double) * (size_t)n_sets * P, cudaMemcpyHostToDevice),
                         "binned")))
    return RF_E_CUDA;
  rf_status s = launch_binned(m, n_sets, (const double*)m->counts.p, (const double*)m->theta.p, (double*)m->out.p,
                              (int32_t*)m->flags.p, nullptr);
  if (s != RF_OK) return s;
  if (!cuda_ok(cudaMemcpy(m->h_out.p, m->out.p, sizeof(double) * (size_t)n_sets * (1 + P), cudaMemcpyDeviceToHost),
               "binned") ||
      !cuda_ok(cudaMemcpy(m->h_flags.p, m->flags.p, sizeof(int32_t) * n_sets, cudaMemcpyDeviceToHost), "binned"))
    return RF_E_CUDA;
  const double* o = (const double*)m->h_out.p;
  const int32_t* f = (const int32_t*)m->h_flags.p;
  rf_status st = RF_OK;
  for (int t = 0; t < n_sets; ++t) {
    nll[t] = o[(size_t)t * (1 + P)];
    for (int k = 0; k < P; ++k) grad[(size_t)t * P + k] = o[(size_t)t * (1 + P) + 1 + k];
    if (f[t]) st = RF_E_DOMAIN;
  }
  if (st == RF_E_DOMAIN) set_error("expected count <= 0 in some bin");
  return st;
}

rf_status rf_binned_expected(rf_binned* m, int32_t n_sets, const double* d_theta, double* d_nu, void* stream) {
  if (!m || n_sets < 0 || (n_sets > 0 && (!d_theta || !d_nu))) {
    set_error("rf_binned_expected: bad argument");
    return RF_E_INVALID;
  }
  if (n_sets == 0) return RF_OK;
  note_launches(1, (cudaStream_t)stream);
  binned_expected_kernel<<<std::min(n_sets, m->grid), kBinnedThreads, m->smem, (cudaStream_t)stream>>>(
      m->dev, n_sets, d_theta, d_nu, (double*)m->scratch.p);
  return cuda_ok(cudaGetLastError(), "binned launch") ? RF_OK : RF_E_CUDA;
}

rf_status rf_binned_fit(rf_binned* m, int32_t n_sets, const double* counts, const double* theta0, const double* lo,
                        const double* hi, const rf_fit_opts* opts, double* theta_hat, double* nll_min, double* cov,
                        int32_t* n_evals, int32_t* fit_status) {
  if (!m || n_sets < 0 || (n_sets > 0 && (!counts || !theta0 || !lo || !hi || !theta_hat || !nll_min || !n_evals ||
                                          !fit_status))) {
    set_error("rf_binned_fit: bad argument");
    return RF_E_INVALID;
  }
  if (n_sets == 0) return RF_OK;
  const int P = m->n_params, B = m->n_bins, S = n_sets;
  const double tol = (opts && opts->tol_edm > 0.0) ? opts->tol_edm : 1e-7;
  const int max_evals = (opts && opts->max_evals > 0) ? opts->max_evals : 1000;
  const bool want_cov = opts && opts->want_cov && cov;
  if (!m->counts.ensure(sizeof(double) * (size_t)S * B) || !m->theta.ensure(sizeof(double) * (size_t)S * std::max(P, 1)) ||
      !m->out.ensure(sizeof(double) * (size_t)S * (1 + P)) || !m->flags.ensure(sizeof(int32_t) * S) ||
      !m->sets.ensure(sizeof(int32_t) * S) || !m->h_out.ensure(sizeof(double) * (size_t)S * (1 + P)) ||
      !m->h_theta.ensure(sizeof(double) * (size_t)S * std::max(P, 1)) || !m->h_sets.ensure(sizeof(int32_t) * S))
    return RF_E_OOM;
  if (!cuda_ok(cudaMemcpy(m->counts.p, counts, sizeof(double) * (size_t)S * B, cudaMemcpyHostToDevice), "binned fit"))
    return RF_E_CUDA;
  cudaStream_t st = nullptr;
  // One round: the active sets' points packed, one launch, results scattered.
  auto eval = [&](const std::vector<int32_t>& active, std::vector<double>& th, std::vector<double>& nll,
                  std::vector<double>& grad) -> rf_status {
    const int n = (int)active.size();
    double* ht = (double*)m->h_theta.p;
    int32_t* hs = (int32_t*)m->h_sets.p;
    for (int a = 0; a < n; ++a) {
      hs[a] = active[a];
      std::memcpy(ht + (size_t)a * P, &th[(size_t)active[a] * P], sizeof(double) * P);
    }
    if (!cuda_ok(cudaMemcpyAsync(m->theta.p, ht, sizeof(double) * (size_t)n * P, cudaMemcpyHostToDevice, st),
                 "binned fit") ||
        !cuda_ok(cudaMemcpyAsync(m->sets.p, hs, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st), "binned fit"))
      return RF_E_CUDA;
    const rf_status r = launch_binned(m, n, (const double*)m->counts.p, (const double*)m->theta.p, (double*)m->out.p,
                                      (int32_t*)m->flags.p, st, (const int32_t*)m->sets.p);
    if (r != RF_OK) return r;
    if (!cuda_ok(cudaMemcpyAsync(m->h_out.p, m->out.p, sizeof(double) * (size_t)n * (1 + P), cudaMemcpyDeviceToHost,
                                 st),
                 "binned fit") ||
        !cuda_ok(cudaStreamSynchronize(st), "binned fit"))
      return RF_E_CUDA;
    const double* o = (const double*)m->h_out.p;
    for (int a = 0; a < n; ++a) {
      const int s = active[a];
      nll[s] = o[(size_t)a * (1 + P)];
      for (int k = 0; k < P; ++k) grad[(size_t)s * P + k] = o[(size_t)a * (1 + P) + 1 + k];
    }
    return RF_OK;
  };
  return fit_batch(S, P, lo, hi, theta0, tol, max_evals, want_cov, eval, nullptr, theta_hat, nll_min,
                   want_cov ? cov : nullptr, n_evals, fit_status);
}

}  // extern "C"
