// Binned (HistFactory-style) likelihood: NLL and gradient of many datasets
// of bin counts at once (paper Sec. 3: models built from histograms --
// channels of samples with +-1 sigma systematic variations).
//
// nu_s[i] = prod(normfactors) prod(normsys eta) (h_s[i] + sum histosys
// delta), eta = k_hi^alpha (alpha >= 0) or k_lo^-alpha, delta = alpha (h_hi
// - h) or alpha (h - h_lo); nu_b = sum over the samples on bin b; NLL =
// sum_b (nu_b - n_b log nu_b) + sum over constrained parameters theta^2/2.
// d NLL / d theta_k = sum_b w_b d nu_b / d theta_k + [constrained] theta_k,
// w_b = 1 - n_b / nu_b; per modifier of parameter k: a normfactor or normsys
// on sample s contributes dlog(factor)/dtheta_k sum_i w nu_s[i], a histosys
// contributes F_s sum_i w slope[i].
//
// One block per dataset (persistent over datasets), FP64 throughout, every
// sum in a fixed order (each thread's bins / samples / modifiers in index
// order, a fixed tree across threads), so results do not depend on the
// launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"

namespace rf {

namespace {

constexpr int kBinnedThreads = 256;
constexpr int kMaxBinnedBins = 8192, kMaxBinnedSamples = 2048;

// Dynamic shared memory of the kernels: theta, F and Ssum per sample, W per
// bin, one partial sum per thread, then the parameters' signs.
size_t binned_smem(int n_params, int n_samples, int n_bins) {
  return sizeof(double) * ((size_t)n_params + 2 * (size_t)n_samples + (size_t)n_bins + kBinnedThreads) +
         sizeof(int) * (size_t)n_params;
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
  const double* lk_lo;        // normsys: log k_lo, log k_hi
  const double* lk_hi;
  const int32_t* hs_param;    // per histosys: parameter, sample
  const int32_t* hs_sample;
  const int64_t* hs_ofs;      // per histosys: its slopes (h - h_lo) then (h_hi - h), nb each, in `slope`
  const double* slope;
  // The same slopes transposed per sample for the weighted sums: sample s's
  // histosys j (its j-th in shs order) at local bin i sits at
  // tbase[s] + i * (histosys of s) + j, in slope_dn (h - h_lo) and slope_up.
  const int64_t* tbase;
  const int32_t* g_sample;    // per position in shs: its sample
  const double* slope_dn;
  const double* slope_up;
  const int32_t* bin_start;   // per bin: its entries (CSR, sample order)
  const int32_t* bin_entry;
  const int32_t* pmod_start;  // per parameter: its modifiers (CSR, modifier order)
  const int32_t* pmod;
  const int32_t* constrained;
};

// The slopes of histosys h for a parameter value of sign `up` (1: alpha >=
// 0, the h_hi side).  The sign is decided once per parameter and dataset as
// an integer: an FP64 comparison per term would occupy the FP64 unit as
// long as the multiply-add itself.
__device__ __forceinline__ const double* hs_slopes(const BinnedDev& m, int h, int n, int up) {
  return m.slope + m.hs_ofs[h] + (up ? n : 0);
}

// theta and its signs into smem, then the sample factors F (normfactors and
// normsys).
__device__ __forceinline__ void sample_factors(const BinnedDev& m, const double* th_g, double* th, int* up,
                                               double* F) {
  for (int k = threadIdx.x; k < m.n_params; k += kBinnedThreads) {
    const double a = th_g[k];
    th[k] = a;
    up[k] = a >= 0.0;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < m.n_samples; s += kBinnedThreads) {
    double f = 1.0;
    for (int j = m.smod_start[s]; j < m.smod_start[s + 1]; ++j) {
      const int md = m.smod[j];
      const double a = th[m.param[md]];
      if (m.kind[md] == MOD_NORMFACTOR) f *= a;
      else f *= a >= 0.0 ? exp(a * m.lk_hi[md]) : exp(-a * m.lk_lo[md]);
    }
    F[s] = f;
  }
  __syncthreads();
}

// nu of every (sample, bin) entry: consecutive threads take consecutive
// bins of a sample, so its histosys slopes are read coalesced.
__device__ __forceinline__ void entry_rates(const BinnedDev& m, const double* th, const int* up, const double* F,
                                            double* nu_e) {
  for (int e = threadIdx.x; e < m.n_entries; e += kBinnedThreads) {
    const int s = m.esample[e], i = e - m.eofs[s], n = m.nb[s];
    double shape = m.nominal[e];
    for (int j = m.shs_start[s]; j < m.shs_start[s + 1]; ++j) {
      const int h = m.shs[j], k = m.hs_param[h];
      shape = fma(th[k], hs_slopes(m, h, n, up[k])[i], shape);
    }
    nu_e[e] = F[s] * shape;
  }
}

// out[set]: NLL then gradient (1 + n_params); flags[set]: 1 if some bin has
// nu <= 0 (NLL +inf).  scratch: per block n_entries (entry rates) +
// n_hs (histosys sums) doubles.
__global__ void __launch_bounds__(kBinnedThreads) binned_kernel(const BinnedDev m, int n_sets, const double* counts,
                                                                 const double* theta, double* out, int32_t* flags,
                                                                 double* scratch) {
  extern __shared__ double smem[];
  double* th = smem;
  double* F = th + m.n_params;
  double* Ssum = F + m.n_samples;
  double* W = Ssum + m.n_samples;
  double* part = W + m.n_bins;
  int* up = (int*)(part + kBinnedThreads);
  __shared__ int bad;
  const int tid = threadIdx.x;
  double* nu_e = scratch + (size_t)blockIdx.x * (m.n_entries + m.n_hs);
  double* T = nu_e + m.n_entries;
  for (int set = blockIdx.x; set < n_sets; set += gridDim.x) {
    const double* n = counts + (size_t)set * m.n_bins;
    if (tid == 0) bad = 0;
    sample_factors(m, theta + (size_t)set * m.n_params, th, up, F);
    entry_rates(m, th, up, F, nu_e);
    __syncthreads();
    // bins: expected count, weight 1 - n/nu, the Poisson term
    double acc = 0.0;
    for (int b = tid; b < m.n_bins; b += kBinnedThreads) {
      double nu = 0.0;
      for (int j = m.bin_start[b]; j < m.bin_start[b + 1]; ++j) nu += nu_e[m.bin_entry[j]];
      if (!(nu > 0.0) || !isfinite(nu)) {
        bad = 1;
        W[b] = 0.0;
        continue;
      }
      W[b] = 1.0 - n[b] / nu;
      acc += nu - (n[b] != 0.0 ? n[b] * log(nu) : 0.0);
    }
    part[tid] = acc;
    __syncthreads();
    // per sample sum_i w nu_s[i] (a thread each); per histosys sum_i w
    // slope[i] (a warp each: lanes over bins, then a butterfly)
    for (int s = tid; s < m.n_samples; s += kBinnedThreads) {
      double a = 0.0;
      for (int i = 0; i < m.nb[s]; ++i) a += W[m.bin0[s] + i] * nu_e[m.eofs[s] + i];
      Ssum[s] = a;
    }
    // (a thread each, bins in order; consecutive threads read consecutive
    // slopes of the transposed layout)
    for (int g = tid; g < m.n_hs; g += kBinnedThreads) {
      const int s = m.g_sample[g], h = m.shs[g];
      const int nh = m.shs_start[s + 1] - m.shs_start[s], j = g - m.shs_start[s];
      const double* sl = (up[m.hs_param[h]] ? m.slope_up : m.slope_dn) + m.tbase[s] + j;
      const double* w = W + m.bin0[s];
      double a = 0.0;
      for (int i = 0; i < m.nb[s]; ++i) a = fma(w[i], sl[(size_t)i * nh], a);
      T[h] = a;
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
        else if (m.kind[md] == MOD_NORMSYS) g += Ssum[s] * (up[k] ? m.lk_hi[md] : -m.lk_lo[md]);
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
  int* up = (int*)(F + m.n_samples);
  double* nu_e = scratch + (size_t)blockIdx.x * (m.n_entries + m.n_hs);
  for (int set = blockIdx.x; set < n_sets; set += gridDim.x) {
    sample_factors(m, theta + (size_t)set * m.n_params, th, up, F);
    entry_rates(m, th, up, F, nu_e);
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
  rf::DevBuf bin0, nb, eofs, esample, nominal, smod_start, smod, shs_start, shs, kind, param, msample, mhs, lk_lo,
      lk_hi, hs_param, hs_sample, hs_ofs, slope, tbase, g_sample, slope_dn, slope_up, bin_start, bin_entry, pmod_start,
      pmod, constrained;
  rf::DevBuf scratch, counts, theta, out, flags;
  rf::HostBuf h_out, h_flags;
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
                        int32_t* d_flags, cudaStream_t st) {
  if (n_sets == 0) return RF_OK;
  const int grid = std::min(n_sets, m->grid);
  binned_kernel<<<grid, kBinnedThreads, m->smem, st>>>(m->dev, n_sets, d_counts, d_theta, d_out, d_flags,
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
  std::vector<double> lk_lo(n_mods, 0.0), lk_hi(n_mods, 0.0);
  std::vector<int32_t> hs_param, hs_sample;
  std::vector<int64_t> hs_ofs;
  std::vector<double> slope;
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
      lk_lo[j] = std::log(md.k_lo);
      lk_hi[j] = std::log(md.k_hi);
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
      hs_ofs.push_back((int64_t)slope.size());
      for (int i = 0; i < n; ++i) slope.push_back(h[i] - lo[i]);  // alpha < 0
      for (int i = 0; i < n; ++i) slope.push_back(hi[i] - h[i]);  // alpha >= 0
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
  // transposed slopes per sample
  std::vector<int64_t> tbase(n_samples);
  std::vector<int32_t> g_sample(shs.size());
  std::vector<double> slope_dn, slope_up;
  for (int s = 0; s < n_samples; ++s) {
    const int nh = shs_start[s + 1] - shs_start[s], n = nbins[s];
    tbase[s] = (int64_t)slope_dn.size();
    for (int g = shs_start[s]; g < shs_start[s + 1]; ++g) g_sample[g] = s;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < nh; ++j) {
        const int h = shs[shs_start[s] + j];
        slope_dn.push_back(slope[hs_ofs[h] + i]);
        slope_up.push_back(slope[hs_ofs[h] + n + i]);
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
  const bool ok = upload(m->bin0, vb0) && upload(m->nb, vnb) && upload(m->eofs, eofs) && upload(m->esample, esample) &&
                  upload(m->nominal, vnom) && upload(m->smod_start, smod_start) && upload(m->smod, smod) &&
                  upload(m->shs_start, shs_start) && upload(m->shs, shs) && upload(m->kind, kind) &&
                  upload(m->param, param) && upload(m->msample, msample) && upload(m->mhs, mhs) &&
                  upload(m->lk_lo, lk_lo) && upload(m->lk_hi, lk_hi) && upload(m->hs_param, hs_param) &&
                  upload(m->hs_sample, hs_sample) && upload(m->hs_ofs, hs_ofs) && upload(m->slope, slope) &&
                  upload(m->tbase, tbase) && upload(m->g_sample, g_sample) && upload(m->slope_dn, slope_dn) &&
                  upload(m->slope_up, slope_up) &&
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
  D.lk_lo = (const double*)m->lk_lo.p;
  D.lk_hi = (const double*)m->lk_hi.p;
  D.hs_param = (const int32_t*)m->hs_param.p;
  D.hs_sample = (const int32_t*)m->hs_sample.p;
  D.hs_ofs = (const int64_t*)m->hs_ofs.p;
  D.slope = (const double*)m->slope.p;
  D.tbase = (const int64_t*)m->tbase.p;
  D.g_sample = (const int32_t*)m->g_sample.p;
  D.slope_dn = (const double*)m->slope_dn.p;
  D.slope_up = (const double*)m->slope_up.p;
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
  binned_expected_kernel<<<std::min(n_sets, m->grid), kBinnedThreads, m->smem, (cudaStream_t)stream>>>(
      m->dev, n_sets, d_theta, d_nu, (double*)m->scratch.p);
  return cuda_ok(cudaGetLastError(), "binned launch") ? RF_OK : RF_E_CUDA;
}

}  // extern "C"
