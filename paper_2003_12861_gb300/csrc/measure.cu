// Measurement support: kernel timing with CUDA events on the launching
// stream, the slow-path event count, host-column refills, and the roofline
// probes (FP64/FP32 FMA rate, the per-event transcendental set, streaming
// read bandwidth).
#include <cuda_runtime.h>

#include <cstring>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "api_internal.h"
#include "ff.cuh"
#include "nll_kernels.cuh"

namespace rf {

namespace {

std::mutex g_tmu;
bool g_timing = false;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_pairs;
cudaEvent_t g_open = nullptr;

cudaEvent_t new_event() {
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// ----------------------------------------------------------------- probes

__global__ void probe_dfma(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void probe_ffma(double* out, int iters, float a, float b) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
        x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)(x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7);
}

// Float-float multiply-adds (ff_fma: a b + c on float pairs), eight
// independent chains per thread.
__global__ void probe_fffma(double* out, int iters, float a, float b) {
  const ff A = {a, a * 1e-9f}, B = {b, b * 1e-9f};
  ff x[8];
  for (int j = 0; j < 8; ++j) x[j] = {threadIdx.x * 1e-3f + j, 0.0f};
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = ff_fma(x[j], A, B);
  double sum = 0.0;
  for (int j = 0; j < 8; ++j) sum += ff_to_double(x[j]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

// Per "event": the requested numbers of exp, erfc, log and reciprocal calls on
// arguments that change every event (so nothing is hoisted), summed.
__global__ void probe_trans(double* out, int events, int n_exp, int n_erfc, int n_log, int n_rcp) {
  double acc = 0.0;
  double x = 0.5 + (blockIdx.x * blockDim.x + threadIdx.x) * 1e-9;
  for (int i = 0; i < events; ++i) {
    for (int k = 0; k < n_exp; ++k) acc += exp(-x * (1.0 + 0.25 * k));
    for (int k = 0; k < n_erfc; ++k) acc += erfc(x * (1.0 + 0.25 * k) - 0.3);
    for (int k = 0; k < n_log; ++k) acc += log(x + (double)k);
    for (int k = 0; k < n_rcp; ++k) acc += 1.0 / (x + (double)k);
    x += 1e-6;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// The same per-event set with the library's float-float implementations.
__global__ void probe_trans_ff(double* out, int events, int n_exp, int n_erfc, int n_log, int n_rcp) {
  __shared__ FFTables T;
  ff_load_tables(T);
  __syncthreads();
  ff acc = {0.f, 0.f};
  bool ok = true;
  ff x = ff_from_double(0.5 + (blockIdx.x * blockDim.x + threadIdx.x) * 1e-9);
  const ff step = {1e-6f, 0.f};
  for (int i = 0; i < events; ++i) {
    for (int k = 0; k < n_exp; ++k) ff_acc(acc, ff_exp_in_range(T, ff_mul_f(x, -(1.0f + 0.25f * k))));
    for (int k = 0; k < n_erfc; ++k) ff_acc(acc, ff_erfcx(T, ff_add_f(ff_mul_f(x, 1.0f + 0.25f * k), 0.3f), ok));
    for (int k = 0; k < n_log; ++k) ff_acc(acc, ff_log(T, ff_add_f(x, (float)k), ok));
    for (int k = 0; k < n_rcp; ++k) ff_acc(acc, ff_rcp_u(ff_add_f(x, (float)k)));
    x = ff_add(x, step);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = ok ? ff_to_double(acc) : -1.0;
}

// Elementwise evaluation of the library's float-float functions (fn 0-3) and
// of CUDA's FP64 functions (fn 10-13), for validation.
__global__ void math_eval_kernel(int fn, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  __shared__ FFTables T;
  ff_load_tables(T);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double xv = x[i];
    bool ok = true;
    ff r = {0.f, 0.f};
    double out = 0.0;
    switch (fn) {
      case 0: r = ff_exp(T, ff_from_double(xv), ok); out = ff_to_double(r); break;
      case 1: r = ff_log(T, ff_from_double(xv), ok); out = ff_to_double(r); break;
      case 2: r = ff_rcp(ff_from_double(xv)); out = ff_to_double(r); break;
      case 3: r = ff_erfcx(T, ff_from_double(xv), ok); out = ff_to_double(r); break;
      case 10: out = exp(xv); break;
      case 11: out = log(xv); break;
      case 12: out = 1.0 / xv; break;
      case 13: out = erfcx(xv); break;
      default: ok = false;
    }
    y[i] = ok ? out : __longlong_as_double(0x7ff8000000000000ll);
  }
}

__global__ void probe_read(const double2* __restrict__ p, size_t n, double* out) {
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = __ldcs(p + i);
    s += v.x + v.y;
  }
  if (s == 1.2345e-300) out[0] = s;  // keeps the loads alive
}

}  // namespace

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

void timing_begin(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (!g_timing || capturing(st)) return;
  g_open = new_event();
  if (g_open) cudaEventRecord(g_open, st);
}

void timing_end(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (!g_timing || !g_open || capturing(st)) return;
  cudaEvent_t e = new_event();
  if (!e) return;
  cudaEventRecord(e, st);
  g_pairs.emplace_back(g_open, e);
  g_open = nullptr;
}

}  // namespace rf

using namespace rf;

extern "C" {

rf_status rf_kernel_timing(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_timing = enable != 0;
  return RF_OK;
}

rf_status rf_kernel_time(double* total_ms, int64_t* launches, int32_t reset) {
  if (!total_ms || !launches) {
    set_error("rf_kernel_time: NULL output");
    return RF_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_tmu);
  double sum = 0.0;
  for (auto& pr : g_pairs) {
    if (!cuda_ok(cudaEventSynchronize(pr.second), "rf_kernel_time")) return RF_E_CUDA;
    float ms = 0.f;
    if (!cuda_ok(cudaEventElapsedTime(&ms, pr.first, pr.second), "rf_kernel_time")) return RF_E_CUDA;
    sum += ms;
  }
  *total_ms = sum;
  *launches = (int64_t)g_pairs.size();
  if (reset) {
    for (auto& pr : g_pairs) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    g_pairs.clear();
  }
  return RF_OK;
}

rf_status rf_slow_events(const rf_data* d, int64_t* count) {
  if (!d || !count) {
    set_error("rf_slow_events: bad argument");
    return RF_E_INVALID;
  }
  unsigned long long v = 0;
  if (d->ws.slow.p && !cuda_ok(cudaMemcpy(&v, d->ws.slow.p, sizeof v, cudaMemcpyDeviceToHost), "rf_slow_events"))
    return RF_E_CUDA;
  *count = (int64_t)v;
  return RF_OK;
}

rf_status rf_data_refill(rf_data* d, const void* const* cols, void* stream) {
  if (!d || !cols || !d->owns_cols) {
    set_error("rf_data_refill: bad argument or a dataset with borrowed columns");
    return RF_E_INVALID;
  }
  for (int c = 0; c < d->n_obs; ++c) {
    const size_t bytes = (size_t)d->n_events * (d->dtype[c] == RF_F32 ? 4 : 8);
    if (bytes && !cuda_ok(cudaMemcpyAsync(d->cols[c], cols[c], bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream),
                          "rf_data_refill"))
      return RF_E_CUDA;
  }
  return RF_OK;
}

rf_status rf_probe(int32_t kind, int32_t n_exp, int32_t n_erfc, int32_t n_log, int32_t n_rcp, double* rate) {
  if (!rate || kind < 0 || kind > 6 || n_exp < 0 || n_erfc < 0 || n_log < 0 || n_rcp < 0) {
    set_error("rf_probe: bad argument");
    return RF_E_INVALID;
  }
  const int nsm = sm_count();
  const int threads = 256, blocks = nsm * 8;
  DevBuf out;
  if (!out.ensure(sizeof(double) * threads * blocks)) return RF_E_OOM;
  cudaEvent_t e0 = new_event(), e1 = new_event();
  if (!e0 || !e1) return RF_E_CUDA;
  DevBuf buf;
  HostBuf hbuf;
  const double2* src = nullptr;
  size_t n2 = 0;
  if (kind == 3) {
    n2 = (size_t)1 << 27;  // 2 GiB of double2
    if (!buf.ensure(n2 * sizeof(double2))) return RF_E_OOM;
    if (!cuda_ok(cudaMemset(buf.p, 0, n2 * sizeof(double2)), "probe memset")) return RF_E_CUDA;
    src = (const double2*)buf.p;
  } else if (kind == 5) {
    n2 = (size_t)1 << 25;  // 512 MiB of pinned host memory, read in place by the SMs
    if (!hbuf.ensure(n2 * sizeof(double2))) return RF_E_OOM;
    std::memset(hbuf.p, 0, n2 * sizeof(double2));
    void* dp = nullptr;
    if (!cuda_ok(cudaHostGetDevicePointer(&dp, hbuf.p, 0), "probe host pointer")) return RF_E_CUDA;
    src = (const double2*)dp;
  }
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    double work = 0.0;
    if (kind == 0) {
      const int it = 2048;
      probe_dfma<<<blocks, threads>>>((double*)out.p, it, 0.999999, 1e-7);
      work = 2.0 * 8 * it * (double)threads * blocks;
    } else if (kind == 1) {
      const int it = 32768;
      probe_ffma<<<blocks, threads>>>((double*)out.p, it, 0.999999f, 1e-7f);
      work = 2.0 * 8 * it * (double)threads * blocks;
    } else if (kind == 2) {
      const int ev = 128;
      probe_trans<<<blocks, threads>>>((double*)out.p, ev, n_exp, n_erfc, n_log, n_rcp);
      work = (double)ev * threads * blocks;
    } else if (kind == 4) {
      const int ev = 512;
      probe_trans_ff<<<blocks, threads>>>((double*)out.p, ev, n_exp, n_erfc, n_log, n_rcp);
      work = (double)ev * threads * blocks;
    } else if (kind == 6) {
      const int it = 2048;
      probe_fffma<<<blocks, threads>>>((double*)out.p, it, 0.999999f, 1e-7f);
      work = 8.0 * it * (double)threads * blocks;  // multiply-adds
    } else {
      probe_read<<<nsm * 4, 512>>>(src, n2, (double*)out.p);
      work = (double)n2 * sizeof(double2);
    }
    cudaEventRecord(e1);
    if (!cuda_ok(cudaEventSynchronize(e1), "probe")) return RF_E_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::max(best, work / (ms * 1e-3));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!cuda_ok(cudaGetLastError(), "probe")) return RF_E_CUDA;
  *rate = best;
  return RF_OK;
}

rf_status rf_math_eval(int32_t fn, const double* d_x, double* d_y, int64_t n, void* stream) {
  if (!d_x || !d_y || n < 0 || !((fn >= 0 && fn <= 3) || (fn >= 10 && fn <= 13))) {
    set_error("rf_math_eval: bad argument");
    return RF_E_INVALID;
  }
  if (n == 0) return RF_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  math_eval_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(fn, d_x, d_y, n);
  return cuda_ok(cudaGetLastError(), "rf_math_eval") ? RF_OK : RF_E_CUDA;
}

}  // extern "C"
