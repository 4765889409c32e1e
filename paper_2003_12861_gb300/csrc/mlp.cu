// Learned fit start: a multilayer perceptron from the 64-bin histogram of a
// toy dataset to a starting point for its fit (the paper has no learned part;
// this is the learned-start configuration: 64 -> 128 -> 128 -> 128 -> 6 with
// GELU, BF16 operands, FP32 accumulation, trained on the GPU).
//
// Kernels: a tensor-core GEMM on the fifth-generation tensor cores (tcgen05:
// BF16 x BF16 -> FP32 accumulated in tensor memory; the operands are rounded
// to BF16, nearest even, as they are staged into shared memory) with a fused
// bias / GELU / pre-activation epilogue, used for the forward pass and both
// backward products; GELU backward; bias gradients
// (column sums in fixed order); MSE loss and its gradient; Adam (Kingma & Ba
// 2015) on FP32 master weights; a row gather for shuffled mini-batches; and
// target standardisation.  Every reduction has a fixed order, so training is
// bitwise reproducible.
//
// Parameter layout (flat FP32): for each layer W[n_in x n_out] row-major,
// then b[n_out].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "api_internal.h"

namespace rf {

// Learned starts of bounded parameters stay this fraction of the range
// inside the bounds (rf_mlp_predict).
constexpr double kStartMargin = 0.05;

namespace {

struct GemmArgs {
  const float* A;  // M x K (or K x M when transA)
  const float* B;  // K x N (or N x K when transB)
  float* C;        // M x N
  const float* bias;  // N or null
  float* Z;        // pre-activation out (M x N) or null
  int M, N, K, lda, ldb, ldc;
  int transA, transB, gelu;
  // split K: block z takes K rows [z kc, (z + 1) kc) and writes its raw
  // partial tile to part + z M N (row-major) instead of the epilogue; null
  // for one block over all of K
  float* part;
  int kc;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * __expf(-0.5f * z * z) * 0.3989422804014327f;
}

// Set when a GEMM's wait for its tensor-core work gave up (checked by the
// synchronous entry points).
__device__ int g_gemm_timeout;

// The GEMM's tile: 128 rows (the MMA's M, one TMEM lane per row) x 32
// columns (N; 32 FP32 accumulator columns of TMEM, the smallest allocation),
// K staged 64 at a time.  (64 columns measured 4-25 % slower on the
// network's shapes: half as many blocks for these small GEMMs.)
constexpr int TM = 128, TN = 32, TK = 64;
constexpr int kSmemA = TM * TK * 2, kSmemB = TN * TK * 2;
// Dynamic shared memory per block: the two operand tiles and the barrier;
// 40 KB also keeps at most 5 blocks (160 TMEM columns of 512) on an SM.
constexpr int kGemmSmem = 40 * 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// A K-major operand tile without swizzle is stored as core matrices of 8
// rows x 8 BF16 (16 bytes per row, 128 contiguous bytes); rows 8g.., k
// 8j.. at byte (g * TK / 8 + j) * 128.  Its shared-memory descriptor: start
// address, the leading byte offset (next core matrix along K: 128), the
// stride byte offset (next 8 rows: TK / 8 * 128), descriptor version 1, no
// swizzle.
__device__ __forceinline__ int core_off(int r, int k) {
  return ((r >> 3) * (TK / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}
__device__ __forceinline__ uint64_t operand_desc(uint32_t saddr) {
  const uint64_t lbo = 128, sbo = (TK / 8) * 128;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((lbo >> 4) & 0x3FFF) << 16 | ((sbo >> 4) & 0x3FFF) << 32 |
         (uint64_t)1 << 46;
}
// The instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B,
// both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Waits for phase `parity` of the barrier; gives up (false) after 2^22 tries.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// C = act(op(A) op(B) + bias), a 128 x 32 tile per block of 4 warps.  Per K
// stage the block converts its A and B tiles to BF16 into shared memory (out
// of range: zero), one thread issues four 128 x 32 x 16 MMAs accumulating in
// tensor memory and commits them to a barrier that every thread waits on;
// then each warp reads its 32 rows of the accumulator (tcgen05.ld) for the
// epilogue.  Warp 0 allocates and frees the 32 TMEM columns.
__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g) {
  extern __shared__ __align__(128) unsigned char gsm[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(gsm);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(gsm + kSmemA);
  uint64_t* bar = reinterpret_cast<uint64_t*>(gsm + kSmemA + kSmemB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(gsm + kSmemA + kSmemB + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int kb = g.part ? blockIdx.z * g.kc : 0, ke = g.part ? min(g.K, kb + g.kc) : g.K;
  const uint32_t bar_a = smem_u32(bar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)), "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  uint32_t parity = 0;
  bool ok = true;
  for (int k0 = kb; k0 < ke && ok; k0 += TK) {
    for (int idx = tid; idx < TM * TK; idx += 128) {
      const int r = idx / TK, k = idx % TK, m = m0 + r, kk = k0 + k;
      float v = 0.f;
      if (m < g.M && kk < ke) v = g.transA ? g.A[(size_t)kk * g.lda + m] : g.A[(size_t)m * g.lda + kk];
      As[core_off(r, k)] = __float2bfloat16_rn(v);
    }
    for (int idx = tid; idx < TN * TK; idx += 128) {
      const int c = idx / TK, k = idx % TK, n = n0 + c, kk = k0 + k;
      float v = 0.f;
      if (n < g.N && kk < ke) v = g.transB ? g.B[(size_t)n * g.ldb + kk] : g.B[(size_t)kk * g.ldb + n];
      Bs[core_off(c, k)] = __float2bfloat16_rn(v);
    }
    // the tiles were written through the generic proxy; the MMAs read them
    // through the async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sa = smem_u32(As), sb = smem_u32(Bs);
      for (int s = 0; s < TK / 16; ++s) {
        const uint64_t da = operand_desc(sa + s * 256), db = operand_desc(sb + s * 256);
        const uint32_t accumulate = (k0 > kb || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(mma_idesc(TM, TN)), "r"(accumulate)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_a)
                   : "memory");
    }
    ok = mbar_wait(bar_a, parity);
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    ok = __syncthreads_and(ok) != 0;  // block-uniform: every warp takes the same path
  }
  if (!ok) {
    if (tid == 0) atomicExch(&g_gemm_timeout, 1);
    mbar_wait(bar_a, parity ^ 1u);  // once more (bounded) for MMAs still in flight
  } else {
    for (int c0 = 0; c0 < TN; c0 += 8) {
      uint32_t r[8];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                   : "r"(ta)
                   : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      const int row = m0 + warp * 32 + lane;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = n0 + c0 + j;
        if (row < g.M && col < g.N && g.part) {
          g.part[((size_t)blockIdx.z * g.M + row) * g.N + col] = __uint_as_float(r[j]);
        } else if (row < g.M && col < g.N) {
          float v = __uint_as_float(r[j]) + (g.bias ? g.bias[col] : 0.f);
          if (g.Z) g.Z[(size_t)row * g.ldc + col] = v;
          if (g.gelu) v = gelu_f(v);
          g.C[(size_t)row * g.ldc + col] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TN) : "memory");
}

// The epilogue of a split-K GEMM: per element the splits' partial sums in
// split order, then bias, pre-activation and activation as in the GEMM.
__global__ void splitk_reduce_kernel(GemmArgs g, int splits) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)g.M * g.N) return;
  const int row = (int)(e / g.N), col = (int)(e % g.N);
  float v = 0.f;
  for (int z = 0; z < splits; ++z) v += g.part[((size_t)z * g.M + row) * g.N + col];
  v += g.bias ? g.bias[col] : 0.f;
  if (g.Z) g.Z[(size_t)row * g.ldc + col] = v;
  if (g.gelu) v = gelu_f(v);
  g.C[(size_t)row * g.ldc + col] = v;
}

// dA *= GELU'(Z), elementwise.
__global__ void gelu_backward_kernel(float* dA, const float* Z, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dA[i] *= gelu_grad_f(Z[i]);
}

// db[c] = sum over rows of dZ[r][c], rows in order (one thread per column).
__global__ void colsum_kernel(const float* dZ, int M, int N, float* db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.f;
  for (int r = 0; r < M; ++r) s += dZ[(size_t)r * N + c];
  db[c] = s;
}

// MSE: dY = 2 (Y - T) / (M N); loss = mean (Y - T)^2, summed in fixed order by one block.
__global__ void mse_kernel(const float* Y, const float* T, int64_t n, float* dY, float* loss) {
  __shared__ double red[256];
  double s = 0.0;
  const float scale = 2.0f / (float)n;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = scale * d;
    s += (double)d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)(red[0] / (double)n);
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void gather_rows_kernel(const float* src, const int32_t* idx, int rows, int cols, float* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  dst[i] = src[(size_t)idx[r] * cols + c];
}

// Per-column mean and standard deviation of T (rows x cols), fixed order.
__global__ void col_stats_kernel(const float* T, int rows, int cols, float* mean, float* sd) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0, s2 = 0.0;
  for (int r = 0; r < rows; ++r) {
    const double x = T[(size_t)r * cols + c];
    s += x;
    s2 += x * x;
  }
  const double mu = s / rows;
  const double var = s2 / rows - mu * mu;
  mean[c] = (float)mu;
  sd[c] = (float)(var > 1e-30 ? sqrt(var) : 1.0);
}

__global__ void standardise_kernel(const float* T, int rows, int cols, const float* mean, const float* sd, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const int c = (int)(i % cols);
  out[i] = (T[i] - mean[c]) / sd[c];
}

// y = y * scale + shift per column (the output affine of a standardised net).
__global__ void affine_cols_kernel(float* Y, int rows, int cols, const float* scale, const float* shift) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const int c = (int)(i % cols);
  Y[i] = Y[i] * scale[c] + shift[c];
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// A GEMM whose output tiles are few and whose K is long (the weight
// gradients: K = the batch) splits K over up to kMaxSplits blocks per tile,
// each at least two stages long, into `ws` (splits x M x N floats), and sums
// the splits in order in a second kernel.
constexpr int kMaxSplits = 16;
int gemm_splits(int M, int N, int K) {
  const int tiles = ((N + TN - 1) / TN) * ((M + TM - 1) / TM);
  if (tiles >= 32 || K < 4 * TK) return 1;
  return std::max(1, std::min(kMaxSplits, K / (2 * TK)));
}
size_t gemm_ws_floats(int M, int N, int K) {
  const int s = gemm_splits(M, N, K);
  return s > 1 ? (size_t)s * M * N : 0;
}
void gemm_bf16(const float* A, int lda, bool tA, const float* B, int ldb, bool tB, float* C, int ldc, int M, int N,
               int K, const float* bias, float* Z, bool gelu, float* ws, size_t ws_floats, cudaStream_t st) {
  GemmArgs g{A, B, C, bias, Z, M, N, K, lda, ldb, ldc, tA ? 1 : 0, tB ? 1 : 0, gelu ? 1 : 0, nullptr, K};
  const int splits = (ws && gemm_ws_floats(M, N, K) <= ws_floats) ? gemm_splits(M, N, K) : 1;
  if (splits > 1) {
    g.kc = ((K + splits - 1) / splits + TK - 1) / TK * TK;
    g.part = ws;
  }
  const int used = splits > 1 ? (K + g.kc - 1) / g.kc : 1;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, used);
  note_launches(1, st);
  gemm_bf16_kernel<<<grid, 128, kGemmSmem, st>>>(g);
  if (used > 1) {
    note_launches(1, st);
    splitk_reduce_kernel<<<blocks_for((int64_t)M * N, 256), 256, 0, st>>>(g, used);
  }
}

// After a synchronisation: RF_E_TIMEOUT (and the flag cleared) if a GEMM gave
// up waiting for its tensor-core work since the last check.
rf_status gemm_status(const char* what) {
  int flag = 0;
  if (!cuda_ok(cudaMemcpyFromSymbol(&flag, g_gemm_timeout, sizeof(int)), what)) return RF_E_CUDA;
  if (!flag) return RF_OK;
  const int zero = 0;
  cudaMemcpyToSymbol(g_gemm_timeout, &zero, sizeof(int));
  set_error(std::string(what) + ": a GEMM's wait for its tensor-core work gave up");
  return RF_E_TIMEOUT;
}

}  // namespace rf

using namespace rf;

struct rf_mlp {
  std::vector<int> dims;  // n_in, hidden..., n_out
  int64_t n_params = 0;
  std::vector<int64_t> w_off, b_off;
  DevBuf params, grads, m, v;
  DevBuf acts, zs, dbuf, dbuf2, y, t_std, loss, idx, xb, tb, mean, sd, scale, shift;
  DevBuf pred_h, pred_y;  // rf_mlp_predict: histograms and outputs of the sets
  DevBuf splitk;          // partial tiles of the split-K GEMMs
  int cap = 0;  // batch capacity of the activation buffers
  int64_t step = 0;
  bool has_affine = false;
};

namespace rf {
namespace {

bool mlp_reserve(rf_mlp* n, int batch) {
  if (batch <= n->cap) return true;
  int64_t act = 0, z = 0;
  for (size_t l = 0; l + 1 < n->dims.size(); ++l) {
    act += (int64_t)batch * n->dims[l];
    z += (int64_t)batch * n->dims[l + 1];
  }
  int wmax = *std::max_element(n->dims.begin(), n->dims.end());
  const int nout = n->dims.back();
  size_t ws = 0;  // the split-K GEMMs' partial tiles: forward, weight gradient, input gradient
  for (size_t l = 0; l + 1 < n->dims.size(); ++l) {
    const int ni = n->dims[l], no = n->dims[l + 1];
    ws = std::max({ws, gemm_ws_floats(batch, no, ni), gemm_ws_floats(ni, no, batch), gemm_ws_floats(batch, ni, no)});
  }
  if (ws && !n->splitk.ensure(sizeof(float) * ws)) return false;
  bool ok = n->acts.ensure(sizeof(float) * act) && n->zs.ensure(sizeof(float) * z) &&
            n->dbuf.ensure(sizeof(float) * (size_t)batch * wmax) && n->dbuf2.ensure(sizeof(float) * (size_t)batch * wmax) &&
            n->y.ensure(sizeof(float) * (size_t)batch * nout) && n->t_std.ensure(sizeof(float) * (size_t)batch * nout) &&
            n->loss.ensure(sizeof(float)) && n->xb.ensure(sizeof(float) * (size_t)batch * n->dims[0]) &&
            n->tb.ensure(sizeof(float) * (size_t)batch * nout) && n->idx.ensure(sizeof(int32_t) * batch);
  if (!ok) return false;
  n->cap = batch;
  return true;
}

// Forward over `batch` rows of x; keeps every layer's input activation and
// pre-activation for the backward pass; output into n->y.
void mlp_forward(rf_mlp* n, const float* x, int batch, cudaStream_t st) {
  const float* P = (const float*)n->params.p;
  float* acts = (float*)n->acts.p;
  float* zs = (float*)n->zs.p;
  const int L = (int)n->dims.size() - 1;
  cudaMemcpyAsync(acts, x, sizeof(float) * (size_t)batch * n->dims[0], cudaMemcpyDeviceToDevice, st);
  int64_t ao = 0, zo = 0;
  for (int l = 0; l < L; ++l) {
    const int ni = n->dims[l], no = n->dims[l + 1];
    float* a_in = acts + ao;
    float* out = (l == L - 1) ? (float*)n->y.p : acts + ao + (int64_t)batch * ni;
    gemm_bf16(a_in, ni, false, P + n->w_off[l], no, false, out, no, batch, no, ni, P + n->b_off[l], zs + zo,
              l < L - 1, (float*)n->splitk.p, n->splitk.bytes / sizeof(float), st);
    ao += (int64_t)batch * ni;
    zo += (int64_t)batch * no;
  }
}

// Backward from dY (batch x n_out, in n->dbuf) into n->grads.
void mlp_backward(rf_mlp* n, int batch, cudaStream_t st) {
  const float* P = (const float*)n->params.p;
  float* G = (float*)n->grads.p;
  const float* acts = (const float*)n->acts.p;
  const float* zs = (const float*)n->zs.p;
  const int L = (int)n->dims.size() - 1;
  std::vector<int64_t> ao(L), zo(L);
  int64_t a = 0, z = 0;
  for (int l = 0; l < L; ++l) {
    ao[l] = a;
    zo[l] = z;
    a += (int64_t)batch * n->dims[l];
    z += (int64_t)batch * n->dims[l + 1];
  }
  float* d = (float*)n->dbuf.p;
  float* d2 = (float*)n->dbuf2.p;
  for (int l = L - 1; l >= 0; --l) {
    const int ni = n->dims[l], no = n->dims[l + 1];
    if (l < L - 1) {
      const int64_t cnt = (int64_t)batch * no;
      note_launches(1, st);
      gelu_backward_kernel<<<blocks_for(cnt, 256), 256, 0, st>>>(d, zs + zo[l], cnt);
    }
    // dW = a_in^T dZ  (ni x no), db = column sums of dZ
    gemm_bf16(acts + ao[l], ni, true, d, no, false, G + n->w_off[l], no, ni, no, batch, nullptr, nullptr, false,
              (float*)n->splitk.p, n->splitk.bytes / sizeof(float), st);
    note_launches(1, st);
    colsum_kernel<<<blocks_for(no, 128), 128, 0, st>>>(d, batch, no, G + n->b_off[l]);
    if (l > 0) {
      // dA_in = dZ W^T  (batch x ni)
      gemm_bf16(d, no, false, P + n->w_off[l], no, true, d2, ni, batch, ni, no, nullptr, nullptr, false,
                (float*)n->splitk.p, n->splitk.bytes / sizeof(float), st);
      std::swap(d, d2);
    }
  }
}

// Loss and gradient for targets already standardised (in t).
rf_status mlp_loss_grad(rf_mlp* n, const float* x, const float* t, int batch, cudaStream_t st) {
  mlp_forward(n, x, batch, st);
  const int64_t cnt = (int64_t)batch * n->dims.back();
  note_launches(1, st);
  mse_kernel<<<1, 256, 0, st>>>((const float*)n->y.p, t, cnt, (float*)n->dbuf.p, (float*)n->loss.p);
  mlp_backward(n, batch, st);
  return cuda_ok(cudaGetLastError(), "mlp launch") ? RF_OK : RF_E_CUDA;
}

void mlp_adam(rf_mlp* n, float lr, cudaStream_t st) {
  ++n->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
  note_launches(1, st);
  adam_kernel<<<blocks_for(n->n_params, 256), 256, 0, st>>>((float*)n->params.p, (const float*)n->grads.p,
                                                             (float*)n->m.p, (float*)n->v.p, n->n_params, lr, b1, b2,
                                                             1e-8f, c1, c2);
}

}  // namespace
}  // namespace rf

extern "C" {

rf_status rf_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_hidden_layers, int32_t n_out, uint64_t seed,
                        rf_mlp** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_hidden_layers < 0 || n_out < 1 || n_in > 4096 || n_hidden > 4096 ||
      n_out > 4096 || n_hidden_layers > 16) {
    set_error("rf_mlp_create: bad dimensions");
    return RF_E_INVALID;
  }
  rf_mlp* n = new (std::nothrow) rf_mlp();
  if (!n) return RF_E_OOM;
  n->dims.push_back(n_in);
  for (int i = 0; i < n_hidden_layers; ++i) n->dims.push_back(n_hidden);
  n->dims.push_back(n_out);
  int64_t off = 0;
  for (size_t l = 0; l + 1 < n->dims.size(); ++l) {
    n->w_off.push_back(off);
    off += (int64_t)n->dims[l] * n->dims[l + 1];
    n->b_off.push_back(off);
    off += n->dims[l + 1];
  }
  n->n_params = off;
  // Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, from a seeded mt19937_64.
  std::vector<float> h(off, 0.f);
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (size_t l = 0; l + 1 < n->dims.size(); ++l) {
    const double bound = 1.0 / std::sqrt((double)n->dims[l]);
    for (int64_t i = 0; i < (int64_t)n->dims[l] * n->dims[l + 1]; ++i) h[n->w_off[l] + i] = (float)(bound * U(rng));
  }
  std::vector<float> zeros(off, 0.f);
  if (!n->params.ensure(sizeof(float) * off) || !n->grads.ensure(sizeof(float) * off) ||
      !n->m.ensure(sizeof(float) * off) || !n->v.ensure(sizeof(float) * off) ||
      !n->scale.ensure(sizeof(float) * n_out) || !n->shift.ensure(sizeof(float) * n_out) ||
      !n->mean.ensure(sizeof(float) * n_out) || !n->sd.ensure(sizeof(float) * n_out)) {
    delete n;
    return RF_E_OOM;
  }
  if (!cuda_ok(cudaMemcpy(n->params.p, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice), "mlp init") ||
      !cuda_ok(cudaMemcpy(n->m.p, zeros.data(), sizeof(float) * off, cudaMemcpyHostToDevice), "mlp init") ||
      !cuda_ok(cudaMemcpy(n->v.p, zeros.data(), sizeof(float) * off, cudaMemcpyHostToDevice), "mlp init") ||
      !cuda_ok(cudaMemcpy(n->grads.p, zeros.data(), sizeof(float) * off, cudaMemcpyHostToDevice), "mlp init")) {
    delete n;
    return RF_E_CUDA;
  }
  *out = n;
  return RF_OK;
}

void rf_mlp_destroy(rf_mlp* n) { delete n; }

int64_t rf_mlp_n_params(const rf_mlp* n) { return n ? n->n_params : 0; }

rf_status rf_mlp_get_params(const rf_mlp* n, float* host) {
  if (!n || !host) { set_error("rf_mlp_get_params: bad argument"); return RF_E_INVALID; }
  return cuda_ok(cudaMemcpy(host, n->params.p, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost), "mlp params")
             ? RF_OK : RF_E_CUDA;
}

rf_status rf_mlp_set_params(rf_mlp* n, const float* host) {
  if (!n || !host) { set_error("rf_mlp_set_params: bad argument"); return RF_E_INVALID; }
  return cuda_ok(cudaMemcpy(n->params.p, host, sizeof(float) * n->n_params, cudaMemcpyHostToDevice), "mlp params")
             ? RF_OK : RF_E_CUDA;
}

rf_status rf_mlp_forward(rf_mlp* n, const float* d_x, int32_t batch, float* d_y, void* stream) {
  if (!n || !d_x || !d_y || batch < 0) { set_error("rf_mlp_forward: bad argument"); return RF_E_INVALID; }
  if (batch == 0) return RF_OK;
  if (!mlp_reserve(n, batch)) return RF_E_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  mlp_forward(n, d_x, batch, st);
  const int no = n->dims.back();
  if (n->has_affine) {
    note_launches(1, st);
    affine_cols_kernel<<<blocks_for((int64_t)batch * no, 256), 256, 0, st>>>((float*)n->y.p, batch, no,
                                                                            (const float*)n->scale.p,
                                                                            (const float*)n->shift.p);
  }
  cudaMemcpyAsync(d_y, n->y.p, sizeof(float) * (size_t)batch * no, cudaMemcpyDeviceToDevice, st);
  return cuda_ok(cudaGetLastError(), "rf_mlp_forward") ? RF_OK : RF_E_CUDA;
}

rf_status rf_mlp_grad(rf_mlp* n, const float* d_x, const float* d_t, int32_t batch, float* loss, float* d_grad,
                      void* stream) {
  if (!n || !d_x || !d_t || batch < 1) { set_error("rf_mlp_grad: bad argument"); return RF_E_INVALID; }
  if (!mlp_reserve(n, batch)) return RF_E_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  rf_status s = mlp_loss_grad(n, d_x, d_t, batch, st);
  if (s != RF_OK) return s;
  if (d_grad) cudaMemcpyAsync(d_grad, n->grads.p, sizeof(float) * n->n_params, cudaMemcpyDeviceToDevice, st);
  if (loss) {
    if (!cuda_ok(cudaMemcpyAsync(loss, n->loss.p, sizeof(float), cudaMemcpyDeviceToHost, st), "loss") ||
        !cuda_ok(cudaStreamSynchronize(st), "loss"))
      return RF_E_CUDA;
    return gemm_status("rf_mlp_grad");
  }
  return RF_OK;
}

rf_status rf_mlp_adam(rf_mlp* n, float lr, void* stream) {
  if (!n || !(lr >= 0.f)) { set_error("rf_mlp_adam: bad argument"); return RF_E_INVALID; }
  mlp_adam(n, lr, (cudaStream_t)stream);
  return cuda_ok(cudaGetLastError(), "rf_mlp_adam") ? RF_OK : RF_E_CUDA;
}

rf_status rf_mlp_train(rf_mlp* n, const float* d_x, const float* d_t, int32_t rows, int32_t batch, int32_t epochs,
                       float lr, uint64_t seed, int32_t standardise, float* final_loss) {
  if (!n || !d_x || !d_t || rows < 1 || batch < 1 || epochs < 1 || !(lr > 0.f)) {
    set_error("rf_mlp_train: bad argument");
    return RF_E_INVALID;
  }
  batch = std::min(batch, rows);
  if (!mlp_reserve(n, batch)) return RF_E_OOM;
  const int ni = n->dims[0], no = n->dims.back();
  DevBuf tstd;
  const float* targets = d_t;
  if (standardise) {
    if (!tstd.ensure(sizeof(float) * (size_t)rows * no)) return RF_E_OOM;
    note_launches(1, nullptr);
    col_stats_kernel<<<1, 128>>>(d_t, rows, no, (float*)n->mean.p, (float*)n->sd.p);
    note_launches(1, nullptr);
    standardise_kernel<<<blocks_for((int64_t)rows * no, 256), 256>>>(d_t, rows, no, (const float*)n->mean.p,
                                                                    (const float*)n->sd.p, (float*)tstd.p);
    targets = (const float*)tstd.p;
    cudaMemcpy(n->scale.p, n->sd.p, sizeof(float) * no, cudaMemcpyDeviceToDevice);
    cudaMemcpy(n->shift.p, n->mean.p, sizeof(float) * no, cudaMemcpyDeviceToDevice);
    n->has_affine = true;
  }
  std::mt19937_64 rng(seed);
  std::vector<int32_t> perm(rows);
  for (int i = 0; i < rows; ++i) perm[i] = i;
  DevBuf dperm;
  if (!dperm.ensure(sizeof(int32_t) * rows)) return RF_E_OOM;
  const int steps_per_epoch = rows / batch;  // drop the ragged remainder
  const int64_t total = (int64_t)steps_per_epoch * epochs;
  int64_t it = 0;
  double last_epoch = 0.0;
  std::vector<float> losses(steps_per_epoch);
  for (int e = 0; e < epochs; ++e) {
    std::shuffle(perm.begin(), perm.end(), rng);
    if (!cuda_ok(cudaMemcpy(dperm.p, perm.data(), sizeof(int32_t) * rows, cudaMemcpyHostToDevice), "perm"))
      return RF_E_CUDA;
    double sum = 0.0;
    for (int s = 0; s < steps_per_epoch; ++s, ++it) {
      const int32_t* ids = (const int32_t*)dperm.p + (size_t)s * batch;
      note_launches(1, nullptr);
      gather_rows_kernel<<<blocks_for((int64_t)batch * ni, 256), 256>>>(d_x, ids, batch, ni, (float*)n->xb.p);
      note_launches(1, nullptr);
      gather_rows_kernel<<<blocks_for((int64_t)batch * no, 256), 256>>>(targets, ids, batch, no, (float*)n->tb.p);
      rf_status st = mlp_loss_grad(n, (const float*)n->xb.p, (const float*)n->tb.p, batch, 0);
      if (st != RF_OK) return st;
      // cosine decay from lr to 0 over all steps
      const float lr_t = (float)(0.5 * lr * (1.0 + std::cos(M_PI * (double)it / (double)total)));
      mlp_adam(n, lr_t, 0);
      cudaMemcpyAsync(&losses[s], n->loss.p, sizeof(float), cudaMemcpyDeviceToHost, 0);
    }
    if (!cuda_ok(cudaDeviceSynchronize(), "rf_mlp_train")) return RF_E_CUDA;
    const rf_status gs = gemm_status("rf_mlp_train");
    if (gs != RF_OK) return gs;
    for (float l : losses) sum += l;
    last_epoch = steps_per_epoch > 0 ? sum / steps_per_epoch : 0.0;
  }
  if (final_loss) *final_loss = (float)last_epoch;
  return RF_OK;
}

rf_status rf_mlp_save(const rf_mlp* n, const char* path) {
  if (!n || !path) { set_error("rf_mlp_save: bad argument"); return RF_E_INVALID; }
  const int no = n->dims.back();
  std::vector<float> p(n->n_params), m(n->n_params), v(n->n_params), sc(no), sh(no);
  cudaMemcpy(p.data(), n->params.p, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost);
  cudaMemcpy(m.data(), n->m.p, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost);
  cudaMemcpy(v.data(), n->v.p, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost);
  cudaMemcpy(sc.data(), n->scale.p, sizeof(float) * no, cudaMemcpyDeviceToHost);
  cudaMemcpy(sh.data(), n->shift.p, sizeof(float) * no, cudaMemcpyDeviceToHost);
  if (!cuda_ok(cudaGetLastError(), "rf_mlp_save")) return RF_E_CUDA;
  FILE* f = std::fopen(path, "wb");
  if (!f) { set_error("rf_mlp_save: cannot open file"); return RF_E_INVALID; }
  const int32_t magic = 0x524d4c50, nd = (int32_t)n->dims.size(), aff = n->has_affine ? 1 : 0;
  std::fwrite(&magic, 4, 1, f);
  std::fwrite(&nd, 4, 1, f);
  std::fwrite(n->dims.data(), 4, nd, f);
  std::fwrite(&n->step, 8, 1, f);
  std::fwrite(&aff, 4, 1, f);
  std::fwrite(p.data(), 4, n->n_params, f);
  std::fwrite(m.data(), 4, n->n_params, f);
  std::fwrite(v.data(), 4, n->n_params, f);
  std::fwrite(sc.data(), 4, no, f);
  std::fwrite(sh.data(), 4, no, f);
  const bool ok = std::fclose(f) == 0;
  if (!ok) { set_error("rf_mlp_save: write failed"); return RF_E_INVALID; }
  return RF_OK;
}

rf_status rf_mlp_load(const char* path, rf_mlp** out) {
  if (!path || !out) { set_error("rf_mlp_load: bad argument"); return RF_E_INVALID; }
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) { set_error("rf_mlp_load: cannot open file"); return RF_E_INVALID; }
  int32_t magic = 0, nd = 0;
  bool ok = std::fread(&magic, 4, 1, f) == 1 && magic == 0x524d4c50 && std::fread(&nd, 4, 1, f) == 1 && nd >= 2 && nd <= 18;
  std::vector<int32_t> dims(ok ? nd : 0);
  ok = ok && std::fread(dims.data(), 4, nd, f) == (size_t)nd;
  if (!ok || dims[1] < 1) {
    std::fclose(f);
    set_error("rf_mlp_load: not a model file");
    return RF_E_INVALID;
  }
  rf_mlp* n = nullptr;
  rf_status s = rf_mlp_create(dims[0], nd > 2 ? dims[1] : 1, nd - 2, dims[nd - 1], 0, &n);
  if (s != RF_OK) {
    std::fclose(f);
    return s;
  }
  int32_t aff = 0;
  const int no = dims[nd - 1];
  std::vector<float> p(n->n_params), m(n->n_params), v(n->n_params), sc(no), sh(no);
  ok = std::fread(&n->step, 8, 1, f) == 1 && std::fread(&aff, 4, 1, f) == 1 &&
       std::fread(p.data(), 4, n->n_params, f) == (size_t)n->n_params &&
       std::fread(m.data(), 4, n->n_params, f) == (size_t)n->n_params &&
       std::fread(v.data(), 4, n->n_params, f) == (size_t)n->n_params && std::fread(sc.data(), 4, no, f) == (size_t)no &&
       std::fread(sh.data(), 4, no, f) == (size_t)no;
  std::fclose(f);
  if (!ok) {
    delete n;
    set_error("rf_mlp_load: truncated file");
    return RF_E_INVALID;
  }
  n->has_affine = aff != 0;
  cudaMemcpy(n->params.p, p.data(), sizeof(float) * n->n_params, cudaMemcpyHostToDevice);
  cudaMemcpy(n->m.p, m.data(), sizeof(float) * n->n_params, cudaMemcpyHostToDevice);
  cudaMemcpy(n->v.p, v.data(), sizeof(float) * n->n_params, cudaMemcpyHostToDevice);
  cudaMemcpy(n->scale.p, sc.data(), sizeof(float) * no, cudaMemcpyHostToDevice);
  cudaMemcpy(n->shift.p, sh.data(), sizeof(float) * no, cudaMemcpyHostToDevice);
  if (!cuda_ok(cudaGetLastError(), "rf_mlp_load")) {
    delete n;
    return RF_E_CUDA;
  }
  *out = n;
  return RF_OK;
}

}  // extern "C"

extern "C" rf_status rf_mlp_predict(rf_mlp* n, const rf_model* m, const rf_data* d, int32_t col, double* theta0) {
  if (!n || !m || !d || !theta0) {
    set_error("rf_mlp_predict: bad argument (NULL)");
    return RF_E_INVALID;
  }
  const int S = rf_data_n_sets(d), no = n->dims.back();
  if (n->dims.front() != 64 || no != rf_model_n_free(m)) {
    set_error("rf_mlp_predict: the network must map 64 histogram bins to the model's free parameters");
    return RF_E_INVALID;
  }
  if (S == 0) return RF_OK;
  if (!n->pred_h.ensure(sizeof(float) * (size_t)S * 64) || !n->pred_y.ensure(sizeof(float) * (size_t)S * no))
    return RF_E_OOM;
  rf_status st = rf_hist64(m, d, col, (float*)n->pred_h.p, nullptr);
  if (st != RF_OK) return st;
  st = rf_mlp_forward(n, (const float*)n->pred_h.p, S, (float*)n->pred_y.p, nullptr);
  if (st != RF_OK) return st;
  std::vector<float> y((size_t)S * no);
  if (!cuda_ok(cudaMemcpy(y.data(), n->pred_y.p, sizeof(float) * y.size(), cudaMemcpyDeviceToHost), "rf_mlp_predict"))
    return RF_E_CUDA;
  st = gemm_status("rf_mlp_predict");
  if (st != RF_OK) return st;
  // A start on (or beyond) a bound sits where the fit's bound transform is
  // stationary (d theta / d phi = 0): that parameter barely moves.  Bounded
  // predictions are kept kStartMargin of the range inside the bounds.
  const std::vector<double>& lo = m->m.lo;
  const std::vector<double>& hi = m->m.hi;
  for (int s = 0; s < S; ++s)
    for (int k = 0; k < no; ++k) {
      double t = (double)y[(size_t)s * no + k];
      if (lo[k] < hi[k] && std::isfinite(lo[k]) && std::isfinite(hi[k])) {
        const double a = lo[k] + kStartMargin * (hi[k] - lo[k]), b = hi[k] - kStartMargin * (hi[k] - lo[k]);
        t = t < a ? a : (t > b ? b : t);
      }
      theta0[(size_t)s * no + k] = t;
    }
  return RF_OK;
}
