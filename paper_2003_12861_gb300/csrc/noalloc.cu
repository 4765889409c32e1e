// rf_nll_grad_noalloc: NLL and gradient of one dataset without any device
// allocation.  For callers that cannot call cudaMalloc while they run -- e.g.
// an online event filter or any service that reserves all of its GPU memory
// at start-up, because an allocation in the middle of data taking has
// unbounded latency, may fail once memory is fragmented, and can synchronise
// the device behind the caller's back -- the scratch of the pass (constant
// block, work items, reduction tree, arrival tickets, counters) lives in the
// file-scope static device array below instead of library-allocated buffers.
//
// The array is part of the library's module: every GPU that loads the
// library holds kScratchBytes of it until the process exits, and every call
// on that GPU shares it.  Calls that overlap on the GPU (different streams
// or threads) race on it; serialise them.  The first call on each device
// looks up the array's device address with cudaGetSymbolAddress while that
// device is current; make that first call before any stream capture.  No
// device memory is allocated by any call; a rejected call copies its message
// into the library's thread-local error string (host memory).
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "api_internal.h"
#include "nll_ff.cuh"
#include "nll_kernels.cuh"

namespace rf {

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of the pass's scratch inside the array.
struct Layout {
  size_t consts, ffc, items, bad, tickets, tree, part_m, part_fb, part_info, total;
};

// Header (first 256 bytes): int32 counter @0, u64 slow-event count @8,
// int64 offsets[2] @16, int64 tree base @32, int32 active set @40.
Layout layout_for(int64_t chunks, int64_t nodes, int n_const, int Q, bool parts, int shape) {
  const size_t np = (size_t)parts_for(chunks, shape);
  Layout L{};
  L.consts = 256;
  L.ffc = L.consts + up256(sizeof(double) * (size_t)(n_const > 0 ? n_const : 1));
  L.items = L.ffc + up256(sizeof(float) * kFFConst);
  L.bad = L.items + up256(sizeof(int2) * (size_t)(chunks > 0 ? chunks : 1));
  L.tickets = L.bad + up256(sizeof(int32_t) * (size_t)(nodes > 0 ? nodes : 1));
  L.tree = L.tickets + up256(sizeof(int32_t) * (size_t)(nodes > 0 ? nodes : 1));
  // float-float kernels only: the part records of every chunk
  const size_t nn = parts ? (size_t)(nodes > 0 ? nodes : 1) : 0;
  L.part_m = L.tree + up256(sizeof(double) * 2 * (size_t)Q * (size_t)(nodes > 0 ? nodes : 1));
  L.part_fb = L.part_m + up256(sizeof(float) * np * kPartFloats * nn);
  L.part_info = L.part_fb + up256(sizeof(double) * np * (size_t)Q * nn);
  L.total = L.part_info + sizeof(int32_t) * np * nn;
  return L;
}

// Fills the header, the work items and clears the tickets (the array keeps
// the previous call's contents).
__global__ void noalloc_setup(unsigned char* base, Layout L, int64_t n_events, int64_t chunks, int64_t nodes) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i0 == 0) {
    *(int32_t*)(base + 0) = 0;
    *(unsigned long long*)(base + 8) = 0ull;
    ((int64_t*)(base + 16))[0] = 0;
    ((int64_t*)(base + 16))[1] = n_events;
    *(int64_t*)(base + 32) = 0;
    *(int32_t*)(base + 40) = 0;
  }
  int2* items = (int2*)(base + L.items);
  int32_t* tickets = (int32_t*)(base + L.tickets);
  const int64_t n = chunks > nodes ? chunks : nodes;
  for (int64_t i = i0; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < chunks) items[i] = make_int2(0, (int)i);
    if (i < nodes) tickets[i] = 0;
  }
}

// Scratch bytes of a pass over n_events events of model m.
size_t scratch_bytes(const rf_model* m, int64_t n_events) {
  const Program& P = m->m.prog;
  const int64_t chunks = (n_events + kChunk - 1) / kChunk;
  return layout_for(chunks, tree_nodes(chunks), P.n_const, 1 + P.n_slots, m->m.shape != SHAPE_GENERIC, m->m.shape).total;
}

}  // namespace

}  // namespace rf

using namespace rf;

extern "C" rf_status rf_nll_grad_noalloc_max_events(const rf_model* m, int64_t* max_events) {
  if (!m || !max_events) {
    set_error("rf_nll_grad_noalloc_max_events: bad argument");
    return RF_E_INVALID;
  }
  // the scratch grows with the chunk count: bisect on whole chunks, then
  // every event count up to the last fitting chunk's end fits too
  int64_t lo = 0, hi = int64_t(1) << 31;  // chunks; 2^31 chunks never fit 16 MiB
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (scratch_bytes(m, mid * kChunk) <= kScratchBytes) lo = mid;
    else hi = mid;
  }
  *max_events = lo * kChunk;
  return RF_OK;
}

extern "C" rf_status rf_nll_grad_noalloc(const rf_model* m, const void* const* d_cols, const int32_t* dtype,
                                         int64_t n_events, const double* d_theta, double* d_out, int32_t* d_flags,
                                         void* stream) {
  if (!m || (n_events > 0 && !d_cols) || n_events < 0 || !d_out || !d_flags ||
      (m->m.prog.n_free > 0 && !d_theta)) {
    set_error("rf_nll_grad_noalloc: bad argument");
    return RF_E_INVALID;
  }
  const Program& P = m->m.prog;
  const int64_t chunks = (n_events + kChunk - 1) / kChunk;
  const int64_t nodes = tree_nodes(chunks);
  const int Q = 1 + P.n_slots;
  const Layout L = layout_for(chunks, nodes, P.n_const, Q, m->m.shape != SHAPE_GENERIC, m->m.shape);
  if (L.total > kScratchBytes || chunks > (int64_t)0x7fffffff) {
    const double per_chunk = (double)L.total / (double)(chunks > 0 ? chunks : 1);
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "rf_nll_grad_noalloc: %lld events need %zu bytes of scratch; the static array holds %zu bytes "
                  "(about %lld events for this model)",
                  (long long)n_events, L.total, kScratchBytes, (long long)(kScratchBytes / per_chunk) * kChunk);
    set_error(msg);
    return RF_E_INVALID;
  }
  Columns cols{};
  for (int c = 0; c < P.n_obs; ++c) {
    const int32_t dt = dtype ? dtype[c] : RF_F64;
    if (dt != RF_F64 && dt != RF_F32) {
      set_error("rf_nll_grad_noalloc: dtype must be RF_F64 or RF_F32");
      return RF_E_INVALID;
    }
    cols.ptr[c] = n_events > 0 ? d_cols[c] : nullptr;
    cols.is_f32[c] = dt == RF_F32;
  }
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "rf_nll_grad_noalloc")) return RF_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("rf_nll_grad_noalloc: device index beyond 63");
    return RF_E_INVALID;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (!cuda_ok(cudaGetSymbolAddress(&p, g_scratch), "rf_nll_grad_noalloc: cudaGetSymbolAddress")) return RF_E_CUDA;
      g_addr[dev] = p;
    }
    base = (unsigned char*)g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t work = chunks > nodes ? chunks : nodes;
  const int blocks = (int)((work + 255) / 256) > 0 ? (int)((work + 255) / 256) : 1;
  noalloc_setup<<<blocks < 1024 ? blocks : 1024, 256, 0, st>>>(base, L, n_events, chunks, nodes);
  note_launches(1, st);
  Pass pass{};
  pass.counter = (int32_t*)(base + 0);
  pass.slow = (unsigned long long*)(base + 8);
  pass.offsets = (const int64_t*)(base + 16);
  pass.tree_base = (const int64_t*)(base + 32);
  pass.sets = (const int32_t*)(base + 40);
  pass.n_active = 1;
  pass.items = (const int2*)(base + L.items);
  pass.n_items = (int32_t)chunks;
  pass.theta = d_theta;
  pass.consts = (double*)(base + L.consts);
  pass.tree = (double*)(base + L.tree);
  pass.tree_bad = (int32_t*)(base + L.bad);
  pass.tickets = (int32_t*)(base + L.tickets);
  pass.out = d_out;
  pass.flags = d_flags;
  pass.Q = Q;
  pass.want_grad = 1;
  pass.ff_shape = m->m.shape;
  pass.ffc = (float*)(base + L.ffc);
  pass.part_m = (float*)(base + L.part_m);
  pass.part_fb = (double*)(base + L.part_fb);
  pass.part_info = (int32_t*)(base + L.part_info);
  pass.parts = parts_for(chunks, m->m.shape);
  launch_param_point(P, pass, st);
  launch_events(P, m->m.shape, cols, pass, m->m.threads_per_block, m->m.blocks_per_sm, sm_count(), st);
  return cuda_ok(cudaGetLastError(), "rf_nll_grad_noalloc launch") ? RF_OK : RF_E_CUDA;
}
