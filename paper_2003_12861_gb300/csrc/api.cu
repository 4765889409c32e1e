// C ABI: models, datasets, likelihood entry points.
#include <atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.h"
#include "nll_ff.cuh"
#include "nll_kernels.cuh"

namespace rf {

static thread_local std::string g_error;
void set_error(const std::string& msg) { g_error = msg; }

bool cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return false;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

DevBuf::~DevBuf() { release(); }
Workspace::~Workspace() {
  for (cudaEvent_t& e : seg_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t& e : comp_ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t& c : comp_stream)
    if (c) cudaStreamDestroy(c);
  if (copy_stream) cudaStreamDestroy(copy_stream);
}
void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}
bool DevBuf::ensure(size_t b) {
  if (b <= bytes && p) return true;
  release();
  if (b == 0) b = 8;
  if (cudaMalloc(&p, b) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    set_error("device allocation of " + std::to_string(b) + " bytes failed");
    return false;
  }
  bytes = b;
  return true;
}

HostBuf::~HostBuf() {
  if (p) cudaFreeHost(p);
}
bool HostBuf::ensure(size_t b) {
  if (b <= bytes && p) return true;
  if (p) cudaFreeHost(p);
  p = nullptr;
  bytes = 0;
  if (b == 0) b = 8;
  if (cudaMallocHost(&p, b) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    set_error("pinned host allocation failed");
    return false;
  }
  bytes = b;
  return true;
}

// Radix-32 tree over `chunks` leaves: total node count.
int64_t tree_nodes(int64_t chunks) {
  if (chunks <= 0) return 0;
  int64_t total = chunks, n = chunks;
  while (n > 1) {
    n = (n + kRadix - 1) / kRadix;
    total += n;
  }
  return total;
}

// Build the (set, chunk) work items and tree bases for a list of active sets.
bool build_plan(const rf_data* d, const std::vector<int32_t>& sets, Plan* plan) {
  std::vector<int2> items;
  for (int32_t s : sets) {
    const int64_t c = d->chunks[s];
    for (int64_t k = 0; k < c; ++k) items.push_back(make_int2(s, (int)k));
  }
  plan->n_active = (int)sets.size();
  plan->n_items = (int)items.size();
  plan->host_sets = sets;
  if (!plan->sets.ensure(sizeof(int32_t) * std::max<size_t>(1, sets.size()))) return false;
  if (!plan->items.ensure(sizeof(int2) * std::max<size_t>(1, items.size()))) return false;
  if (!sets.empty() && !cuda_ok(cudaMemcpy(plan->sets.p, sets.data(), sizeof(int32_t) * sets.size(), cudaMemcpyHostToDevice), "plan upload"))
    return false;
  if (!items.empty() && !cuda_ok(cudaMemcpy(plan->items.p, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice), "plan upload"))
    return false;
  return true;
}

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

void note_launches(int n, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;
  g_launches.fetch_add(n, std::memory_order_relaxed);
}

bool ensure_workspace(const rf_model* m, rf_data* d) {
  Workspace& w = d->ws;
  const Program& P = m->m.prog;
  const int Q = 1 + P.n_slots;
  if (w.ready && w.n_const == P.n_const && w.n_free == P.n_free && w.Q == Q &&
      (m->m.shape == SHAPE_GENERIC || w.ffc.p))
    return true;
  const size_t S = d->n_sets;
  const size_t nodes = (size_t)std::max<int64_t>(1, d->total_nodes);
  bool ok = w.consts.ensure(sizeof(double) * S * std::max(1, P.n_const)) &&
            w.theta.ensure(sizeof(double) * S * std::max(1, P.n_free)) &&
            w.out.ensure(sizeof(double) * S * (1 + P.n_free)) && w.flags.ensure(sizeof(int32_t) * S) &&
            w.tree.ensure(sizeof(double) * std::max<int64_t>(1, d->total_nodes) * 2 * Q) &&
            w.tree_bad.ensure(sizeof(int32_t) * std::max<int64_t>(1, d->total_nodes)) &&
            w.tickets.ensure(sizeof(int32_t) * std::max<int64_t>(1, d->total_nodes)) &&
            w.counter.ensure(sizeof(int32_t)) && w.slow.ensure(sizeof(unsigned long long)) &&
            w.slot_counter.ensure(sizeof(int32_t) * kPassSlots) &&
            w.slot_slow.ensure(sizeof(unsigned long long) * kPassSlots) &&
            (m->m.shape == SHAPE_GENERIC ||
             (w.ffc.ensure(sizeof(float) * S * kFFConst) &&
              w.part_m.ensure(sizeof(float) * nodes * kMaxParts * kPartFloats) &&
              w.part_fb.ensure(sizeof(double) * nodes * kMaxParts * Q) &&
              w.part_info.ensure(sizeof(int32_t) * nodes * kMaxParts))) &&
            w.h_theta.ensure(sizeof(double) * S * std::max(1, P.n_free)) &&
            w.h_out.ensure(sizeof(double) * S * (1 + P.n_free)) && w.h_flags.ensure(sizeof(int32_t) * S);
  if (!ok) return false;
  if (!cuda_ok(cudaMemset(w.tickets.p, 0, sizeof(int32_t) * std::max<int64_t>(1, d->total_nodes)), "ticket reset"))
    return false;
  if (!d->all_plan_ready) {
    std::vector<int32_t> all(d->n_sets);
    for (int s = 0; s < d->n_sets; ++s) all[s] = s;
    if (!build_plan(d, all, &d->all_plan)) return false;
    d->all_plan_ready = true;
  }
  w.n_const = P.n_const;
  w.n_free = P.n_free;
  w.Q = Q;
  w.ready = true;
  return true;
}

Pass make_pass(const rf_model* m, rf_data* d, const Plan& plan, const double* d_theta, double* d_out,
               int32_t* d_flags, bool grad) {
  Workspace& w = d->ws;
  Pass p{};
  p.offsets = (const int64_t*)d->offsets_dev.p;
  p.sets = (const int32_t*)plan.sets.p;
  p.n_active = plan.n_active;
  p.items = (const int2*)plan.items.p;
  p.n_items = plan.n_items;
  p.tree_base = (const int64_t*)d->tree_base_dev.p;
  p.theta = d_theta;
  p.consts = (double*)w.consts.p;
  p.tree = (double*)w.tree.p;
  p.tree_bad = (int32_t*)w.tree_bad.p;
  p.tickets = (int32_t*)w.tickets.p;
  p.counter = (int32_t*)w.counter.p;
  p.slow = (unsigned long long*)w.slow.p;
  p.out = d_out;
  p.flags = d_flags;
  p.Q = grad ? 1 + m->m.prog.n_slots : 1;
  p.want_grad = grad ? 1 : 0;
  p.ff_shape = m->m.shape;
  p.ffc = m->m.shape == SHAPE_GENERIC ? nullptr : (float*)w.ffc.p;
  p.part_m = (float*)w.part_m.p;
  p.part_fb = (double*)w.part_fb.p;
  p.part_info = (int32_t*)w.part_info.p;
  p.parts = parts_for(d->total_chunks, m->m.shape);
  p.pairs = nullptr;
  return p;
}

Columns make_columns(const rf_data* d) {
  Columns c{};
  for (int i = 0; i < d->n_obs; ++i) {
    c.ptr[i] = d->cols[i];
    c.is_f32[i] = d->dtype[i] == RF_F32;
  }
  return c;
}

bool launch_pass(const rf_model* m, rf_data* d, const Plan& plan, const double* d_theta, double* d_out,
                 int32_t* d_flags, bool grad, cudaStream_t st, int slot, const int32_t* dyn) {
  Pass pass = make_pass(m, d, plan, d_theta, d_out, d_flags, grad);
  pass.dyn = dyn;
  if (slot >= 0 && slot < kPassSlots) {
    pass.counter = (int32_t*)d->ws.slot_counter.p + slot;
    pass.slow = (unsigned long long*)d->ws.slot_slow.p + slot;
  }
  launch_param_point(m->m.prog, pass, st);
  launch_events(m->m.prog, m->m.shape, make_columns(d), pass, m->m.threads_per_block, m->m.blocks_per_sm,
                sm_count(), st);
  return cuda_ok(cudaGetLastError(), "kernel launch");
}

// Host-buffer evaluation of the sets in `plan` (theta/out indexed by set).
rf_status finish_host(const rf_model* m, rf_data* d, const Plan& plan, double* nll, double* grad, cudaStream_t st);

rf_status eval_host(const rf_model* m, rf_data* d, const Plan& plan, const double* theta, double* nll,
                    double* grad, cudaStream_t st) {
  if (!ensure_workspace(m, d)) return RF_E_OOM;
  Workspace& w = d->ws;
  const int P = m->m.prog.n_free, S = d->n_sets;
  std::memcpy(w.h_theta.p, theta, sizeof(double) * S * P);
  if (P > 0 && !cuda_ok(cudaMemcpyAsync(w.theta.p, w.h_theta.p, sizeof(double) * S * P, cudaMemcpyHostToDevice, st), "theta upload"))
    return RF_E_CUDA;
  if (!launch_pass(m, d, plan, (const double*)w.theta.p, (double*)w.out.p, (int32_t*)w.flags.p, grad != nullptr, st))
    return RF_E_CUDA;
  return finish_host(m, d, plan, nll, grad, st);
}

// Downloads a pass's results (issued on st), waits, and fills nll / grad.
rf_status finish_host(const rf_model* m, rf_data* d, const Plan& plan, double* nll, double* grad, cudaStream_t st) {
  Workspace& w = d->ws;
  const int P = m->m.prog.n_free, S = d->n_sets;
  if (!cuda_ok(cudaMemcpyAsync(w.h_out.p, w.out.p, sizeof(double) * S * (1 + P), cudaMemcpyDeviceToHost, st), "result download") ||
      !cuda_ok(cudaMemcpyAsync(w.h_flags.p, w.flags.p, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, st), "flag download") ||
      !cuda_ok(cudaStreamSynchronize(st), "stream sync"))
    return RF_E_CUDA;
  const double* o = (const double*)w.h_out.p;
  const int32_t* f = (const int32_t*)w.h_flags.p;
  rf_status st_out = RF_OK;
  for (int s : plan.host_sets) {
    nll[s] = o[(size_t)s * (1 + P)];
    if (grad)
      for (int k = 0; k < P; ++k) grad[(size_t)s * P + k] = o[(size_t)s * (1 + P) + 1 + k];
    if (f[s] != 0) st_out = RF_E_DOMAIN;
  }
  if (st_out == RF_E_DOMAIN) set_error("pdf <= 0 or not finite for some event, or parameters outside a pdf's domain");
  return st_out;
}

}  // namespace rf

using namespace rf;

extern "C" {

const char* rf_last_error(void) { return g_error.c_str(); }
const char* rf_version(void) { return "rfgpu 0.1 (sm_103a)"; }

rf_status rf_model_create(const rf_node* nodes, int32_t n, int32_t root, rf_model** out) {
  if (!out) { set_error("rf_model_create: out is NULL"); return RF_E_INVALID; }
  *out = nullptr;
  rf_model* m = new (std::nothrow) rf_model();
  if (!m) return RF_E_OOM;
  const rf_status s = compile_model(nodes, n, root, &m->m);
  if (s != RF_OK) { delete m; return s; }
  *out = m;
  return RF_OK;
}

rf_status rf_model_create_expr(const rf_node* nodes, int32_t n, int32_t root, const rf_expr* exprs,
                               int32_t n_exprs, rf_model** out) {
  if (!out || n_exprs < 0 || (n_exprs > 0 && !exprs)) { set_error("rf_model_create_expr: bad argument"); return RF_E_INVALID; }
  *out = nullptr;
  rf_model* m = new (std::nothrow) rf_model();
  if (!m) return RF_E_OOM;
  const rf_status s = compile_model(nodes, n, root, &m->m, exprs, n_exprs);
  if (s != RF_OK) { delete m; return s; }
  *out = m;
  return RF_OK;
}

void rf_model_destroy(rf_model* m) { delete m; }
int32_t rf_model_n_free(const rf_model* m) { return m ? m->m.prog.n_free : 0; }
int32_t rf_model_n_obs(const rf_model* m) { return m ? m->m.prog.n_obs : 0; }

rf_status rf_model_describe(const rf_model* m, char* buf, int32_t cap) {
  if (!m || !buf || cap <= 0) { set_error("rf_model_describe: bad argument"); return RF_E_INVALID; }
  static const char* shapes[] = {"generic_fp64", "ff_sum_gauss_poly1", "ff_sum_gaussexp_cheb2", "ff_prod3"};
  std::snprintf(buf, cap, "%s kernel=%s pdf_nodes=%d free=%d slots=%d consts=%d", m->m.signature.c_str(),
                shapes[m->m.shape], m->m.prog.n_pdf, m->m.prog.n_free, m->m.prog.n_slots, m->m.prog.n_const);
  return RF_OK;
}

rf_status rf_model_set_fp64(rf_model* m, int32_t on) {
  if (!m || (on != 0 && on != 1)) { set_error("rf_model_set_fp64: bad argument"); return RF_E_INVALID; }
  m->m.shape = on ? SHAPE_GENERIC : m->m.detected_shape;
  return RF_OK;
}

rf_status rf_set_launch(rf_model* m, int32_t threads_per_block, int32_t blocks_per_sm) {
  if (!m) { set_error("rf_set_launch: model is NULL"); return RF_E_INVALID; }
  if (threads_per_block != 0 && threads_per_block != kLanes) {
    set_error("rf_set_launch: threads_per_block must be 0 or 128 (the reduction's fixed lane-to-event map)");
    return RF_E_INVALID;
  }
  if (blocks_per_sm < 0 || blocks_per_sm > 32) { set_error("rf_set_launch: blocks_per_sm must be 0..32"); return RF_E_INVALID; }
  m->m.threads_per_block = threads_per_block;
  m->m.blocks_per_sm = blocks_per_sm;
  return RF_OK;
}

rf_status rf_data_upload(const rf_model* m, const void* const* cols, const int32_t* dtype, int64_t n_events,
                         const int64_t* offsets, int32_t n_sets, int32_t cols_on_device, rf_data** out) {
  if (!m || !out || n_events < 0 || n_sets < 1 || (n_events > 0 && !cols)) {
    set_error("rf_data_upload: bad argument");
    return RF_E_INVALID;
  }
  *out = nullptr;
  const int nobs = m->m.prog.n_obs;
  std::vector<int64_t> off(n_sets + 1);
  if (offsets) {
    off.assign(offsets, offsets + n_sets + 1);
    if (off[0] != 0 || off[n_sets] != n_events) { set_error("rf_data_upload: offsets must run from 0 to n_events"); return RF_E_INVALID; }
    for (int s = 0; s < n_sets; ++s)
      if (off[s + 1] < off[s]) { set_error("rf_data_upload: offsets must not decrease"); return RF_E_INVALID; }
  } else {
    if (n_sets != 1) { set_error("rf_data_upload: offsets are required for n_sets > 1"); return RF_E_INVALID; }
    off[0] = 0;
    off[1] = n_events;
  }
  for (int s = 0; s < n_sets; ++s)
    if ((off[s + 1] - off[s] + kChunk - 1) / kChunk > (int64_t)0x7fffffff) { set_error("rf_data_upload: set too large"); return RF_E_INVALID; }
  rf_data* d = new (std::nothrow) rf_data();
  if (!d) return RF_E_OOM;
  d->n_obs = nobs;
  d->n_sets = n_sets;
  d->n_events = n_events;
  d->offsets = off;
  d->owns_cols = !cols_on_device;
  for (int c = 0; c < nobs; ++c) {
    d->dtype[c] = dtype ? dtype[c] : RF_F64;
    if (d->dtype[c] != RF_F64 && d->dtype[c] != RF_F32) { delete d; set_error("rf_data_upload: dtype must be RF_F64 or RF_F32"); return RF_E_INVALID; }
    const size_t bytes = (size_t)n_events * (d->dtype[c] == RF_F32 ? 4 : 8);
    if (cols_on_device) {
      d->cols[c] = nullptr;
      if (n_events > 0) {
        // Device or managed memory, or pinned host memory that the GPU reads
        // in place (over the host link; its device address may differ);
        // anything else would fault in the kernel and is refused here.
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, cols[c]) != cudaSuccess) cudaGetLastError();
        if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
          d->cols[c] = const_cast<void*>(cols[c]);
        } else if (a.type == cudaMemoryTypeHost && a.devicePointer) {
          d->cols[c] = a.devicePointer;
        } else {
          delete d;
          set_error("rf_data_upload: borrowed columns must be device, managed or pinned host memory");
          return RF_E_INVALID;
        }
      }
    } else {
      if (!d->col_bufs[c].ensure(bytes)) { delete d; return RF_E_OOM; }
      d->cols[c] = d->col_bufs[c].p;
      if (n_events > 0 && !cuda_ok(cudaMemcpy(d->cols[c], cols[c], bytes, cudaMemcpyHostToDevice), "column upload")) {
        delete d;
        return RF_E_CUDA;
      }
    }
  }
  rf_status st = finish_data(d);
  if (st != RF_OK) { delete d; return st; }
  *out = d;
  return RF_OK;
}

void rf_data_destroy(rf_data* d) { delete d; }
int64_t rf_data_n_events(const rf_data* d) { return d ? d->n_events : 0; }
int32_t rf_data_n_sets(const rf_data* d) { return d ? d->n_sets : 0; }

rf_status rf_data_read(const rf_data* d, int32_t col, int64_t i0, int64_t i1, double* out) {
  if (!d || col < 0 || col >= d->n_obs || i0 < 0 || i1 < i0 || i1 > d->n_events || (i1 > i0 && !out)) {
    set_error("rf_data_read: bad argument");
    return RF_E_INVALID;
  }
  const int64_t n = i1 - i0;
  if (n == 0) return RF_OK;
  if (d->dtype[col] == RF_F32) {
    std::vector<float> tmp(n);
    if (!cuda_ok(cudaMemcpy(tmp.data(), (const float*)d->cols[col] + i0, n * 4, cudaMemcpyDeviceToHost), "column read")) return RF_E_CUDA;
    for (int64_t i = 0; i < n; ++i) out[i] = (double)tmp[i];
  } else {
    if (!cuda_ok(cudaMemcpy(out, (const double*)d->cols[col] + i0, n * 8, cudaMemcpyDeviceToHost), "column read")) return RF_E_CUDA;
  }
  return RF_OK;
}

rf_status rf_data_offsets(const rf_data* d, int64_t* out) {
  if (!d || !out) { set_error("rf_data_offsets: bad argument"); return RF_E_INVALID; }
  std::copy(d->offsets.begin(), d->offsets.end(), out);
  return RF_OK;
}

static rf_status check_eval_args(const rf_model* m, const rf_data* d, const void* theta, const void* nll) {
  if (!m || !d || !nll || (m->m.prog.n_free > 0 && !theta)) { set_error("bad argument (NULL)"); return RF_E_INVALID; }
  if (d->n_obs != m->m.prog.n_obs) { set_error("data and model have different observable counts"); return RF_E_INVALID; }
  return RF_OK;
}

rf_status rf_nll(const rf_model* m, const rf_data* d, const double* theta, double* nll, void* stream) {
  rf_status s = check_eval_args(m, d, theta, nll);
  if (s != RF_OK) return s;
  rf_data* dd = const_cast<rf_data*>(d);
  if (!ensure_workspace(m, dd)) return RF_E_OOM;
  return eval_host(m, dd, dd->all_plan, theta, nll, nullptr, (cudaStream_t)stream);
}

rf_status rf_nll_grad(const rf_model* m, const rf_data* d, const double* theta, double* nll, double* grad,
                      void* stream) {
  rf_status s = check_eval_args(m, d, theta, nll);
  if (s != RF_OK) return s;
  if (!grad && m->m.prog.n_free > 0) { set_error("rf_nll_grad: grad is NULL"); return RF_E_INVALID; }
  rf_data* dd = const_cast<rf_data*>(d);
  if (!ensure_workspace(m, dd)) return RF_E_OOM;
  double dummy;
  return eval_host(m, dd, dd->all_plan, theta, nll, grad ? grad : &dummy, (cudaStream_t)stream);
}

rf_status rf_nll_grad_async(const rf_model* m, const rf_data* d, const double* d_theta, double* d_out,
                            int32_t* d_flags, void* stream) {
  rf_status s = check_eval_args(m, d, d_theta, d_out);
  if (s != RF_OK) return s;
  if (!d_flags) { set_error("rf_nll_grad_async: d_flags is NULL"); return RF_E_INVALID; }
  rf_data* dd = const_cast<rf_data*>(d);
  if (!ensure_workspace(m, dd)) return RF_E_OOM;
  return launch_pass(m, dd, dd->all_plan, d_theta, d_out, d_flags, true, (cudaStream_t)stream) ? RF_OK : RF_E_CUDA;
}

rf_status rf_nll_grad_partial(const rf_model* m, const rf_data* d, const double* d_theta, double* d_pairs,
                              int32_t* d_flags, void* stream) {
  rf_status s = check_eval_args(m, d, d_theta, d_pairs);
  if (s != RF_OK) return s;
  if (!d_flags) { set_error("rf_nll_grad_partial: d_flags is NULL"); return RF_E_INVALID; }
  if (m->m.extended) {
    set_error("rf_nll_grad_partial: an extended model's term depends on the whole dataset's size");
    return RF_E_INVALID;
  }
  rf_data* dd = const_cast<rf_data*>(d);
  if (!ensure_workspace(m, dd)) return RF_E_OOM;
  Pass pass = make_pass(m, dd, dd->all_plan, d_theta, (double*)dd->ws.out.p, d_flags, true);
  pass.pairs = d_pairs;
  const cudaStream_t st = (cudaStream_t)stream;
  launch_param_point(m->m.prog, pass, st);
  launch_events(m->m.prog, m->m.shape, make_columns(dd), pass, m->m.threads_per_block, m->m.blocks_per_sm,
                sm_count(), st);
  return cuda_ok(cudaGetLastError(), "kernel launch") ? RF_OK : RF_E_CUDA;
}

rf_status rf_nll_chunks(const rf_model* m, const rf_data* d, const double* theta, int32_t set, double* out,
                        int32_t max_chunks, int32_t* n_chunks) {
  rf_status s = check_eval_args(m, d, theta, out);
  if (s != RF_OK) return s;
  if (set < 0 || set >= d->n_sets || !n_chunks || max_chunks < 0) { set_error("rf_nll_chunks: bad set"); return RF_E_INVALID; }
  rf_data* dd = const_cast<rf_data*>(d);
  const int P = m->m.prog.n_free, Q = 1 + m->m.prog.n_slots;
  std::vector<double> nll(d->n_sets), grad((size_t)d->n_sets * std::max(1, P));
  s = rf_nll_grad(m, d, theta, nll.data(), grad.data(), nullptr);
  if (s != RF_OK && s != RF_E_DOMAIN) return s;
  const int64_t C = d->chunks[set];
  *n_chunks = (int32_t)C;
  const int64_t n = std::min<int64_t>(C, max_chunks);
  if (n <= 0) return s;
  // Level-0 nodes of the set's tree: (sum, compensation) per quantity, slots
  // mapped to free parameters as the root does.
  std::vector<double> buf((size_t)2 * Q * n);
  const double* tree = (const double*)dd->ws.tree.p;
  if (!cuda_ok(cudaMemcpy(buf.data(), tree + d->tree_base[set] * 2 * Q, sizeof(double) * 2 * Q * n,
                          cudaMemcpyDeviceToHost), "chunk read"))
    return RF_E_CUDA;
  for (int64_t c = 0; c < n; ++c) {
    const double* node = buf.data() + (size_t)2 * Q * c;
    double* o = out + (size_t)c * (1 + P);
    o[0] = node[0] + node[Q];
    for (int k = 0; k < P; ++k) {
      double gk = 0.0;
      for (int sl = 0; sl < m->m.prog.n_slots; ++sl)
        if (m->m.prog.slot_free[sl] == k) gk += node[1 + sl] + node[Q + 1 + sl];
      o[1 + k] = gk;
    }
  }
  return s;
}

}  // extern "C"

namespace rf {

rf_status finish_data(rf_data* d) {
  const int S = d->n_sets;
  d->chunks.resize(S);
  d->tree_base.resize(S);
  int64_t total = 0;
  for (int s = 0; s < S; ++s) {
    const int64_t n = d->offsets[s + 1] - d->offsets[s];
    d->chunks[s] = (n + kChunk - 1) / kChunk;
    d->tree_base[s] = total;
    total += tree_nodes(d->chunks[s]);
  }
  d->total_nodes = total;
  d->total_chunks = 0;
  for (int s = 0; s < S; ++s) d->total_chunks += d->chunks[s];
  if (!d->offsets_dev.ensure(sizeof(int64_t) * (S + 1)) || !d->tree_base_dev.ensure(sizeof(int64_t) * S)) return RF_E_OOM;
  if (!cuda_ok(cudaMemcpy(d->offsets_dev.p, d->offsets.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice), "offsets upload") ||
      !cuda_ok(cudaMemcpy(d->tree_base_dev.p, d->tree_base.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice), "tree upload"))
    return RF_E_CUDA;
  return RF_OK;
}

}  // namespace rf

extern "C" rf_status rf_autotune_scan(rf_model* m, rf_data* d, int32_t passes, int32_t cap, int32_t* blocks_per_sm,
                                      double* ms_out, int32_t* n) {
  if (!m || !d || passes < 1 || cap < 1 || !blocks_per_sm || !ms_out || !n) {
    set_error("rf_autotune: bad argument");
    return RF_E_INVALID;
  }
  *n = 0;
  if (d->n_obs != m->m.prog.n_obs) {
    set_error("rf_autotune: data and model have different observable counts");
    return RF_E_INVALID;
  }
  if (!ensure_workspace(m, d)) return RF_E_OOM;
  Workspace& w = d->ws;
  const int P = m->m.prog.n_free, S = d->n_sets;
  std::vector<double> th((size_t)S * std::max(1, P));
  for (int s = 0; s < S; ++s)
    for (int k = 0; k < P; ++k) th[(size_t)s * P + k] = m->m.theta_default[k];
  if (P > 0 && !cuda_ok(cudaMemcpy(w.theta.p, th.data(), sizeof(double) * S * P, cudaMemcpyHostToDevice), "autotune"))
    return RF_E_CUDA;
  cudaEvent_t e0, e1;
  if (!cuda_ok(cudaEventCreate(&e0), "autotune") || !cuda_ok(cudaEventCreate(&e1), "autotune")) return RF_E_CUDA;
  static const int kBps[] = {1, 2, 3, 4, 5, 6, 7, 8, 12, 16};
  const int save_b = m->m.blocks_per_sm;
  double best = 1e300;
  int bb = 0;
  for (int b : kBps) {
    if (!launch_fits(m->m.shape, kLanes, b) || *n >= cap) continue;
    m->m.threads_per_block = kLanes;
    m->m.blocks_per_sm = b;
    launch_pass(m, d, d->all_plan, (const double*)w.theta.p, (double*)w.out.p, (int32_t*)w.flags.p, true, 0);
    cudaEventRecord(e0, 0);
    for (int i = 0; i < passes; ++i)
      launch_pass(m, d, d->all_plan, (const double*)w.theta.p, (double*)w.out.p, (int32_t*)w.flags.p, true, 0);
    cudaEventRecord(e1, 0);
    if (!cuda_ok(cudaEventSynchronize(e1), "autotune")) {
      m->m.blocks_per_sm = save_b;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return RF_E_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    blocks_per_sm[*n] = b;
    ms_out[*n] = ms / passes;
    ++*n;
    if (ms / passes < best) {
      best = ms / passes;
      bb = b;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->m.threads_per_block = kLanes;
  m->m.blocks_per_sm = bb;
  return RF_OK;
}

extern "C" rf_status rf_autotune(rf_model* m, rf_data* d, int32_t passes, int32_t* threads_per_block,
                                 int32_t* blocks_per_sm, double* best_ms) {
  if (!threads_per_block || !blocks_per_sm || !best_ms) {
    set_error("rf_autotune: bad argument");
    return RF_E_INVALID;
  }
  int32_t bps[16], n = 0;
  double ms[16];
  const rf_status s = rf_autotune_scan(m, d, passes, 16, bps, ms, &n);
  if (s != RF_OK) return s;
  int best = 0;
  for (int i = 1; i < n; ++i)
    if (ms[i] < ms[best]) best = i;
  *threads_per_block = kLanes;
  *blocks_per_sm = n > 0 ? bps[best] : 0;
  *best_ms = n > 0 ? ms[best] : 0.0;
  return RF_OK;
}

namespace rf {

// Event range [first, last) of work items [i0, i1) of the all-sets plan
// (items run set by set, chunk by chunk, over back-to-back sets).
static void item_events(const rf_data* d, int64_t i0, int64_t i1, int64_t* first, int64_t* last) {
  int64_t it = 0;
  *first = *last = -1;
  for (int s = 0; s < d->n_sets && it < i1; ++s) {
    const int64_t c = d->chunks[s];
    if (it + c > i0) {
      const int64_t k0 = std::max<int64_t>(i0 - it, 0), k1 = std::min<int64_t>(i1 - it, c);
      const int64_t e0 = d->offsets[s] + k0 * kChunk, e1 = std::min(d->offsets[s] + k1 * kChunk, d->offsets[s + 1]);
      if (*first < 0) *first = e0;
      *last = e1;
    }
    it += c;
  }
  if (*first < 0) *first = *last = 0;
}

}  // namespace rf

extern "C" rf_status rf_nll_grad_stream(const rf_model* m, rf_data* d, const void* const* host_cols,
                                        const double* theta, double* nll, double* grad, void* stream) {
  rf_status s = check_eval_args(m, d, theta, nll);
  if (s != RF_OK) return s;
  if (!grad || !host_cols || !d->owns_cols) {
    set_error("rf_nll_grad_stream: bad argument or a dataset with borrowed columns");
    return RF_E_INVALID;
  }
  if (!ensure_workspace(m, d)) return RF_E_OOM;
  Workspace& w = d->ws;
  const cudaStream_t st = (cudaStream_t)stream;
  if (!w.copy_stream) {
    bool ok = cuda_ok(cudaStreamCreateWithFlags(&w.copy_stream, cudaStreamNonBlocking), "rf_nll_grad_stream");
    for (cudaStream_t& c : w.comp_stream)
      ok = ok && cuda_ok(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking), "rf_nll_grad_stream");
    for (cudaEvent_t& e : w.seg_ev)
      ok = ok && cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "rf_nll_grad_stream");
    for (cudaEvent_t& e : w.comp_ev)
      ok = ok && cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "rf_nll_grad_stream");
    if (!ok) return RF_E_CUDA;
  }
  if (!w.seg_counters.ensure(sizeof(int32_t) * kMaxSegments)) return RF_E_OOM;
  const Plan& plan = d->all_plan;
  const int P = m->m.prog.n_free, S = d->n_sets;
  // Up to 8 segments of >= 128 chunks (512 Ki events); the last two are a
  // half and a quarter of the others, so the pass left after the last copy
  // is short.
  const int64_t n_items = plan.n_items;
  const int K = (int)std::max<int64_t>(1, std::min<int64_t>(8, n_items / 128));
  int64_t bound[kMaxSegments + 1];
  {
    int64_t wsum = 0, wc[kMaxSegments + 1];
    wc[0] = 0;
    for (int k = 0; k < K; ++k) wc[k + 1] = (wsum += (K >= 3 && k == K - 1) ? 1 : (K >= 3 && k == K - 2) ? 2 : 4);
    for (int k = 0; k <= K; ++k) bound[k] = n_items * wc[k] / wsum;
  }
  // The copy stream starts after everything already queued on `stream` (a
  // previous pass may still read the columns), alongside the theta upload;
  // then K1 on `stream`; the compute streams start after K1.
  cudaEvent_t ev_start = w.seg_ev[kMaxSegments], ev_k1 = w.seg_ev[kMaxSegments + 1];
  if (!cuda_ok(cudaEventRecord(ev_start, st), "rf_nll_grad_stream") ||
      !cuda_ok(cudaStreamWaitEvent(w.copy_stream, ev_start, 0), "rf_nll_grad_stream"))
    return RF_E_CUDA;
  std::memcpy(w.h_theta.p, theta, sizeof(double) * S * P);
  if (P > 0 && !cuda_ok(cudaMemcpyAsync(w.theta.p, w.h_theta.p, sizeof(double) * S * P, cudaMemcpyHostToDevice, st),
                        "theta upload"))
    return RF_E_CUDA;
  Pass pass = make_pass(m, d, plan, (const double*)w.theta.p, (double*)w.out.p, (int32_t*)w.flags.p, true);
  pass.counter = (int32_t*)w.seg_counters.p;
  pass.n_counters = K;
  launch_param_point(m->m.prog, pass, st);
  if (!cuda_ok(cudaEventRecord(ev_k1, st), "rf_nll_grad_stream")) return RF_E_CUDA;
  const int n_comp = std::min(K, kCompStreams);
  for (int j = 0; j < n_comp; ++j)
    if (!cuda_ok(cudaStreamWaitEvent(w.comp_stream[j], ev_k1, 0), "rf_nll_grad_stream")) return RF_E_CUDA;
  const Columns cols = make_columns(d);
  for (int k = 0; k < K; ++k) {
    const int64_t i0 = bound[k], i1 = bound[k + 1];
    int64_t e0, e1;
    item_events(d, i0, i1, &e0, &e1);
    if (k == 0) e0 = 0;                 // events before the first item: none, but copy from 0
    if (k == K - 1) e1 = d->n_events;   // and to the end
    for (int c = 0; c < d->n_obs; ++c) {
      const size_t es = d->dtype[c] == RF_F32 ? 4 : 8;
      if (e1 > e0 &&
          !cuda_ok(cudaMemcpyAsync((char*)d->cols[c] + e0 * es, (const char*)host_cols[c] + e0 * es, (e1 - e0) * es,
                                   cudaMemcpyHostToDevice, w.copy_stream),
                   "rf_nll_grad_stream copy"))
        return RF_E_CUDA;
    }
    const cudaStream_t cs = w.comp_stream[k % n_comp];
    if (!cuda_ok(cudaEventRecord(w.seg_ev[k], w.copy_stream), "rf_nll_grad_stream") ||
        !cuda_ok(cudaStreamWaitEvent(cs, w.seg_ev[k], 0), "rf_nll_grad_stream"))
      return RF_E_CUDA;
    Pass seg = pass;
    seg.items = (const int2*)plan.items.p + i0;
    seg.n_items = (int32_t)(i1 - i0);
    seg.counter = pass.counter + k;
    launch_events(m->m.prog, m->m.shape, cols, seg, m->m.threads_per_block, m->m.blocks_per_sm, sm_count(), cs);
  }
  // `stream` waits for every compute stream, then downloads the results.
  for (int j = 0; j < n_comp; ++j)
    if (!cuda_ok(cudaEventRecord(w.comp_ev[j], w.comp_stream[j]), "rf_nll_grad_stream") ||
        !cuda_ok(cudaStreamWaitEvent(st, w.comp_ev[j], 0), "rf_nll_grad_stream"))
      return RF_E_CUDA;
  if (!cuda_ok(cudaGetLastError(), "kernel launch")) return RF_E_CUDA;
  return finish_host(m, d, plan, nll, grad, st);
}

extern "C" rf_status rf_launch_count(int64_t* n) {
  if (!n) {
    set_error("rf_launch_count: NULL output");
    return RF_E_INVALID;
  }
  *n = g_launches.load(std::memory_order_relaxed);
  return RF_OK;
}
