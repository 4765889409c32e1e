// Host-side handle layouts shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "rf_internal.h"

namespace rf {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf();
  bool ensure(size_t b);
  void release();
};

struct HostBuf {
  void* p = nullptr;
  size_t bytes = 0;
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf();
  bool ensure(size_t b);
};

// Active sets and their (set, chunk) work items.
struct Plan {
  DevBuf sets, items;
  std::vector<int32_t> host_sets;
  int32_t n_active = 0, n_items = 0;
};

// Per-dataset evaluation buffers for the model last used with it.
// Segments of the streamed host-column pass (rf_nll_grad_stream).
constexpr int kMaxSegments = 16;
// Compute streams the segments rotate over, so that one segment's pass
// starts while the previous one finishes its last work units.
constexpr int kCompStreams = 4;

struct Workspace {
  bool ready = false;
  int n_const = -1, n_free = -1, Q = -1;
  DevBuf consts, theta, out, flags, tree, tree_bad, tickets, counter, slow, ffc, part_m, part_fb, part_info;
  // work and slow-event counters of passes that may run concurrently on
  // other streams (launch_pass with slot >= 0)
  DevBuf slot_counter, slot_slow;
  HostBuf h_theta, h_out, h_flags;
  // rf_nll_grad_stream: its copy stream, compute streams and events
  // (created on first use)
  cudaStream_t copy_stream = nullptr;
  cudaStream_t comp_stream[kCompStreams] = {};
  cudaEvent_t seg_ev[kMaxSegments + 2] = {};
  cudaEvent_t comp_ev[kCompStreams] = {};
  DevBuf seg_counters;
  Workspace() = default;
  Workspace(const Workspace&) = delete;
  Workspace& operator=(const Workspace&) = delete;
  ~Workspace();
};

bool cuda_ok(cudaError_t e, const char* what);

// The batched BFGS fit driver (fit.cpp): S independent problems of P
// parameters, bounds lo/hi (lo >= hi: unbounded), start S x P.  Each round
// evaluates all active problems' trial points with one call of `eval`
// (active set indices; theta S x P in; nll S and gradient S x P out, all
// indexed by set).  cov (S x P x P) may be null.
using BatchEval = std::function<rf_status(const std::vector<int32_t>&, std::vector<double>&, std::vector<double>&,
                                          std::vector<double>&)>;
// Optional split evaluation for pipelined rounds: the sets [0, split) and
// [split, S) are evaluated as separate passes, launch queueing one and wait
// finishing it, so the host updates one half while the other is evaluated;
// events(sets) counts events, and fit_batch returns to whole-batch rounds
// once the active events fall below min_events.
struct SplitEval {
  int64_t split = 0, min_events = 0;
  std::function<rf_status(int, const std::vector<int32_t>&, const std::vector<double>&)> launch;
  std::function<rf_status(int, std::vector<double>&, std::vector<double>&)> wait;
  std::function<int64_t(const std::vector<int32_t>&)> events;
};
// Below this many active events a pass is short enough that the launch
// latency of two half passes costs more than the host work they hide.
constexpr int64_t kPipelineMinEvents = int64_t(1) << 21;
// Device-resident rounds for the end of a fit (fit.cpp): the evaluator of
// the fit's dataset and, for a fit of some sets only, problem -> set.
struct DeviceSteps;
rf_status fit_batch(int S, int P, const double* lo, const double* hi, const double* start, double tol, int max_evals,
                    bool want_cov, const BatchEval& eval, const SplitEval* split, double* theta_hat,
                    double* nll_min, double* cov, int32_t* n_evals, int32_t* fit_status,
                    DeviceSteps* dev = nullptr);

// One quasi-Newton step per listed set on the device (fit_dev.cu), a warp
// per set: set i (record i of `state`, of qn::tail_record_words(P) doubles;
// dataset set set_of[i], with chunks[i] chunks) takes the pass's result
// out[set] (nll, gradient in theta), advances its state machine and, unless
// done, writes its next trial point to theta[set]; phase[i] gets its phase.
// The last block to finish then compacts the plan of the next pass: the
// sets still going (increasing) into plan_sets, their (set, chunk) items
// into plan_items, the counts into dyn = {sets, items}.  Skipped when dyn reads no active set.  ticket: a counter
// at zero, left at zero.
struct FitStepArgs {
  double* state;
  const int32_t* set_of;
  const int32_t* chunks;
  int32_t n, P;
  const double* out;
  double* theta;
  const double *lo, *hi;
  const char* bounded;
  double tol;
  int32_t max_evals;
  int32_t* phase;
  int32_t* plan_sets;
  int2* plan_items;
  int32_t* dyn;
  int32_t* ticket;
};
void launch_fit_step(const FitStepArgs& a, cudaStream_t st);
int sm_count();
// Counts n kernel launches on st for rf_launch_count (not while st is being
// captured into a graph).
void note_launches(int n, cudaStream_t st);
int64_t tree_nodes(int64_t chunks);

}  // namespace rf

struct rf_model {
  rf::Model m;
};

struct rf_data {
  int n_obs = 0, n_sets = 0;
  int64_t n_events = 0;
  void* cols[rf::kMaxObs] = {};
  int32_t dtype[rf::kMaxObs] = {};
  rf::DevBuf col_bufs[rf::kMaxObs];
  bool owns_cols = true;
  std::vector<int64_t> offsets, chunks, tree_base;
  int64_t total_nodes = 0;
  int64_t total_chunks = 0;  // over all sets (parts_for)
  rf::DevBuf offsets_dev, tree_base_dev;
  rf::Workspace ws;
  rf::Plan all_plan;
  bool all_plan_ready = false;
};

namespace rf {
rf_status finish_data(rf_data* d);
bool build_plan(const rf_data* d, const std::vector<int32_t>& sets, Plan* plan);
bool ensure_workspace(const rf_model* m, rf_data* d);
// Queues K1 and the event kernel for the plan's sets.  slot >= 0 (below
// kPassSlots) gives the pass its own work and slow-event counters, for
// passes over disjoint sets that run at the same time on different streams.
constexpr int kPassSlots = 4;
// dyn: null, or device counts {active sets, work items} that replace the
// plan's (whose sets and items buffers then hold the device-compacted plan
// of a device-resident fit); no active set skips the pass.
bool launch_pass(const rf_model* m, rf_data* d, const Plan& plan, const double* d_theta, double* d_out,
                 int32_t* d_flags, bool grad, cudaStream_t st, int slot = -1, const int32_t* dyn = nullptr);
rf_status eval_host(const rf_model* m, rf_data* d, const Plan& plan, const double* theta, double* nll,
                    double* grad, cudaStream_t st);
}  // namespace rf
