// Maximum-likelihood fits (paper Sec. 1: "compute likelihoods and perform
// fits to data"; Sec. 3: fits converge faster when the likelihood is faster).
//
// The paper does not describe its minimiser.  Each set is fitted by BFGS
// with a strong-Wolfe line search over internal coordinates (the state
// machine in fit_step.h, shared with the device step); a fit stops when
// EDM = g^T H g / 2 < tol_edm.  The covariance is the inverse of the NLL's
// Hessian in theta, by central differences of the analytic gradient (an NLL
// has "up" = 1/2, so cov = Hessian^-1).
//
// Every set of a dataset is fitted by its own state machine; each round asks
// every active set for one trial point and evaluates all of them in a single
// device pass (the batched toy fit), so a round costs one pass whatever the
// number of sets.  Once few events remain active, the rounds run on the
// device: the pass and every set's step (fit_step_kernel) are replayed as one
// CUDA graph of several rounds, without a host round trip between them.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <limits>
#include <mutex>
#include <thread>
#include <vector>

#include "api_internal.h"
#include "fit_step.h"

namespace rf {

namespace {

const double kInf = std::numeric_limits<double>::infinity();
// Rounds per graph launch of the device-resident rounds: a host round trip
// per kDeviceRounds rounds, and at most kDeviceRounds - 1 skipped rounds
// (a launch and a flag read each) after the last set is done.
constexpr int kDeviceRounds = 8;
// A batched fit hands its rounds to the device once fewer than this many
// events are still being fitted (the pipelined halves stop there).
constexpr int64_t kDeviceRoundEvents = int64_t(1) << 23;

struct Coords {
  int P;
  std::vector<double> lo, hi;
  std::vector<char> bounded;
  void to_theta(const double* x, double* th) const {
    qn::to_theta_jac(P, lo.data(), hi.data(), bounded.data(), x, th, nullptr);
  }
  void to_internal(const double* th, double* x) const {
    for (int k = 0; k < P; ++k) {
      if (!bounded[k]) {
        x[k] = th[k];
        continue;
      }
      const double r = std::min(1.0, std::max(-1.0, 2.0 * (th[k] - lo[k]) / (hi[k] - lo[k]) - 1.0));
      x[k] = std::asin(r);
    }
  }
  // d theta / d x
  double jac(int k, double xk) const {
    if (!bounded[k]) return 1.0;
    double sn, cs;
    qn::sin_cos(xk, &sn, &cs);
    return (hi[k] - lo[k]) * 0.5 * cs;
  }
  // theta and d theta / d x at x
  void to_theta_jac(const double* x, double* th, double* jc) const {
    qn::to_theta_jac(P, lo.data(), hi.data(), bounded.data(), x, th, jc);
  }
};

// A fixed set of worker threads for the per-set host work of a round (the
// sets' state machines are independent, so the split does not change any
// result).  run(n, f) calls f(i) for i in [0, n) on the caller and the
// workers, chunk by chunk, and returns when all are done.
class Pool {
 public:
  explicit Pool(int threads) {
    for (int t = 1; t < threads; ++t) workers_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (std::thread& t : workers_) t.join();
  }
  int size() const { return 1 + (int)workers_.size(); }
  // min_n: the smallest n worth splitting (the dispatch costs ~10 us)
  void run(int64_t n, const std::function<void(int64_t)>& f, int64_t min_n = 1024) {
    if (workers_.empty() || n < min_n) {
      for (int64_t i = 0; i < n; ++i) f(i);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &f;
      n_ = n;
      chunk_ = std::max<int64_t>(1, std::min<int64_t>(64, n / (4 * size())));
      next_.store(0);
      busy_ = (int)workers_.size();
      ++gen_;
    }
    cv_.notify_all();
    work(f, n);
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [this] { return busy_ == 0; });
    job_ = nullptr;
  }

 private:
  int64_t chunk_ = 64;
  void work(const std::function<void(int64_t)>& f, int64_t n) {
    while (true) {
      const int64_t i0 = next_.fetch_add(chunk_);
      if (i0 >= n) return;
      const int64_t i1 = std::min(n, i0 + chunk_);
      for (int64_t i = i0; i < i1; ++i) f(i);
    }
  }
  void loop() {
    uint64_t seen = 0;
    while (true) {
      const std::function<void(int64_t)>* f;
      int64_t n;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        f = job_;
        n = n_;
      }
      work(*f, n);
      std::lock_guard<std::mutex> lk(mu_);
      if (--busy_ == 0) done_cv_.notify_one();
    }
  }
  std::vector<std::thread> workers_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int64_t)>* job_ = nullptr;
  int64_t n_ = 0;
  std::atomic<int64_t> next_{0};
  int busy_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

int pool_threads() {
  const unsigned hc = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(8u, hc / 2));
}

double dot(const double* a, const double* b, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

// One set's fit: the shared state machine and its vectors.
struct SetFit {
  int P = 0;
  qn::State c = qn::initial_state();
  std::vector<double> x, g, H, p, g_lo, trial, w_s, w_y, w_hy, w_r, w_ga;
  void init(int n) {
    P = n;
    for (std::vector<double>* v : {&x, &g, &p, &g_lo, &trial, &w_s, &w_y, &w_hy, &w_r, &w_ga}) v->assign(n, 0.0);
    H.assign((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) H[(size_t)k * n + k] = 1.0;
    c = qn::initial_state();
  }
  qn::Vecs vecs() {
    return {x.data(), g.data(), H.data(), p.data(), g_lo.data(), trial.data(),
            w_s.data(), w_y.data(), w_hy.data(), w_r.data()};
  }
  bool done() const { return c.phase == qn::DONE; }
  // Deliver f and the gradient (internal) at the last trial point.
  void deliver(double fa, const double* ga, double tol, int max_evals) {
    qn::deliver<qn::SeqLoop>(P, c, vecs(), fa, ga, tol, max_evals);
  }
};

// Gauss-Jordan inverse with partial pivoting; false if singular.
bool invert(std::vector<double> A, int n, double* inv) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0 || !std::isfinite(A[piv * n + c])) return false;
    for (int k = 0; k < n; ++k) {
      std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(I[c * n + k], I[piv * n + k]);
    }
    const double d = A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] /= d;
      I[c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double fct = A[r * n + c];
      if (fct == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= fct * A[c * n + k];
        I[r * n + k] -= fct * I[c * n + k];
      }
    }
  }
  std::copy(I.begin(), I.end(), inv);
  return true;
}

}  // namespace

// Device passes over active sets at their trial points (theta), results
// into nll/grad (indexed by set).  A pass (parameter upload, the two
// kernels, result download) is captured once per work plan as a CUDA graph
// and replayed.  A plan covers a superset of the active sets and is rebuilt
// only when the events of still-active sets fall below 15/16 of the planned
// events (finished sets are re-evaluated at their last point and their
// results ignored) or a set outside the plan becomes active.  Groups 0 and 1
// serve the two halves of a pipelined fit (launch, then wait: while one
// half's pass runs, the host updates the other half), group 2 whole-batch
// passes (run).  The halves run on streams of their own with their own work
// counters (their sets, constants, trees and result ranges are disjoint), so
// one half's parameter point and the start of its event pass overlap the
// end of the other half's event pass; group 2 shares group 0's stream and
// runs only when neither half has a pass in flight.  Only the planned sets'
// range of theta and results is copied.
struct Evaluator {
  struct Group {
    Plan plan;
    std::vector<int32_t> planned;
    int64_t planned_events = 0;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
  };
  const rf_model* m;
  rf_data* d;
  cudaStream_t streams[2] = {nullptr, nullptr};
  bool use_graph = true;
  Group grp[4];  // 0, 1: the halves; 2: whole-batch passes; 3: device-resident rounds
  // device-resident rounds: the sets' records, their dataset sets, chunk
  // counts and phases, the plan counts {sets, items} and the step's ticket,
  // the bounds (lo, hi, bounded), the plan the step compacts, the graph and
  // the plan size it was captured for
  DevBuf r_state, r_sets, r_chunks, r_phase, r_dyn, r_bounds;
  HostBuf h_phase;
  Plan r_plan;
  cudaGraphExec_t r_exec = nullptr;
  int32_t r_cap_sets = 0, r_cap_items = 0;

  Evaluator(const rf_model* mm, rf_data* dd, bool graph) : m(mm), d(dd), use_graph(graph) {}
  ~Evaluator() {
    for (cudaStream_t s : streams)
      if (s) cudaStreamSynchronize(s);
    for (Group& G : grp) {
      if (G.exec) cudaGraphExecDestroy(G.exec);
      if (G.done) cudaEventDestroy(G.done);
    }
    if (r_exec) cudaGraphExecDestroy(r_exec);
    for (cudaStream_t s : streams)
      if (s) cudaStreamDestroy(s);
  }

  static int stream_of(int g) { return g == 1 ? 1 : 0; }

  int64_t events_of(const std::vector<int32_t>& sets) const {
    int64_t n = 0;
    for (int32_t s : sets) n += d->offsets[s + 1] - d->offsets[s];
    return n;
  }

  // Keeps or rebuilds G's plan for `active`; *rebuilt tells which.
  bool replan(Group& G, const std::vector<int32_t>& active, bool* rebuilt) {
    bool covered = !G.planned.empty();
    if (covered) {
      size_t j = 0;  // active and planned are both increasing
      for (int32_t s : active) {
        while (j < G.planned.size() && G.planned[j] < s) ++j;
        if (j == G.planned.size() || G.planned[j] != s) {
          covered = false;
          break;
        }
      }
    }
    const int64_t need = events_of(active);
    *rebuilt = !covered || 16 * need < 15 * G.planned_events;
    if (*rebuilt) {
      if (!build_plan(d, active, &G.plan)) return false;
      G.planned = active;
      G.planned_events = need;
    }
    return true;
  }

  rf_status capture(int g) {
    Group& G = grp[g];
    cudaStream_t st = streams[stream_of(g)];
    if (G.exec) {
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
    Workspace& w = d->ws;
    const int P = m->m.prog.n_free;
    const size_t s0 = G.planned.front(), ns = (size_t)G.planned.back() + 1 - s0;
    cudaGraph_t graph = nullptr;
    if (!cuda_ok(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "graph capture")) return RF_E_CUDA;
    cudaMemcpyAsync((double*)w.theta.p + s0 * P, (const double*)w.h_theta.p + s0 * P, sizeof(double) * ns * P,
                    cudaMemcpyHostToDevice, st);
    launch_pass(m, d, G.plan, (const double*)w.theta.p, (double*)w.out.p, (int32_t*)w.flags.p, true, st, g);
    cudaMemcpyAsync((double*)w.h_out.p + s0 * (1 + P), (const double*)w.out.p + s0 * (1 + P),
                    sizeof(double) * ns * (1 + P), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync((int32_t*)w.h_flags.p + s0, (const int32_t*)w.flags.p + s0, sizeof(int32_t) * ns,
                    cudaMemcpyDeviceToHost, st);
    if (!cuda_ok(cudaStreamEndCapture(st, &graph), "graph capture")) return RF_E_CUDA;
    const bool ok = cuda_ok(cudaGraphInstantiate(&G.exec, graph, 0), "graph instantiate");
    cudaGraphDestroy(graph);
    return ok ? RF_OK : RF_E_CUDA;
  }

  // Queues group g's pass over `active` (non-empty, within the group's sets).
  rf_status launch(int g, const std::vector<int32_t>& active, const std::vector<double>& theta) {
    Group& G = grp[g];
    bool rebuilt = false;
    if (!replan(G, active, &rebuilt)) return RF_E_OOM;
    cudaStream_t& st = streams[stream_of(g)];
    if (!st && !cuda_ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream")) return RF_E_CUDA;
    if (!G.done && !cuda_ok(cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming), "event")) return RF_E_CUDA;
    if (rebuilt || !G.exec) {
      const rf_status s = capture(g);
      if (s != RF_OK) return s;
    }
    Workspace& w = d->ws;
    const int P = m->m.prog.n_free;
    const size_t s0 = G.planned.front(), ns = (size_t)G.planned.back() + 1 - s0;
    std::memcpy((double*)w.h_theta.p + s0 * P, theta.data() + s0 * P, sizeof(double) * ns * P);
    if (!cuda_ok(cudaGraphLaunch(G.exec, st), "graph launch") || !cuda_ok(cudaEventRecord(G.done, st), "event"))
      return RF_E_CUDA;
    note_launches(2, st);  // the graph's K1 and event kernel
    return RF_OK;
  }

  // Waits for group g's pass and reads its results.
  rf_status wait(int g, std::vector<double>& nll, std::vector<double>& grad) {
    Group& G = grp[g];
    if (!cuda_ok(cudaEventSynchronize(G.done), "graph sync")) return RF_E_CUDA;
    const int P = m->m.prog.n_free;
    const double* o = (const double*)d->ws.h_out.p;
    for (int32_t s : G.planned) {
      nll[s] = o[(size_t)s * (1 + P)];
      for (int k = 0; k < P; ++k) grad[(size_t)s * P + k] = o[(size_t)s * (1 + P) + 1 + k];
    }
    return RF_OK;
  }

  // Captures kDeviceRounds rounds of the n sets whose records are in
  // r_state: the pass over the plan the previous step compacted (r_plan,
  // counts in r_dyn), then the step.  The launch shapes are those of
  // n_sets sets and n_items items (at least the counts the rounds see);
  // ends with the phases' download.
  rf_status capture_rounds(int n, int32_t n_sets, int32_t n_items, double tol, int max_evals) {
    cudaStream_t st = streams[0];
    if (r_exec) {
      cudaGraphExecDestroy(r_exec);
      r_exec = nullptr;
    }
    Workspace& w = d->ws;
    const int P = m->m.prog.n_free;
    int32_t* dyn = (int32_t*)r_dyn.p;
    const double* bounds = (const double*)r_bounds.p;
    r_plan.n_active = n_sets;
    r_plan.n_items = n_items;
    r_cap_sets = n_sets;
    r_cap_items = n_items;
    FitStepArgs a;
    a.state = (double*)r_state.p;
    a.set_of = (const int32_t*)r_sets.p;
    a.chunks = (const int32_t*)r_chunks.p;
    a.n = n;
    a.P = P;
    a.out = (const double*)w.out.p;
    a.theta = (double*)w.theta.p;
    a.lo = bounds;
    a.hi = bounds + P;
    a.bounded = (const char*)(bounds + 2 * P);
    a.tol = tol;
    a.max_evals = max_evals;
    a.phase = (int32_t*)r_phase.p;
    a.plan_sets = (int32_t*)r_plan.sets.p;
    a.plan_items = (int2*)r_plan.items.p;
    a.dyn = dyn;
    a.ticket = dyn + 2;
    cudaGraph_t graph = nullptr;
    if (!cuda_ok(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "graph capture")) return RF_E_CUDA;
    for (int r = 0; r < kDeviceRounds; ++r) {
      launch_pass(m, d, r_plan, (const double*)w.theta.p, (double*)w.out.p, (int32_t*)w.flags.p, true, st, 3, dyn);
      launch_fit_step(a, st);
    }
    cudaMemcpyAsync(h_phase.p, r_phase.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
    if (!cuda_ok(cudaStreamEndCapture(st, &graph), "graph capture")) return RF_E_CUDA;
    const bool ok = cuda_ok(cudaGraphInstantiate(&r_exec, graph, 0), "graph instantiate");
    cudaGraphDestroy(graph);
    return ok ? RF_OK : RF_E_CUDA;
  }

  // One synchronous whole-batch pass.
  rf_status run(const std::vector<int32_t>& active, const std::vector<double>& theta, std::vector<double>& nll,
                std::vector<double>& grad) {
    if (!use_graph) {
      bool rebuilt = false;
      if (!replan(grp[2], active, &rebuilt)) return RF_E_OOM;
      const rf_status s = eval_host(m, d, grp[2].plan, theta.data(), nll.data(), grad.data(), nullptr);
      return s == RF_E_DOMAIN ? RF_OK : s;
    }
    const rf_status s = launch(2, active, theta);
    return s != RF_OK ? s : wait(2, nll, grad);
  }
};

struct DeviceSteps {
  Evaluator* ev;
  const int32_t* set_of;  // problem -> dataset set; null: the identity
};

namespace {

// Runs the rounds of the still-active problems `active` (increasing) on the
// device until all are done or max_evals rounds have run.  Their states go
// to the device as records; each graph launch runs kDeviceRounds rounds of
// parameter point, event pass and step, the step compacting the next
// pass's plan to the sets still going; between launches the host only
// reads the phases (and captures the rounds again, with smaller launch
// shapes, once the items have shrunk 4-fold).  The states come back at the end (th and jc
// refreshed for any problem not done).  Every problem takes the same trial
// points as in host rounds: the step is the same code, rounding the same
// way (fit_step.h), and a set's pass result does not depend on the plan.
rf_status device_rounds(DeviceSteps& dv, const std::vector<int32_t>& active, std::vector<SetFit>& fits,
                        const Coords& co, double tol, int max_evals, std::vector<double>& th, std::vector<double>& jc) {
  Evaluator& ev = *dv.ev;
  rf_data* d = ev.d;
  Workspace& w = d->ws;
  const int P = co.P, n = (int)active.size(), W = qn::tail_record_words(P);
  cudaStream_t& st = ev.streams[0];
  if (!st && !cuda_ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream")) return RF_E_CUDA;
  std::vector<int32_t> sets(n), chunks(n), phase(n);
  for (int i = 0; i < n; ++i) {
    sets[i] = dv.set_of ? dv.set_of[active[i]] : active[i];
    chunks[i] = (int32_t)d->chunks[sets[i]];
  }
  std::vector<double> rec((size_t)n * W);
  for (int i = 0; i < n; ++i) {
    const SetFit& F = fits[active[i]];
    double* r = rec.data() + (size_t)i * W;
    std::memcpy(r, &F.c, sizeof(qn::State));
    double* v = r + qn::kStateWords;
    const std::vector<double>* parts[5] = {&F.x, &F.g, &F.p, &F.g_lo, &F.trial};
    for (int j = 0; j < 5; ++j) std::copy(parts[j]->begin(), parts[j]->end(), v + (size_t)j * P);
    std::copy(jc.begin() + (size_t)active[i] * P, jc.begin() + (size_t)(active[i] + 1) * P, v + (size_t)5 * P);
    std::copy(F.H.begin(), F.H.end(), v + (size_t)6 * P);
    phase[i] = F.c.phase;
  }
  std::vector<char> bounds(sizeof(double) * 2 * P + P);
  std::memcpy(bounds.data(), co.lo.data(), sizeof(double) * P);
  std::memcpy(bounds.data() + sizeof(double) * P, co.hi.data(), sizeof(double) * P);
  std::memcpy(bounds.data() + sizeof(double) * 2 * P, co.bounded.data(), P);
  // the first plan: every set of the list
  if (!build_plan(d, sets, &ev.r_plan)) return RF_E_OOM;
  const int32_t dyn0[3] = {ev.r_plan.n_active, ev.r_plan.n_items, 0};
  if (!ev.r_state.ensure(sizeof(double) * rec.size()) || !ev.r_sets.ensure(sizeof(int32_t) * n) ||
      !ev.r_chunks.ensure(sizeof(int32_t) * n) || !ev.r_phase.ensure(sizeof(int32_t) * n) ||
      !ev.r_dyn.ensure(sizeof(dyn0)) || !ev.r_bounds.ensure(bounds.size()) ||
      !ev.h_phase.ensure(sizeof(int32_t) * n))
    return RF_E_OOM;
  double* h_th = (double*)w.h_theta.p;
  for (int i = 0; i < n; ++i)
    std::copy(th.begin() + (size_t)active[i] * P, th.begin() + (size_t)(active[i] + 1) * P, h_th + (size_t)sets[i] * P);
  const size_t s0 = sets.front(), ns = (size_t)sets.back() + 1 - s0;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cuda_ok(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st), "upload");
  };
  if (!up(ev.r_state.p, rec.data(), sizeof(double) * rec.size()) || !up(ev.r_sets.p, sets.data(), sizeof(int32_t) * n) ||
      !up(ev.r_chunks.p, chunks.data(), sizeof(int32_t) * n) || !up(ev.r_phase.p, phase.data(), sizeof(int32_t) * n) ||
      !up(ev.r_dyn.p, dyn0, sizeof(dyn0)) || !up(ev.r_bounds.p, bounds.data(), bounds.size()) ||
      !up((double*)w.theta.p + s0 * P, h_th + s0 * P, sizeof(double) * ns * P) ||
      !cuda_ok(cudaStreamSynchronize(st), "upload"))
    return RF_E_CUDA;
  std::vector<int32_t> going(n);
  for (int i = 0; i < n; ++i) going[i] = i;
  const int32_t* ph = (const int32_t*)ev.h_phase.p;
  const int max_launches = max_evals / kDeviceRounds + 2;
  for (int it = 0; it < max_launches && !going.empty(); ++it) {
    int32_t items = 0;
    for (int i : going) items += chunks[i];
    if (!ev.r_exec || 4 * items < ev.r_cap_items) {
      const rf_status s = ev.capture_rounds(n, (int32_t)going.size(), items, tol, max_evals);
      if (s != RF_OK) return s;
    }
    if (!cuda_ok(cudaGraphLaunch(ev.r_exec, st), "graph launch") || !cuda_ok(cudaStreamSynchronize(st), "graph sync"))
      return RF_E_CUDA;
    note_launches(3 * kDeviceRounds, st);
    going.clear();
    for (int i = 0; i < n; ++i)
      if (ph[i] != qn::DONE) going.push_back(i);
  }
  if (!cuda_ok(cudaMemcpyAsync(rec.data(), ev.r_state.p, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost, st),
               "download") ||
      !cuda_ok(cudaStreamSynchronize(st), "download"))
    return RF_E_CUDA;
  for (int i = 0; i < n; ++i) {
    const int pr = active[i];
    SetFit& F = fits[pr];
    const double* r = rec.data() + (size_t)i * W;
    std::memcpy(&F.c, r, sizeof(qn::State));
    const double* v = r + qn::kStateWords;
    std::vector<double>* parts[5] = {&F.x, &F.g, &F.p, &F.g_lo, &F.trial};
    for (int j = 0; j < 5; ++j) std::copy(v + (size_t)j * P, v + (size_t)(j + 1) * P, parts[j]->begin());
    std::copy(v + (size_t)6 * P, v + (size_t)6 * P + (size_t)P * P, F.H.begin());
    if (!F.done()) co.to_theta_jac(F.trial.data(), &th[(size_t)pr * P], &jc[(size_t)pr * P]);
  }
  return RF_OK;
}

}  // namespace

// The batched fit driver: S independent problems of P parameters with
// bounds lo/hi (lo >= hi: unbounded), started at `start` (S x P).  Each
// round asks every active problem for one trial point and evaluates all of
// them with one call of `eval` (active sets, theta S x P in, nll S and
// gradient S x P out, indexed by set).  cov (S x P x P) may be null.
rf_status fit_batch(int S, int P, const double* lo, const double* hi, const double* start, double tol, int max_evals,
                    bool want_cov, const BatchEval& eval, const SplitEval* split, double* theta_hat,
                    double* nll_min, double* cov, int32_t* n_evals, int32_t* fit_status, DeviceSteps* dev) {
  (void)want_cov;
  Coords co;
  co.P = P;
  co.lo.assign(lo, lo + P);
  co.hi.assign(hi, hi + P);
  co.bounded.resize(P);
  for (int k = 0; k < P; ++k)
    co.bounded[k] = co.lo[k] < co.hi[k] && std::isfinite(co.lo[k]) && std::isfinite(co.hi[k]);

  std::vector<SetFit> fits(S);
  std::vector<double> th((size_t)S * P), nll(S), grad((size_t)S * P);
  for (int s = 0; s < S; ++s) {
    fits[s].init(P);
    co.to_internal(start + (size_t)s * P, fits[s].trial.data());
  }
  // The per-set update is O(P^2): with many parameters even a few sets are
  // worth spreading over threads.
  const int64_t min_n = P >= 32 ? 2 : 1024;
  Pool pool(S >= min_n ? pool_threads() : 1);
  std::vector<int32_t> active;
  std::vector<double> jc((size_t)S * std::max(P, 1));
  // One host pass per round: a set's result is delivered and its next trial
  // point mapped to theta (and the Jacobian) in the same task.
  pool.run(S, [&](int64_t s) { co.to_theta_jac(fits[s].trial.data(), &th[(size_t)s * P], &jc[(size_t)s * P]); },
           min_n);
  auto deliver = [&](const std::vector<int32_t>& sets) {
    pool.run((int64_t)sets.size(), [&](int64_t i) {
      const int s = sets[i];
      double* ga = fits[s].w_ga.data();
      for (int k = 0; k < P; ++k) ga[k] = grad[(size_t)s * P + k] * jc[(size_t)s * P + k];
      fits[s].deliver(nll[s], ga, tol, max_evals);
      if (!fits[s].done()) co.to_theta_jac(fits[s].trial.data(), &th[(size_t)s * P], &jc[(size_t)s * P]);
    }, min_n);
  };
  if (split && split->split > 0 && split->split < S) {
    // Pipelined rounds over the halves [0, split) and [split, S): while one
    // half's pass runs on the device the host updates the other half.  Each
    // set's sequence of trial points is the same as in the plain loop below,
    // which takes over once the active events fall below split->min_events.
    std::vector<int32_t> act[2];
    bool busy[2] = {false, false};
    auto collect = [&](int g) {
      act[g].clear();
      const int a = g ? (int)split->split : 0, b = g ? S : (int)split->split;
      for (int s = a; s < b; ++s)
        if (!fits[s].done()) act[g].push_back(s);
    };
    auto drain = [&](rf_status st) {
      for (int g = 0; g < 2; ++g)
        if (busy[g]) split->wait(g, nll, grad);
      return st;
    };
    rf_status st = RF_OK;
    for (int g = 0; g < 2 && st == RF_OK; ++g) {
      collect(g);
      if (!act[g].empty() && (st = split->launch(g, act[g], th)) == RF_OK) busy[g] = true;
    }
    if (st != RF_OK) return drain(st);
    while (busy[0] || busy[1]) {
      for (int g = 0; g < 2; ++g) {
        if (!busy[g]) continue;
        busy[g] = false;
        if ((st = split->wait(g, nll, grad)) != RF_OK) return drain(st);
        deliver(act[g]);
        collect(g);
        if (act[g].empty() || split->events(act[0]) + split->events(act[1]) < split->min_events) continue;
        if ((st = split->launch(g, act[g], th)) != RF_OK) return drain(st);
        busy[g] = true;
      }
    }
  }
  bool dev_used = false;
  while (true) {
    active.clear();
    for (int s = 0; s < S; ++s)
      if (!fits[s].done()) active.push_back(s);
    if (active.empty()) break;
    if (dev && !dev_used && P <= qn::kTailMaxP) {
      // the remaining rounds on the device; a set it leaves unfinished (it
      // stops after max_evals rounds) goes on here
      dev_used = true;
      const rf_status st = device_rounds(*dev, active, fits, co, tol, max_evals, th, jc);
      if (st != RF_OK) return st;
      continue;
    }
    const rf_status st = eval(active, th, nll, grad);
    if (st != RF_OK) return st;
    deliver(active);
  }
  for (int s = 0; s < S; ++s) {
    co.to_theta(fits[s].x.data(), theta_hat + (size_t)s * P);
    nll_min[s] = fits[s].c.status == RF_E_DOMAIN ? kInf : fits[s].c.f;
    n_evals[s] = fits[s].c.evals;
    fit_status[s] = fits[s].c.status;
  }
  if (cov) {
    // Central differences of the analytic gradient, all sets per pass; the
    // step is 1e-3 of each parameter's BFGS error estimate.
    std::vector<double> Hs((size_t)S * P * P, 0.0), h((size_t)S * P);
    std::vector<int32_t> ok_sets;
    for (int s = 0; s < S; ++s) {
      if (fits[s].c.status == RF_E_DOMAIN) continue;
      ok_sets.push_back(s);
      for (int k = 0; k < P; ++k) {
        const double jk = co.jac(k, fits[s].x[k]);
        const double sig = std::sqrt(std::max(0.0, fits[s].H[k * P + k])) * std::fabs(jk);
        const double t = theta_hat[(size_t)s * P + k];
        double hk = 1e-3 * sig;
        if (!(hk > 1e-9 * std::max(1.0, std::fabs(t)))) hk = 1e-6 * std::max(1.0, std::fabs(t));
        h[(size_t)s * P + k] = hk;
      }
    }
    std::vector<double> gp((size_t)S * P), gm((size_t)S * P);
    for (int k = 0; k < P && !ok_sets.empty(); ++k) {
      for (int sign = 0; sign < 2; ++sign) {
        for (int s : ok_sets) {
          for (int j = 0; j < P; ++j) th[(size_t)s * P + j] = theta_hat[(size_t)s * P + j];
          th[(size_t)s * P + k] += (sign == 0 ? 1.0 : -1.0) * h[(size_t)s * P + k];
        }
        const rf_status st = eval(ok_sets, th, nll, sign == 0 ? gp : gm);
        if (st != RF_OK) return st;
      }
      for (int s : ok_sets)
        for (int j = 0; j < P; ++j)
          Hs[(size_t)s * P * P + j * P + k] =
              (gp[(size_t)s * P + j] - gm[(size_t)s * P + j]) / (2.0 * h[(size_t)s * P + k]);
    }
    for (int s = 0; s < S; ++s) {
      double* c = cov + (size_t)s * P * P;
      std::vector<double> A(Hs.begin() + (size_t)s * P * P, Hs.begin() + (size_t)(s + 1) * P * P);
      for (int i = 0; i < P; ++i)
        for (int j = 0; j < i; ++j) A[i * P + j] = A[j * P + i] = 0.5 * (A[i * P + j] + A[j * P + i]);
      if (fits[s].c.status == RF_E_DOMAIN || !invert(A, P, c))
        std::fill(c, c + P * P, std::numeric_limits<double>::quiet_NaN());
    }
  }
  return RF_OK;
}

}  // namespace rf

using namespace rf;

extern "C" rf_status rf_fit(const rf_model* m, const rf_data* d, const double* theta0, const rf_fit_opts* opts,
                            double* theta_hat, double* nll_min, double* cov, int32_t* n_evals,
                            int32_t* fit_status) {
  if (!m || !d || !theta_hat || !nll_min || !n_evals || !fit_status) {
    set_error("rf_fit: bad argument (NULL)");
    return RF_E_INVALID;
  }
  if (d->n_obs != m->m.prog.n_obs) {
    set_error("rf_fit: data and model have different observable counts");
    return RF_E_INVALID;
  }
  const int P = m->m.prog.n_free, S = d->n_sets;
  const double tol = (opts && opts->tol_edm > 0.0) ? opts->tol_edm : 1e-7;
  const int max_evals = (opts && opts->max_evals > 0) ? opts->max_evals : 1000;
  const bool want_cov = opts && opts->want_cov && cov;
  rf_data* dd = const_cast<rf_data*>(d);
  if (!ensure_workspace(m, dd)) return RF_E_OOM;
  if (P == 0) {
    std::vector<double> z(1);
    const rf_status s = rf_nll(m, d, z.data(), nll_min, nullptr);
    for (int s2 = 0; s2 < S; ++s2) {
      n_evals[s2] = 1;
      fit_status[s2] = std::isfinite(nll_min[s2]) ? RF_OK : RF_E_DOMAIN;
    }
    return s == RF_E_DOMAIN ? RF_OK : s;
  }

  std::vector<double> start((size_t)S * P);
  for (int s = 0; s < S; ++s)
    for (int k = 0; k < P; ++k) start[(size_t)s * P + k] = theta0 ? theta0[(size_t)s * P + k] : m->m.theta_default[k];
  Evaluator ev(m, dd, !(opts && opts->no_graph == 1));
  // the halves of a pipelined fit split the events evenly
  SplitEval split;
  split.split = 0;
  if (ev.use_graph && S >= 2) {
    const int64_t total = d->offsets[S] - d->offsets[0];
    int s = 1;
    while (s < S - 1 && 2 * (d->offsets[s] - d->offsets[0]) < total) ++s;
    split.split = s;
  }
  // device rounds for a batch (one set's rounds are faster with host steps:
  // its pass dominates and the step's serial chain on one warp costs more
  // than the host's round trip)
  DeviceSteps dsteps{&ev, nullptr};
  const bool device = ev.use_graph && !(opts && opts->host_steps == 1) && S >= 2;
  split.min_events = device ? std::max(kPipelineMinEvents, kDeviceRoundEvents) : kPipelineMinEvents;
  split.launch = [&](int g, const std::vector<int32_t>& a, const std::vector<double>& th) { return ev.launch(g, a, th); };
  split.wait = [&](int g, std::vector<double>& nll, std::vector<double>& grad) { return ev.wait(g, nll, grad); };
  split.events = [&](const std::vector<int32_t>& a) { return ev.events_of(a); };
  return fit_batch(S, P, m->m.lo.data(), m->m.hi.data(), start.data(), tol, max_evals, want_cov,
                   [&](const std::vector<int32_t>& active, std::vector<double>& th, std::vector<double>& nll,
                       std::vector<double>& grad) { return ev.run(active, th, nll, grad); },
                   split.split > 0 ? &split : nullptr,
                   theta_hat, nll_min, want_cov ? cov : nullptr, n_evals, fit_status, device ? &dsteps : nullptr);
}

extern "C" rf_status rf_fit_sets(const rf_model* m, const rf_data* d, const int32_t* sets, int32_t n,
                                 const double* theta0, const rf_fit_opts* opts, double* theta_hat, double* nll_min,
                                 double* cov, int32_t* n_evals, int32_t* fit_status) {
  if (!m || !d || n < 0 || (n > 0 && (!sets || !theta_hat || !nll_min || !n_evals || !fit_status))) {
    set_error("rf_fit_sets: bad argument (NULL)");
    return RF_E_INVALID;
  }
  if (d->n_obs != m->m.prog.n_obs) {
    set_error("rf_fit_sets: data and model have different observable counts");
    return RF_E_INVALID;
  }
  const int P = m->m.prog.n_free, S = d->n_sets;
  std::vector<char> seen(S, 0);
  for (int i = 0; i < n; ++i) {
    if (sets[i] < 0 || sets[i] >= S || seen[sets[i]]) {
      set_error("rf_fit_sets: set indices must be distinct and in [0, n_sets)");
      return RF_E_INVALID;
    }
    seen[sets[i]] = 1;
  }
  if (n == 0) return RF_OK;
  if (P == 0) {
    set_error("rf_fit_sets: the model has no free parameter");
    return RF_E_INVALID;
  }
  const double tol = (opts && opts->tol_edm > 0.0) ? opts->tol_edm : 1e-7;
  const int max_evals = (opts && opts->max_evals > 0) ? opts->max_evals : 1000;
  const bool want_cov = opts && opts->want_cov && cov;
  rf_data* dd = const_cast<rf_data*>(d);
  if (!ensure_workspace(m, dd)) return RF_E_OOM;
  // Problem i of the batch is set srt[i], the listed sets in increasing
  // order (the evaluator's plans take active sets in increasing order);
  // pos[i] is its place in the caller's list.
  std::vector<int32_t> pos(n), srt(n);
  for (int i = 0; i < n; ++i) pos[i] = i;
  std::sort(pos.begin(), pos.end(), [&](int a, int b) { return sets[a] < sets[b]; });
  for (int i = 0; i < n; ++i) srt[i] = sets[pos[i]];
  std::vector<double> start((size_t)n * P);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < P; ++k)
      start[(size_t)i * P + k] = theta0 ? theta0[(size_t)pos[i] * P + k] : m->m.theta_default[k];
  Evaluator ev(m, dd, !(opts && opts->no_graph == 1));
  DeviceSteps dsteps{&ev, srt.data()};
  const bool device = ev.use_graph && !(opts && opts->host_steps == 1) && n >= 2;
  std::vector<double> th_s((size_t)S * P), nll_s(S), grad_s((size_t)S * P);
  std::vector<int32_t> act_s;
  std::vector<double> th_o((size_t)n * P), nll_o(n), cov_o(want_cov ? (size_t)n * P * P : 0);
  std::vector<int32_t> ne_o(n), st_o(n);
  const rf_status r = fit_batch(
      n, P, m->m.lo.data(), m->m.hi.data(), start.data(), tol, max_evals, want_cov,
      [&](const std::vector<int32_t>& active, std::vector<double>& th, std::vector<double>& nll,
          std::vector<double>& grad) {
        act_s.resize(active.size());
        for (size_t j = 0; j < active.size(); ++j) {
          const int i = active[j], s = srt[i];
          act_s[j] = s;
          for (int k = 0; k < P; ++k) th_s[(size_t)s * P + k] = th[(size_t)i * P + k];
        }
        const rf_status st = ev.run(act_s, th_s, nll_s, grad_s);
        for (size_t j = 0; j < active.size(); ++j) {
          const int i = active[j], s = srt[i];
          nll[i] = nll_s[s];
          for (int k = 0; k < P; ++k) grad[(size_t)i * P + k] = grad_s[(size_t)s * P + k];
        }
        return st;
      },
      nullptr, th_o.data(), nll_o.data(), want_cov ? cov_o.data() : nullptr, ne_o.data(), st_o.data(),
      device ? &dsteps : nullptr);
  for (int i = 0; i < n; ++i) {
    const int o = pos[i];
    for (int k = 0; k < P; ++k) theta_hat[(size_t)o * P + k] = th_o[(size_t)i * P + k];
    nll_min[o] = nll_o[i];
    n_evals[o] = ne_o[i];
    fit_status[o] = st_o[i];
    if (want_cov)
      for (int k = 0; k < P * P; ++k) cov[(size_t)o * P * P + k] = cov_o[(size_t)i * P * P + k];
  }
  return r;
}
