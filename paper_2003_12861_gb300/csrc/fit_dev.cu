// The quasi-Newton step of a batched fit on the device (the rounds of a fit
// that run without the host): a warp per set advances the set's state
// machine (fit_step.h) with the result of the pass that just ran and maps
// its next trial point to theta; the last block to finish compacts the
// next pass's plan to the sets still going, so that the next round's
// parameter point and event pass follow at once.
// Compiled with --fmad=false: the shared state machine must round every
// operation as the host driver does (see fit_step.h).
#include "api_internal.h"
#include "fit_step.h"

namespace rf {

namespace {

// The element loops of the state machine across the lanes of a warp.
struct WarpLoop {
  __device__ static int first() { return threadIdx.x & 31; }
  __device__ static int step() { return 32; }
  __device__ static void sync() { __syncwarp(); }
};

constexpr int kStepWarps = 4;
constexpr int kStepThreads = kStepWarps * 32;
constexpr int kBigSets = 256;
constexpr int kStageSets = 2048;

// Shared doubles per warp: the set's record, then ga, w_s, w_y, w_hy, w_r.
__host__ __device__ inline int step_smem_words(int P) { return qn::tail_record_words(P) + 5 * P; }

// kP: the parameter count when known at compile time (the loops over
// elements then have constant trip counts), 0 for any count.
template <int kP>
__global__ void __launch_bounds__(kStepThreads) fit_step_kernel(FitStepArgs a) {
  extern __shared__ double smem[];
  __shared__ int last;
  __shared__ int scan_a[kStepThreads], scan_i[kStepThreads];
  __shared__ int n_big;
  __shared__ int2 big[kBigSets];  // (set index, first item) of sets of more than 32 chunks
  __shared__ int st_phase[kStageSets], st_chunks[kStageSets], st_set[kStageSets];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = kP ? kP : a.P, W = qn::tail_record_words(P);
  if (a.dyn[0] == 0) return;  // every set is done: nothing to step or plan
  const int i = blockIdx.x * kStepWarps + warp;
  if (i < a.n) {
    double* gr = a.state + (size_t)i * W;
    qn::State c = *reinterpret_cast<const qn::State*>(gr);
    if (c.phase != qn::DONE) {
      double* rec = smem + (size_t)warp * step_smem_words(P);
      double* ga = rec + W;
      for (int k = lane; k < W; k += 32) rec[k] = gr[k];
      __syncwarp();
      const qn::TailView t = qn::tail_view(rec, P);
      const int s = a.set_of[i];
      const double* o = a.out + (size_t)s * (1 + P);
      for (int k = lane; k < P; k += 32) ga[k] = o[1 + k] * t.jc[k];
      __syncwarp();
      const qn::Vecs v{t.x, t.g, t.H, t.p, t.g_lo, t.trial, ga + P, ga + 2 * P, ga + 3 * P, ga + 4 * P};
      qn::deliver<WarpLoop>(P, c, v, o[0], ga, a.tol, a.max_evals);
      if (c.phase != qn::DONE)
        qn::to_theta_jac<WarpLoop>(P, a.lo, a.hi, a.bounded, t.trial, a.theta + (size_t)s * P, t.jc);
      __syncwarp();
      if (lane == 0) *reinterpret_cast<qn::State*>(rec) = c;
      __syncwarp();
      for (int k = lane; k < W; k += 32) gr[k] = rec[k];
      if (lane == 0) a.phase[i] = c.phase;
    }
  }
  // The last block to get here compacts the plan: its threads take
  // contiguous ranges of the sets, count those still going and their
  // chunks, scan the counts, and write sets and items in set order.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(a.ticket, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the sets' phases, chunk counts and dataset sets, staged in shared
  // memory by coalesced loads when they fit
  const bool staged = a.n <= kStageSets;
  if (staged) {
    for (int j = threadIdx.x; j < a.n; j += kStepThreads) {
      st_phase[j] = __ldcg(a.phase + j);
      st_chunks[j] = a.chunks[j];
      st_set[j] = a.set_of[j];
    }
    __syncthreads();
  }
  const int per = (a.n + kStepThreads - 1) / kStepThreads;
  const int b0 = min(a.n, (int)threadIdx.x * per), b1 = min(a.n, b0 + per);
  int na = 0, ni = 0;
  for (int j = b0; j < b1; ++j)
    if ((staged ? st_phase[j] : __ldcg(a.phase + j)) != qn::DONE) {
      ++na;
      ni += staged ? st_chunks[j] : a.chunks[j];
    }
  scan_a[threadIdx.x] = na;
  scan_i[threadIdx.x] = ni;
  __syncthreads();
  for (int off = 1; off < kStepThreads; off <<= 1) {  // inclusive scan
    const int xa = threadIdx.x >= off ? scan_a[threadIdx.x - off] : 0;
    const int xi = threadIdx.x >= off ? scan_i[threadIdx.x - off] : 0;
    __syncthreads();
    scan_a[threadIdx.x] += xa;
    scan_i[threadIdx.x] += xi;
    __syncthreads();
  }
  // each thread writes its sets and the items of its sets of up to 32
  // chunks; larger sets go to a list whose items the warps write, a set per
  // warp, its chunks across the lanes
  if (threadIdx.x == 0) n_big = 0;
  __syncthreads();
  int pa = scan_a[threadIdx.x] - na, pi = scan_i[threadIdx.x] - ni;
  for (int j = b0; j < b1; ++j) {
    if ((staged ? st_phase[j] : __ldcg(a.phase + j)) == qn::DONE) continue;
    const int s = staged ? st_set[j] : a.set_of[j], c = staged ? st_chunks[j] : a.chunks[j];
    a.plan_sets[pa++] = s;
    if (c <= 32) {
      for (int k = 0; k < c; ++k) a.plan_items[pi + k] = make_int2(s, k);
    } else {
      const int b = atomicAdd(&n_big, 1);
      if (b < kBigSets) {
        big[b] = make_int2(j, pi);
      } else {
        for (int k = 0; k < c; ++k) a.plan_items[pi + k] = make_int2(s, k);
      }
    }
    pi += c;
  }
  if (threadIdx.x == kStepThreads - 1) {
    a.dyn[0] = scan_a[threadIdx.x];
    a.dyn[1] = scan_i[threadIdx.x];
    *a.ticket = 0;
  }
  __syncthreads();
  const int nb = n_big < kBigSets ? n_big : kBigSets;
  for (int b = warp; b < nb; b += kStepWarps) {
    const int j = big[b].x, off = big[b].y, s = a.set_of[j];
    for (int k = lane; k < a.chunks[j]; k += 32) a.plan_items[off + k] = make_int2(s, k);
  }
}

}  // namespace

void launch_fit_step(const FitStepArgs& a, cudaStream_t st) {
  if (a.n <= 0) return;
  const int blocks = (a.n + kStepWarps - 1) / kStepWarps;
  const size_t smem = sizeof(double) * kStepWarps * step_smem_words(a.P);
  switch (a.P) {
    case 4: fit_step_kernel<4><<<blocks, kStepThreads, smem, st>>>(a); break;
    case 6: fit_step_kernel<6><<<blocks, kStepThreads, smem, st>>>(a); break;
    case 12: fit_step_kernel<12><<<blocks, kStepThreads, smem, st>>>(a); break;
    default: fit_step_kernel<0><<<blocks, kStepThreads, smem, st>>>(a);
  }
}

}  // namespace rf
