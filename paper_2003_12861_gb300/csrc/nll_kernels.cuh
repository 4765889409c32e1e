// Device side of the likelihood: per-parameter-point constants, the fused
// per-event evaluation with its adjoint, and the deterministic reduction tree.
#pragma once

#include <cuda_runtime.h>

#include "rf_internal.h"

namespace rf {

// Columns of a dataset as seen by the kernels.
struct Columns {
  const void* ptr[kMaxObs];
  int32_t is_f32[kMaxObs];
};

// Work description of one evaluation pass (device pointers).
struct Pass {
  const int64_t* offsets;   // n_sets + 1 event offsets
  const int32_t* sets;      // active set indices
  int32_t n_active;
  const int2* items;        // (set, chunk) work items of the active sets
  int32_t n_items;
  const int64_t* tree_base; // per set: first node of its reduction tree
  const double* theta;      // n_sets x n_free
  double* consts;           // n_sets x n_const
  double* tree;             // tree nodes x (2 Q) doubles: (sum, compensation) per quantity
  int32_t* tree_bad;        // bad-event count per tree node
  int32_t* tickets;         // arrival counters per tree node (self-resetting)
  int32_t* counter;         // work-item counter of the persistent grid
  int32_t n_counters;       // counters K1 resets (several launches over item ranges), 0 = 1
  double* out;              // n_sets x (1 + n_free): nll, gradient
  int32_t* flags;           // n_sets: events with pdf <= 0 / not finite (+2^30: theta outside domain)
  unsigned long long* slow; // events that took a slow path in this pass (reset by K1)
  int32_t Q;                // quantities per node: 1 + n_slots (or 1 for NLL only)
  int32_t want_grad;
  int32_t ff_shape;         // specialised float-float event program (Shape), 0 = generic
  float* ffc;               // n_sets x 512 floats of its parameter-point constants, or null
  // Float-float kernels: per chunk, `parts` part records (indexed by the
  // chunk's level-0 tree node x parts + part; room for kMaxParts).
  int32_t parts;            // work units per chunk (1 or 4), fixed per dataset
  float* part_m;            // 32 floats per part: its moment sums (float-float pairs)
  double* part_fb;          // Q doubles per part: its FP64 fallback sums (valid if info bit 0)
  int32_t* part_info;       // per part: bit 0 = fallback sums present, bits 1.. = bad events
  // Partial mode (null otherwise): per set (1 + n_free) (sum, compensation)
  // pairs of (sum log p, d/dtheta_k sum log p), not negated, for a later
  // ordered combine across shards; out is not written.
  double* pairs;
  // Null, or device counts {active sets, work items} that replace n_active
  // and n_items: the rounds of a device-resident fit compact their plan on
  // the device (sets and items then hold at least that many entries).  No
  // active set: the pass is skipped.
  const int32_t* dyn;
};

// Resident blocks per SM the float-float kernels are compiled for (their
// register budget: 72 registers for 7 blocks, 96 for 5).
__host__ __device__ constexpr int ff_min_blocks(int shape) { return shape == SHAPE_PROD3 ? 5 : 7; }

// Work units per chunk of the float-float kernels (Pass::parts: 1, 2 or
// 4): with P parts, part p of a chunk covers lane l's events l + 128 k for k
// in [32 p / P, 32 (p + 1) / P).  Whole chunks spread the per-unit work (the
// lane log, the warp reduction, the record, the claim) over the most
// events, and measured faster than halves or quarters as soon as the chunks
// fill one round of the grid, short last round included (decay model, 1e7
// events = 2.3 rounds: whole chunks 0.180 ms, halves 0.190, quarters 0.189);
// a dataset with fewer chunks than that takes the smallest P whose units do
// (up to 4), so that more of the GPU works on it.  The round is that of a
// reference grid, 152 SMs (the GB300) x the kernel's resident blocks, so P
// is a function of the dataset's chunk count and the model's kernel only,
// never of the launch: a dataset's results do not depend on how it is
// launched.
constexpr int kMaxParts = 4;
constexpr int kRefSMs = 152;
inline int parts_for(int64_t total_chunks, int shape) {
  const int64_t wave = (int64_t)kRefSMs * ff_min_blocks(shape);
  int P = 1;
  while (P < kMaxParts && total_chunks * P < wave) P *= 2;
  return P;
}
constexpr int kPartFloats = 32;

constexpr int32_t kThetaBad = 1 << 30;

void launch_param_point(const Program& P, const Pass& pass, cudaStream_t st);
void note_launches(int n, cudaStream_t st);  // the library's launch count (api.cu)
// Kernel timing hooks (measure.cu): bracket a launch with CUDA events.
void timing_begin(cudaStream_t st);
void timing_end(cudaStream_t st);

// Tile shapes the event kernel of a shape supports, and whether a launch
// shape fits on an SM (registers, shared memory).
bool launch_supports_threads(Shape shape, int threads);
bool launch_fits(Shape shape, int threads, int blocks_per_sm);

void launch_events(const Program& P, Shape shape, const Columns& cols, const Pass& pass, int threads,
                   int blocks_per_sm, int n_sm, cudaStream_t st);

}  // namespace rf
