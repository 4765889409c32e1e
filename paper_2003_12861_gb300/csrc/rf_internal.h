// Internal layout shared by the library's translation units (host + device).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rf.h"

namespace rf {

constexpr int kMaxNodes = 64;    // graph nodes accepted by rf_model_create
constexpr int kMaxPdf = 24;      // PDF nodes in one program
constexpr int kMaxFree = 16;     // free parameters
constexpr int kMaxSlots = 32;    // gradient slots (per-leaf local parameters + SUM fractions)
constexpr int kMaxObs = 8;       // observables (columns)
constexpr int kMaxConst = 256;   // per-set constant block (doubles)
constexpr int kMaxPar = 7;       // parameters of one leaf

// Deterministic reduction geometry: a chunk is 4096 events split over 128
// lanes (lane l takes events l, l+128, ..., in order); chunks are combined by
// a radix-32 tree.
// Up to this many active sets K1 runs one block per set (latency), beyond
// one thread per set (throughput).
constexpr int kBlockK1MaxSets = 256;
constexpr int kChunk = 4096;
constexpr int kLanes = 128;
constexpr int kPerLane = kChunk / kLanes;  // 32
constexpr int kRadix = 32;

enum Kind : int8_t {
  OBS = 0, PARAM = 1, GAUSS = 2, EXPO = 3, GAUSSEXP = 4, CHEB = 5, POLY = 6, SUM = 7, PROD = 8, POISSON = 9, EXTEND = 10,
  EXPR = 11
};
// RF_EXPR programs: per node at most 64 operations and 16 constants, per
// model 128 and 32 in all; the evaluation stack holds 16 values.
constexpr int kExprMaxOps = 64, kExprMaxConsts = 16, kExprPoolOps = 128, kExprPoolConsts = 32, kExprStack = 16;
// Largest observable range (integers) of a POISSON leaf.
constexpr int kMaxPoissonRange = 100000;

// One PDF node of the compiled program, in dependency order (children first).
struct PNode {
  int8_t kind;
  int8_t col;                // leaves: observable column
  int8_t n_child;            // SUM: components; PROD: factors
  int8_t n_par;              // leaves: parameters; SUM: fractions (n_child - 1)
  int8_t child[8];           // program indices of SUM components / PROD factors
  int8_t pfree[kMaxPar];     // leaves: free index of local parameter j (-1: fixed); SUM: of fraction j
  int16_t cofs;              // offset of the node's constants in the per-set block
  int16_t slot0;             // first gradient slot of this node
  int16_t ex_op0, ex_nops, ex_c0;  // EXPR: its program in the model's pools
  double lo, hi;             // leaves: observable range
  double pfixed[kMaxPar];    // leaves/SUM: value of a fixed parameter
};

// Whole compiled program.  Passed by value to kernels (__grid_constant__).
struct Program {
  int32_t n_pdf;             // nodes in `node`, root last
  int32_t n_obs;
  int32_t n_free;
  int32_t n_slots;           // gradient slots
  int32_t n_const;           // doubles per set in the constant block
  int32_t has_slow;          // 1 if some node has a rare slow path (GAUSSEXP)
  int8_t slot_free[kMaxSlots];  // slot -> free parameter (-1: fixed)
  // Extended likelihood (EXTEND root): the NLL gains nu - N log nu per set.
  int32_t ext;               // 1 if extended
  int32_t ext_free;          // nu's free index, or -1 (fixed: ext_fixed)
  double ext_fixed;
  int32_t has_expr;          // 1 if some node is an EXPR (its K1 needs the block kernel)
  PNode node[kMaxPdf];
  int32_t ex_ops[kExprPoolOps];      // EXPR programs, back to back
  double ex_consts[kExprPoolConsts]; // and their constants
};

// Constant-block layout per node kind (doubles), written by the
// parameter-point kernel and read by the event kernels.
//   GAUSS    [mu, 1/sigma, 1/I, dlogI/dmu, dlogI/dsigma]
//   EXP      [c, x_ref, 1/I_ref, dlogI/dc]            v = exp(c (x - x_ref)) / I_ref
//   GAUSSEXP [mu, 1/sigma, s = sigma/tau, 1/tau, 1/I, dlogI/dtau, dlogI/dmu, dlogI/dsigma]
//   CHEB(n)  [2/(b-a), (a+b)/(b-a), 1/I, dlogI/dc_1..n, c_1..n]
//   POLY(n)  [1/I, dlogI/da_1..n, a_1..n]
//   SUM(n)   [f_1..f_{n-1}, 1 - sum f]
//   PROD     []
//   POISSON  [lambda, log lambda, 1/lambda, 1/I, dlogI/dlambda]   v = pmf(floor x) / I
//   EXPR(n)  [1/I, dlogI/dp_1..n, p_1..n]                v = program(x; p) / I
inline int const_size(int kind, int n_par) {
  switch (kind) {
    case GAUSS: return 5;
    case EXPO: return 4;
    case GAUSSEXP: return 8;
    case CHEB: return 3 + 2 * n_par;
    case POLY: return 1 + 2 * n_par;
    case SUM: return n_par + 1;
    case POISSON: return 5;
    case EXPR: return 1 + 2 * n_par;
    default: return 0;
  }
}

// Which compile-time-specialised fused kernel runs a program (0 = the
// generic graph interpreter).
enum Shape : int32_t {
  SHAPE_GENERIC = 0,
  SHAPE_SUM_GAUSS_POLY1 = 1,      // f Gauss + (1-f) Poly1
  SHAPE_SUM_GAUSSEXP_CHEB2 = 2,   // f (decay (x) Gauss) + (1-f) Chebychev2
  SHAPE_PROD3 = 3,                // [f Gauss + (1-f) Cheb1] x [decay model] x Poly2
};

// Host-side model.
struct Model {
  Program prog;
  Shape shape = SHAPE_GENERIC;
  Shape detected_shape = SHAPE_GENERIC;  // the recognised shape (shape may be forced generic)
  std::vector<rf_node> nodes;
  std::vector<int> free_node;        // free index -> node index
  std::vector<double> theta_default; // free parameter defaults
  std::vector<double> lo, hi;        // free parameter bounds
  std::vector<double> obs_lo, obs_hi;
  std::vector<int> gen_factors;      // program indices of the generation factors
  std::string signature;
  bool extended = false;
  int threads_per_block = 0, blocks_per_sm = 0;
};

void set_error(const std::string& msg);
rf_status compile_model(const rf_node* nodes, int n, int root, Model* m, const rf_expr* exprs = nullptr,
                        int n_exprs = 0);

}  // namespace rf
