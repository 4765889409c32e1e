// Graph compiler: node list -> validated DAG -> per-event program.
//
// The paper's model is a computation graph of observables, parameters,
// functions and PDFs (Sec. 1, Fig. 1).  Evaluating it per event re-does every
// observable-dependent node while parameter-only branches stay cached
// (Sec. 4).  Here the graph is compiled once: PDFs in dependency order,
// observables bound to SoA columns, each leaf's parameter-only constants
// (normalisation integral and its derivatives) assigned a slot in a per-set
// constant block filled once per parameter point, and each local parameter
// a gradient slot for the adjoint pass.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <set>

#include "rf_internal.h"

namespace rf {

namespace {

bool is_leaf(int k) {
  return k == GAUSS || k == EXPO || k == GAUSSEXP || k == CHEB || k == POLY || k == POISSON || k == EXPR;
}
bool is_pdf(int k) { return is_leaf(k) || k == SUM || k == PROD; }  // EXTEND: only as the root

std::string kind_name(int k) {
  static const char* names[] = {"OBS", "PARAM", "GAUSS", "EXP", "GAUSSEXP", "CHEB", "POLY", "SUM", "PROD",
                                "POISSON", "EXTEND", "EXPR"};
  return (k >= 0 && k <= 11) ? names[k] : "?";
}

// An RF_EXPR program as a whole: known operations, arguments in range
// (n_par parameters, n_consts constants), a stack that never underflows nor
// holds more than kExprStack values, and exactly one value at the end.
const char* check_expr(const rf_expr& e, int n_par) {
  if (e.n_ops < 1 || e.n_ops > kExprMaxOps || !e.ops) return "program length must be 1..64";
  if (e.n_consts < 0 || e.n_consts > kExprMaxConsts || (e.n_consts > 0 && !e.consts)) return "at most 16 constants";
  int depth = 0;
  for (int i = 0; i < e.n_ops; ++i) {
    const int code = e.ops[i] & 0xff, arg = e.ops[i] >> 8;
    if (code < RF_EX_X || code > RF_EX_POW) return "unknown operation";
    if (code == RF_EX_PAR && (arg < 0 || arg >= n_par)) return "parameter index out of range";
    if (code == RF_EX_CONST && (arg < 0 || arg >= e.n_consts)) return "constant index out of range";
    if (code > RF_EX_CONST && arg != 0) return "operation with an argument";
    if (code <= RF_EX_CONST) {
      ++depth;
    } else if (code >= RF_EX_NEG && code <= RF_EX_LOG) {
      if (depth < 1) return "stack underflow";
    } else {
      if (depth < 2) return "stack underflow";
      --depth;
    }
    if (depth > kExprStack) return "stack deeper than 16";
  }
  return depth == 1 ? nullptr : "the program must leave exactly one value";
}

}  // namespace

rf_status compile_model(const rf_node* nodes, int n, int root, Model* m, const rf_expr* exprs, int n_exprs) {
  char buf[256];
  auto fail = [&](const char* why, int i) {
    std::snprintf(buf, sizeof buf, "rf_model_create: node %d: %s", i, why);
    set_error(buf);
    return RF_E_INVALID;
  };
  if (!nodes || n <= 0 || n > kMaxNodes) return fail("node count must be 1..64", -1);
  if (root < 0 || root >= n) return fail("root index out of range", root);
  m->nodes.assign(nodes, nodes + n);

  std::vector<int> column(n, -1), free_index(n, -1);
  int n_obs = 0, n_free = 0;
  for (int i = 0; i < n; ++i) {
    const rf_node& nd = nodes[i];
    if (nd.kind < 0 || nd.kind > 11) return fail("unknown kind", i);
    if (nd.n_in < 0 || nd.n_in > 8) return fail("n_in must be 0..8", i);
    for (int j = 0; j < nd.n_in; ++j)
      if (nd.in[j] < 0 || nd.in[j] >= n || nd.in[j] == i) return fail("input index out of range", i);
    if (nd.kind == OBS) {
      if (nd.n_in != 0) return fail("OBS takes no inputs", i);
      if (!(nd.lo < nd.hi) || !std::isfinite(nd.lo) || !std::isfinite(nd.hi)) return fail("OBS range must be finite, lo < hi", i);
      column[i] = n_obs++;
      m->obs_lo.push_back(nd.lo);
      m->obs_hi.push_back(nd.hi);
    } else if (nd.kind == PARAM) {
      if (nd.n_in != 0) return fail("PARAM takes no inputs", i);
      if (nd.is_free) {
        free_index[i] = n_free++;
        m->free_node.push_back(i);
        m->theta_default.push_back(nd.value);
        m->lo.push_back(nd.lo);
        m->hi.push_back(nd.hi);
      }
    } else if (is_leaf(nd.kind)) {
      const int want = nd.kind == GAUSS ? 3 : nd.kind == EXPO || nd.kind == POISSON ? 2 : nd.kind == GAUSSEXP ? 4 : -1;
      if (want > 0 && nd.n_in != want) return fail("wrong number of inputs for this pdf", i);
      if (want < 0 && (nd.n_in < 1 || nd.n_in > 1 + kMaxPar))
        return fail("CHEB/POLY/EXPR take an observable and 0..7 parameters", i);
      if (nodes[nd.in[0]].kind != OBS) return fail("input 0 of a pdf must be an OBS node", i);
      for (int j = 1; j < nd.n_in; ++j)
        if (nodes[nd.in[j]].kind != PARAM) return fail("pdf parameters must be PARAM nodes", i);
      if (nd.kind == POISSON) {
        const rf_node& ob = nodes[nd.in[0]];
        if (!(ob.lo >= 0.0) || ob.lo != std::floor(ob.lo) || ob.hi != std::floor(ob.hi) ||
            ob.hi - ob.lo > kMaxPoissonRange)
          return fail("a POISSON observable needs integer bounds 0 <= lo < hi <= lo + 100000", i);
      }
    } else if (nd.kind == EXTEND) {
      if (i != root) return fail("EXTEND must be the root", i);
      if (nd.n_in != 2 || !is_pdf(nodes[nd.in[0]].kind) || nodes[nd.in[1]].kind != PARAM)
        return fail("EXTEND takes [pdf, expected count]", i);
    } else if (nd.kind == SUM) {
      if (nd.n_in < 3 || nd.n_in % 2 == 0) return fail("SUM takes n pdfs and n-1 fractions, 2 <= n <= 4", i);
      const int nc = (nd.n_in + 1) / 2;
      for (int j = 0; j < nd.n_in; ++j) {
        const int k = nodes[nd.in[j]].kind;
        if (j < nc && !is_pdf(k)) return fail("SUM component is not a pdf", i);
        if (j >= nc && k != PARAM) return fail("SUM fraction is not a PARAM", i);
      }
    } else if (nd.kind == PROD) {
      if (nd.n_in < 1) return fail("PROD needs at least one factor", i);
      for (int j = 0; j < nd.n_in; ++j)
        if (!is_pdf(nodes[nd.in[j]].kind)) return fail("PROD factor is not a pdf", i);
    }
  }
  if (n_obs > kMaxObs) return fail("more than 8 observables", -1);
  if (n_free > kMaxFree) return fail("more than 16 free parameters", -1);
  // An EXTEND root: the program is its pdf; the extended term is per set.
  int ext = 0, ext_free = -1;
  double ext_fixed = 0.0;
  if (nodes[root].kind == EXTEND) {
    ext = 1;
    ext_free = free_index[nodes[root].in[1]];
    ext_fixed = nodes[nodes[root].in[1]].value;
    root = nodes[root].in[0];
  }
  if (!is_pdf(nodes[root].kind)) return fail("root is not a pdf", root);

  // Dependency order of the PDFs under the root (children first); cycle check.
  std::vector<int> state(n, 0), order;
  std::function<bool(int)> visit = [&](int i) -> bool {
    if (state[i] == 2) return true;
    if (state[i] == 1) return false;
    state[i] = 1;
    const rf_node& nd = nodes[i];
    if (nd.kind == SUM || nd.kind == PROD) {
      const int nc = nd.kind == SUM ? (nd.n_in + 1) / 2 : nd.n_in;
      for (int j = 0; j < nc; ++j)
        if (!visit(nd.in[j])) return false;
    }
    state[i] = 2;
    order.push_back(i);
    return true;
  };
  if (!visit(root)) return fail("the graph has a cycle", root);
  if ((int)order.size() > kMaxPdf) return fail("more than 24 pdf nodes", root);

  // Observable sets: SUM components must agree, PROD factors must be disjoint.
  std::vector<std::set<int>> obs(n);
  for (int i : order) {
    const rf_node& nd = nodes[i];
    if (is_leaf(nd.kind)) {
      obs[i] = {column[nd.in[0]]};
    } else if (nd.kind == SUM) {
      const int nc = (nd.n_in + 1) / 2;
      obs[i] = obs[nd.in[0]];
      for (int j = 1; j < nc; ++j)
        if (obs[nd.in[j]] != obs[i]) return fail("SUM components depend on different observables", i);
    } else {
      for (int j = 0; j < nd.n_in; ++j)
        for (int o : obs[nd.in[j]]) {
          if (obs[i].count(o)) return fail("PROD factors share an observable", i);
          obs[i].insert(o);
        }
    }
  }

  // Emit the program.
  Program& P = m->prog;
  std::memset(&P, 0, sizeof P);
  P.n_pdf = (int)order.size();
  P.n_obs = n_obs;
  P.n_free = n_free;
  P.ext = ext;
  P.ext_free = ext_free;
  P.ext_fixed = ext_fixed;
  std::vector<int> prog_index(n, -1);
  int cofs = 0, slot = 0;
  for (int pi = 0; pi < P.n_pdf; ++pi) {
    const int i = order[pi];
    prog_index[i] = pi;
    const rf_node& nd = nodes[i];
    PNode& q = P.node[pi];
    for (int j = 0; j < 8; ++j) q.child[j] = -1;
    for (int j = 0; j < kMaxPar; ++j) { q.pfree[j] = -1; q.pfixed[j] = 0.0; }
    q.kind = (int8_t)nd.kind;
    q.col = -1;
    q.n_child = 0;
    q.n_par = 0;
    q.lo = q.hi = 0.0;
    if (is_leaf(nd.kind)) {
      const rf_node& ob = nodes[nd.in[0]];
      q.col = (int8_t)column[nd.in[0]];
      q.lo = ob.lo;
      q.hi = ob.hi;
      q.n_par = (int8_t)(nd.n_in - 1);
      for (int j = 1; j < nd.n_in; ++j) {
        q.pfree[j - 1] = (int8_t)free_index[nd.in[j]];
        q.pfixed[j - 1] = nodes[nd.in[j]].value;
      }
    } else if (nd.kind == SUM) {
      const int nc = (nd.n_in + 1) / 2;
      q.n_child = (int8_t)nc;
      q.n_par = (int8_t)(nc - 1);
      for (int j = 0; j < nc; ++j) q.child[j] = (int8_t)prog_index[nd.in[j]];
      for (int j = 0; j < nc - 1; ++j) {
        q.pfree[j] = (int8_t)free_index[nd.in[nc + j]];
        q.pfixed[j] = nodes[nd.in[nc + j]].value;
      }
    } else {
      q.n_child = (int8_t)nd.n_in;
      for (int j = 0; j < nd.n_in; ++j) q.child[j] = (int8_t)prog_index[nd.in[j]];
    }
    q.cofs = (int16_t)cofs;
    cofs += const_size(nd.kind, q.n_par);
    q.slot0 = (int16_t)slot;
    for (int j = 0; j < q.n_par; ++j) {
      if (slot >= kMaxSlots) return fail("more than 32 gradient slots", i);
      P.slot_free[slot++] = q.pfree[j];
    }
    if (nd.kind == GAUSSEXP) P.has_slow = 1;
  }
  if (cofs > kMaxConst) return fail("constant block too large", root);
  P.n_const = cofs;
  P.n_slots = slot;

  // RF_EXPR programs into the model's pools, in the order given.
  std::vector<int> has_prog(n, 0);
  int ops_used = 0, consts_used = 0;
  for (int e = 0; e < n_exprs; ++e) {
    const rf_expr& ex = exprs[e];
    if (ex.node < 0 || ex.node >= n || nodes[ex.node].kind != EXPR) return fail("program for a node that is not EXPR", ex.node);
    if (has_prog[ex.node]) return fail("two programs for one EXPR node", ex.node);
    has_prog[ex.node] = 1;
    if (const char* why = check_expr(ex, nodes[ex.node].n_in - 1)) return fail(why, ex.node);
    if (ops_used + ex.n_ops > kExprPoolOps || consts_used + ex.n_consts > kExprPoolConsts)
      return fail("programs longer than 128 operations or 32 constants in all", ex.node);
    if (prog_index[ex.node] >= 0) {
      PNode& q = P.node[prog_index[ex.node]];
      q.ex_op0 = (int16_t)ops_used;
      q.ex_nops = (int16_t)ex.n_ops;
      q.ex_c0 = (int16_t)consts_used;
    }
    for (int k = 0; k < ex.n_ops; ++k) P.ex_ops[ops_used + k] = ex.ops[k];
    for (int k = 0; k < ex.n_consts; ++k) P.ex_consts[consts_used + k] = ex.consts[k];
    ops_used += ex.n_ops;
    consts_used += ex.n_consts;
  }
  for (int pi = 0; pi < P.n_pdf; ++pi)
    if (P.node[pi].kind == EXPR) {
      if (!has_prog[order[pi]]) return fail("EXPR node without a program (rf_model_create_expr)", order[pi]);
      P.has_expr = 1;
    }

  // Signature and specialised shape.
  std::function<std::string(int)> sig = [&](int i) -> std::string {
    const rf_node& nd = nodes[i];
    std::string s = kind_name(nd.kind);
    if (nd.kind == CHEB || nd.kind == POLY) s += std::to_string(nd.n_in - 1);
    if (nd.kind == SUM || nd.kind == PROD) {
      const int nc = nd.kind == SUM ? (nd.n_in + 1) / 2 : nd.n_in;
      s += "(";
      for (int j = 0; j < nc; ++j) s += (j ? "," : "") + sig(nd.in[j]);
      s += ")";
    }
    return s;
  };
  m->signature = sig(root);
  m->extended = ext != 0;
  m->shape = SHAPE_GENERIC;
  if (m->signature == "SUM(GAUSS,POLY1)") m->shape = SHAPE_SUM_GAUSS_POLY1;
  if (m->signature == "SUM(GAUSSEXP,CHEB2)") m->shape = SHAPE_SUM_GAUSSEXP_CHEB2;
  if (m->signature == "PROD(SUM(GAUSS,CHEB1),SUM(GAUSSEXP,CHEB2),POLY2)") m->shape = SHAPE_PROD3;
  m->detected_shape = m->shape;

  // Generation factors: the root, or the factors of (nested) PRODs at the root.
  std::function<void(int)> factors = [&](int i) {
    if (nodes[i].kind == PROD)
      for (int j = 0; j < nodes[i].n_in; ++j) factors(nodes[i].in[j]);
    else
      m->gen_factors.push_back(prog_index[i]);
  };
  factors(root);
  for (int f : m->gen_factors)
    if (obs[order[f]].size() != 1) m->gen_factors.clear();  // toys need 1-D factors
  return RF_OK;
}

}  // namespace rf
