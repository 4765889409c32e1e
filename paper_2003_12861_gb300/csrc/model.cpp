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

bool is_leaf(int k) { return k == GAUSS || k == EXPO || k == GAUSSEXP || k == CHEB || k == POLY || k == POISSON; }
bool is_pdf(int k) { return is_leaf(k) || k == SUM || k == PROD; }  // EXTEND: only as the root

std::string kind_name(int k) {
  static const char* names[] = {"OBS", "PARAM", "GAUSS", "EXP", "GAUSSEXP", "CHEB", "POLY", "SUM", "PROD",
                                "POISSON", "EXTEND"};
  return (k >= 0 && k <= 10) ? names[k] : "?";
}

}  // namespace

rf_status compile_model(const rf_node* nodes, int n, int root, Model* m) {
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
    if (nd.kind < 0 || nd.kind > 10) return fail("unknown kind", i);
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
      if (want < 0 && (nd.n_in < 1 || nd.n_in > 1 + kMaxPar)) return fail("CHEB/POLY take an observable and 0..7 coefficients", i);
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
