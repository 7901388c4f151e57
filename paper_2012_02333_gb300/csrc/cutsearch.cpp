// Exact cut search (Sec. 4.1, Eqs. 4-15) by branch and bound on the host.
//
// The circuit becomes the DAG of Sec. 4.1.1: multi-qubit gates are vertices
// (in circuit order), the qubit wires between consecutive multi-qubit gates
// are directed edges, single-qubit gates are ignored; w_v counts the original
// input qubits whose first multi-qubit gate is v.  Vertices are assigned to
// subcircuits in order, vertex k to one of 0 .. min(k, n_C - 1) (Eq. 12).  When
// vertex v is placed, every edge into it is decided (edges run from earlier
// to later vertices), so alpha (Eq. 4), rho (Eq. 5), O (Eq. 6) and K (Eq. 13)
// are updated incrementally.  A branch is cut when a subcircuit's width
// alpha + rho exceeds D (Eq. 9; both only grow) or when 4^K (n_C - 1), a lower
// bound of the cost since every term of Eq. 14 is at least 4^K, already
// reaches the best complete cost.  The cost L = 4^K sum_{c=2}^{n_C}
// prod_{i<=c} 2^{f_i} (Eq. 14) is a sum of powers of two kept exactly in 128
// bits; the first assignment in vertex order among those of least cost is
// returned.  This replaces the paper's MIP solver for the small circuits an
// exhaustive search can handle; a node budget bounds the work.
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"

namespace cutqc {

namespace {

using u128 = unsigned __int128;

struct Search {
  int nV = 0, nC = 0, D = 0;
  std::vector<int> w;
  std::vector<std::vector<int>> in_edges;   // per vertex: the earlier vertices with an edge into it
  std::vector<int> assign, alpha, rho, out;
  int K = 0;
  int64_t nodes = 0, max_nodes = 0;
  bool have = false, over_budget = false;
  u128 best = 0;
  std::vector<int> best_assign;
  int best_K = 0;

  static bool pow2_sum(u128& acc, int e) {
    if (e < 0 || e > 125) return false;
    const u128 t = u128(1) << e;
    if (acc > ~u128(0) - t) return false;
    acc += t;
    return true;
  }

  void leaf() {
    // Eq. 7 and Eq. 14
    u128 L = 0;
    int F = 0;
    bool ok = true;
    for (int c = 0; c < nC && ok; ++c) {
      F += alpha[c] + rho[c] - out[c];
      if (c >= 1) ok = pow2_sum(L, 2 * K + F);
    }
    if (!ok) return;
    if (!have || L < best) {
      have = true;
      best = L;
      best_assign = assign;
      best_K = K;
    }
  }

  void dfs(int v) {
    if (over_budget) return;
    if (++nodes > max_nodes) {
      over_budget = true;
      return;
    }
    if (v == nV) {
      leaf();
      return;
    }
    const int cmax = std::min(v + 1, nC);
    for (int c = 0; c < cmax; ++c) {
      alpha[c] += w[v];
      int cut = 0;
      for (int u : in_edges[v])
        if (assign[u] != c) {
          ++cut;
          ++out[assign[u]];
          ++rho[c];
        }
      K += cut;
      assign[v] = c;
      bool prune = alpha[c] + rho[c] > D;   // Eq. 9
      if (!prune && have) {
        // 4^K (n_C - 1) <= L for any completion
        const int e = 2 * K;
        prune = e > 120 || ((u128(1) << e) * u128(nC > 1 ? nC - 1 : 1) >= best);
      }
      if (!prune) dfs(v + 1);
      K -= cut;
      for (int u : in_edges[v])
        if (assign[u] != c) {
          --out[assign[u]];
          --rho[c];
        }
      alpha[c] -= w[v];
      assign[v] = -1;
      if (over_budget) return;
    }
  }
};

struct Call {
  const cutqc_gate* gates;
  int32_t n_gates, n_qubits, max_width, max_subcircuits;
  int64_t max_nodes;
  int32_t* cluster;
  int32_t* n_vertices;
  int32_t* n_cuts;
  double* cost;
};

void run(void* ctx) {
  const Call& a = *static_cast<const Call*>(ctx);
  if (a.n_qubits < 1 || a.n_qubits > 4096) fail(CUTQC_ERR_UNSUPPORTED, "need 1 <= n_qubits <= 4096");
  if (a.n_gates < 0 || (a.n_gates && !a.gates)) fail(CUTQC_ERR_ARG, "bad gate list");
  if (!a.cluster || !a.n_vertices || !a.n_cuts || !a.cost) fail(CUTQC_ERR_ARG, "NULL output");
  if (a.max_width < 1) fail(CUTQC_ERR_ARG, "max_width < 1");
  if (a.max_subcircuits < 1 || a.max_subcircuits > 16) fail(CUTQC_ERR_UNSUPPORTED, "need 1 <= n_C <= 16");
  if (a.max_nodes < 1) fail(CUTQC_ERR_ARG, "max_nodes < 1");
  Search S;
  S.nC = a.max_subcircuits;
  S.D = a.max_width;
  S.max_nodes = a.max_nodes;
  std::vector<int> last(a.n_qubits, -1);
  for (int g = 0; g < a.n_gates; ++g) {
    const cutqc_gate& gt = a.gates[g];
    if (gt.op < CUTQC_GATE_H || gt.op > CUTQC_GATE_CP) fail(CUTQC_ERR_ARG, "unknown gate op");
    if (gt.q0 < 0 || gt.q0 >= a.n_qubits) fail(CUTQC_ERR_SHAPE, "gate qubit out of range");
    if (gt.op < CUTQC_GATE_CZ) continue;   // single-qubit gates do not affect connectivity
    if (gt.q1 < 0 || gt.q1 >= a.n_qubits || gt.q1 == gt.q0) fail(CUTQC_ERR_SHAPE, "gate qubit out of range");
    const int v = S.nV++;
    S.w.push_back(0);
    S.in_edges.emplace_back();
    for (int q : {gt.q0, gt.q1}) {
      if (last[q] < 0)
        ++S.w[v];
      else
        S.in_edges[v].push_back(last[q]);
      last[q] = v;
    }
  }
  S.assign.assign(S.nV, -1);
  S.alpha.assign(S.nC, 0);
  S.rho.assign(S.nC, 0);
  S.out.assign(S.nC, 0);
  S.dfs(0);
  if (S.over_budget) fail(CUTQC_ERR_UNSUPPORTED, "cut search exceeded max_nodes");
  if (!S.have) fail(CUTQC_ERR_UNSUPPORTED, "no assignment fits the device width");
  for (int v = 0; v < S.nV; ++v) a.cluster[v] = S.best_assign[v];
  *a.n_vertices = S.nV;
  *a.n_cuts = S.best_K;
  *a.cost = (double)S.best;
}

}  // namespace

}  // namespace cutqc

extern "C" int cutqc_cut_search(const cutqc_gate* gates, int32_t n_gates, int32_t n_qubits, int32_t max_width,
                                int32_t max_subcircuits, int64_t max_nodes, int32_t* cluster, int32_t* n_vertices,
                                int32_t* n_cuts, double* cost) {
  cutqc::Call call{gates, n_gates, n_qubits, max_width, max_subcircuits, max_nodes, cluster, n_vertices,
                   n_cuts, cost};
  return cutqc::run_guarded(&cutqc::run, &call);
}
