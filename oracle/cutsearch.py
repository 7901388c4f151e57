"""Exact cut search by enumeration (Sec. 4.1, Eqs. 4-15).
TEST INFRASTRUCTURE ONLY.

The circuit is the DAG of Sec. 4.1.1: its multi-qubit gates are the vertices
(in circuit order), its qubit wires between consecutive multi-qubit gates are
the directed edges, single-qubit gates are ignored.  w_v counts the original
input qubits that enter v directly (the qubits whose first multi-qubit gate
is v).  For an assignment of vertices to subcircuits c = 0 .. n_C - 1:

  alpha_c = sum_{v in c} w_v                            (Eq. 4)
  rho_c   = #cut edges (a, b) with b in c               (Eq. 5)
  O_c     = #cut edges (a, b) with a in c               (Eq. 6)
  f_c     = alpha_c + rho_c - O_c                       (Eq. 7)
  d_c     = alpha_c + rho_c <= D                        (Eq. 9)
  K       = #cut edges                                  (Eq. 13)
  L       = 4^K sum_{c=2}^{n_C} prod_{i=1}^{c} 2^{f_i}  (Eq. 14, 1-based c)

and every vertex k (0-based) sits in a subcircuit <= k (Eq. 12).  `search`
enumerates every such assignment and returns the smallest L among those that
meet Eq. 9 (ties: the lexicographically smallest assignment in vertex order),
with Python integers, so L is exact.
"""
from __future__ import annotations

import itertools
from typing import List, Optional, Sequence, Tuple


def graph(n_qubits: int, gates) -> Tuple[List[int], List[Tuple[int, int]], List[int]]:
    """(vertex gate indices, edges as vertex-index pairs, w per vertex)."""
    verts = [gi for gi, g in enumerate(gates) if len(g.qubits) > 1]
    vid = {gi: k for k, gi in enumerate(verts)}
    last = [None] * n_qubits
    w = [0] * len(verts)
    edges = []
    for gi in verts:
        v = vid[gi]
        for q in gates[gi].qubits:
            if last[q] is None:
                w[v] += 1
            else:
                edges.append((last[q], v))
            last[q] = v
    return verts, edges, w


def cost(assign: Sequence[int], edges, w, n_C: int) -> dict:
    alpha = [0] * n_C
    rho = [0] * n_C
    O = [0] * n_C
    for v, c in enumerate(assign):
        alpha[c] += w[v]
    K = 0
    for a, b in edges:
        if assign[a] != assign[b]:
            K += 1
            rho[assign[b]] += 1
            O[assign[a]] += 1
    f = [alpha[c] + rho[c] - O[c] for c in range(n_C)]
    d = [alpha[c] + rho[c] for c in range(n_C)]
    L = 0
    for c in range(2, n_C + 1):
        prod = 1
        for i in range(1, c + 1):
            prod *= 2 ** f[i - 1]
        L += prod
    L *= 4 ** K
    return {"alpha": alpha, "rho": rho, "O": O, "f": f, "d": d, "K": K, "L": L}


def search(n_qubits: int, gates, D: int, n_C: int) -> Optional[dict]:
    verts, edges, w = graph(n_qubits, gates)
    best = None
    domains = [range(min(k + 1, n_C)) for k in range(len(verts))]   # Eq. 12
    for assign in itertools.product(*domains):
        r = cost(assign, edges, w, n_C)
        if max(r["d"]) > D:                                        # Eq. 9
            continue
        if best is None or r["L"] < best["L"]:
            best = dict(r, assign=list(assign))
    if best is not None:
        best["gates"] = verts
    return best
