"""Plain FP64 reconstruction: full definition, dynamic definition, gradient.
TEST INFRASTRUCTURE ONLY.

The method reaches exactly (up to rounding order) a result with a plain
definition (Sec. 3.2.3 and Sec. 3.3: the uncut distribution is the sum over
all 4^K cut-edge Pauli assignments of the Kronecker products of the
subcircuits' attributed vectors):

    p(x) = 2^-K  sum_{e in {I,X,Y,Z}^K}  prod_c  T_c[e|c][x|c]

where e|c is subcircuit c's row (a, b): its init-slot digits and its
measurement-slot digits read off e, and x|c its effective output bits.  This
module writes that sum out term by term, with no blocking, reordering or
bipartition.  Dynamic definition (Algorithm 1, Sec. 4.3) is the same sum over
merged tensors; the gradient is the chain rule of the same sum.

Structure arguments are the subcircuits of ``circuits.CutCircuit`` (or any
objects with k_in/k_out/n_eff, in_cut, out_cut, out_qubit attributes).
"""
from __future__ import annotations

import itertools
from typing import List, Sequence

import numpy as np


def _digits(e: int, K: int) -> List[int]:
    """Base-4 digits of e, cut 0 most significant."""
    return [(e >> (2 * (K - 1 - k))) & 3 for k in range(K)]


def row_of(sub, digits: Sequence[int]) -> int:
    """Subcircuit row index (a * 4^k_out + b) that the cut assignment selects."""
    a = 0
    for c in sub.in_cut:
        a = 4 * a + digits[c]
    b = 0
    for c in sub.out_cut:
        b = 4 * b + digits[c]
    return a * 4 ** sub.k_out + b


def _flat(T, sub):
    return np.asarray(T, np.float64).reshape(4 ** sub.k_in * 4 ** sub.k_out, -1)


def _place(vecs, subs, positions, n_out):
    """Kronecker product of per-subcircuit vectors laid out in output order:
    `positions[c][i]` is the output bit position (0 = most significant) of
    subcircuit c's local bit i."""
    prod = np.ones(())
    axes = []
    for v, s, pos in zip(vecs, subs, positions):
        prod = np.multiply.outer(prod, v.reshape([2] * len(pos)))
        axes.extend(pos)
    # axis j of prod is output position axes[j]; transpose into output order
    order = np.argsort(axes)
    return prod.transpose(order).reshape(-1) if n_out else prod.reshape(-1)


def fd_full(subs, tensors, n_qubits: int, n_cuts: int, terms=None) -> np.ndarray:
    """Every one of the 2^n probabilities by the plain sum (Sec. 3.2.3, 3.3).
    `terms` restricts the sum to a subset of the cut assignments e (used only
    to time a sample of the terms, the runtime-scaling method of Sec. 5.2)."""
    K = n_cuts
    Ts = [_flat(T, s) for T, s in zip(tensors, subs)]
    positions = [list(s.out_qubit) for s in subs]
    out = np.zeros(2 ** n_qubits)
    for e in (range(4 ** K) if terms is None else terms):
        dg = _digits(e, K)
        vecs = [T[row_of(s, dg)] for T, s in zip(Ts, subs)]
        out += _place(vecs, subs, positions, n_qubits)
    return out * 2.0 ** -K


def fd_entries(subs, tensors, n_qubits: int, n_cuts: int, xs) -> np.ndarray:
    """p(x) for selected global indices x (a list of Python ints, any n),
    each by the plain sum over all 4^K terms."""
    K = n_cuts
    Ts = [_flat(T, s) for T, s in zip(tensors, subs)]
    rows = np.array([[row_of(s, _digits(e, K)) for s in subs] for e in range(4 ** K)])
    out = np.empty(len(xs))
    for i, x in enumerate(xs):
        bits = [(int(x) >> (n_qubits - 1 - q)) & 1 for q in range(n_qubits)]
        acc = np.ones(4 ** K)
        for c, (T, s) in enumerate(zip(Ts, subs)):
            xc = 0
            for q in s.out_qubit:
                xc = 2 * xc + bits[q]
            acc = acc * T[rows[:, c], xc]
        out[i] = acc.sum() * 2.0 ** -K
    return out


def merge(sub, T, roles) -> np.ndarray:
    """Merged tensor of one subcircuit for a DD recursion (Algorithm 1:
    subcircuit states that share their merged qubits' values are grouped):
    zoomed output qubits are fixed at their bit, merged output qubits summed
    out, active output qubits kept (in increasing qubit order).  roles[q] is
    0 active, 1 merged, 2 zoomed at 0, 3 zoomed at 1."""
    Tf = _flat(T, sub)
    R = Tf.shape[0]
    arr = Tf.reshape([R] + [2] * sub.n_eff)
    idx = [slice(None)]
    keep = []
    for i, q in enumerate(sub.out_qubit):
        r = roles[q]
        if r == 2:
            idx.append(0)
        elif r == 3:
            idx.append(1)
        else:
            idx.append(slice(None))
            keep.append(r)
    arr = arr[tuple(idx)]
    # sum the merged axes (axis 1 + j for keep[j] == 1)
    merged_axes = tuple(1 + j for j, r in enumerate(keep) if r == 1)
    if merged_axes:
        arr = arr.sum(axis=merged_axes)
    return arr.reshape(R, -1)


def dd_bins(subs, tensors, n_qubits: int, n_cuts: int, roles) -> np.ndarray:
    """The 2^#active bin probabilities of one DD recursion: the plain sum over
    the merged tensors.  Bin index: active qubits in increasing order, the
    lowest-numbered active qubit most significant."""
    K = n_cuts
    active = [q for q in range(n_qubits) if roles[q] == 0]
    rank = {q: i for i, q in enumerate(active)}
    Ms = [merge(s, T, roles) for s, T in zip(subs, tensors)]
    positions = [[rank[q] for q in s.out_qubit if roles[q] == 0] for s in subs]
    out = np.zeros(2 ** len(active))
    for e in range(4 ** K):
        dg = _digits(e, K)
        vecs = [M[row_of(s, dg)] for M, s in zip(Ms, subs)]
        out += _place(vecs, subs, positions, len(active))
    return out * 2.0 ** -K


def initial_roles(n_qubits: int, n_active: int) -> List[int]:
    """First recursion: the n_active lowest-numbered qubits active, the rest
    merged (the paper lets the user choose; this is the fixed reading)."""
    return [0 if q < n_active else 1 for q in range(n_qubits)]


def zoom_roles(parent_roles, bin_index: int, n_active: int) -> List[int]:
    """Roles of the recursion that zooms into `bin_index` of a parent
    recursion (Algorithm 1): earlier zoomed qubits stay zoomed, the parent's
    active qubits become zoomed at the bin's bits, and the next
    min(n_active, #merged) lowest-numbered merged qubits become active."""
    roles = list(parent_roles)
    active = [q for q, r in enumerate(roles) if r == 0]
    na = len(active)
    for i, q in enumerate(active):
        bit = (bin_index >> (na - 1 - i)) & 1
        roles[q] = 3 if bit else 2
    merged = [q for q, r in enumerate(roles) if r == 1]
    for q in merged[:n_active]:
        roles[q] = 0
    return roles


def dd_run(subs, tensors, n_qubits: int, n_cuts: int, n_active: int,
           recursions: int, strategy: str = "bfs", follow=None, follow_tol: float = 0.0):
    """Algorithm 1.  Each recursion after the first zooms into one bin taken
    from the list of all bins so far: "bfs" takes the heaviest bin over all
    recursions that has not been zoomed yet and still has merged qubits; "dfs"
    takes the heaviest bin of the latest recursion.  Ties go to the earlier
    recursion, then the lower bin index.  Returns a list of dicts with the
    roles, the bins and the (recursion, bin) that was zoomed into.

    Near ties (the paper ranks bins but says nothing about values that differ
    only by rounding): `follow` may list, per recursion, the (recursion, bin)
    another implementation zoomed into.  Where that bin is eligible and its
    value is within `follow_tol` of the heaviest eligible value, it is taken
    instead and the recursion's dict says so ("followed": True), so a run can
    keep comparing after a choice that rounding alone decided; any other
    choice is ignored."""
    out = []
    expanded = set()
    roles = initial_roles(n_qubits, n_active)
    parent = None
    for r in range(recursions):
        followed = False
        if r > 0:
            best = None
            eligible = {}
            cands = range(len(out)) if strategy == "bfs" else [len(out) - 1]
            for ri in cands:
                rec = out[ri]
                if not any(v == 1 for v in rec["roles"]):
                    continue
                for bi, v in enumerate(rec["bins"]):
                    if (ri, bi) in expanded:
                        continue
                    eligible[(ri, bi)] = v
                    if best is None or v > best[0]:
                        best = (v, ri, bi)
            if best is None:
                break
            _, ri, bi = best
            if follow is not None and r < len(follow) and follow[r] is not None:
                want = tuple(follow[r])
                if want != (ri, bi) and want in eligible and eligible[want] >= best[0] - follow_tol:
                    ri, bi = want
                    followed = True
            expanded.add((ri, bi))
            roles = zoom_roles(out[ri]["roles"], bi, n_active)
            parent = (ri, bi)
        bins = dd_bins(subs, tensors, n_qubits, n_cuts, roles)
        out.append({"roles": roles, "bins": bins, "parent": parent, "followed": followed})
    return out


def dd_entries(subs, slab, n_qubits: int, n_cuts: int, roles, bins, cache=None) -> np.ndarray:
    """Selected bins of one DD recursion by the plain sum over merged tensors
    (Algorithm 1), for sizes where neither the merged tensors nor the bins
    can be formed whole.  slab(c, a) yields the entries of subcircuit c's
    tensor whose active outputs read `a` (bits in output order, the first
    active output most significant) and whose zoomed outputs read their fixed
    bits: pieces (first row, array [rows of the piece][any number of the
    merged outputs' entries]) covering every row and every merged entry once.
    The merged value of a row is the sum over its merged entries; a bin is
    2^-K sum_e prod_c (merged value of subcircuit c at row e|c and its active
    bits of the bin).  Bin index as dd_bins.  `cache` (a dict, optional)
    keeps merged values between calls, keyed by the subcircuit, the roles of
    its outputs and `a`."""
    K = n_cuts
    active = [q for q in range(n_qubits) if roles[q] == 0]
    rank = {q: i for i, q in enumerate(active)}
    na = len(active)
    rows = np.array([[row_of(s, _digits(e, K)) for s in subs] for e in range(4 ** K)], dtype=np.int64)
    merged = {} if cache is None else cache
    out = np.empty(len(bins))
    for i, b in enumerate(bins):
        acc = np.ones(4 ** K)
        for c, s in enumerate(subs):
            a = 0
            for q in s.out_qubit:
                if roles[q] == 0:
                    a = 2 * a + ((int(b) >> (na - 1 - rank[q])) & 1)
            key = (c, tuple(roles[q] for q in s.out_qubit), a)
            if key not in merged:
                m = np.zeros(4 ** s.k_in * 4 ** s.k_out)
                for r0, piece in slab(c, a):
                    piece = np.asarray(piece)
                    m[r0:r0 + piece.shape[0]] += piece.sum(axis=1, dtype=np.float64)
                merged[key] = m
            acc = acc * merged[key][rows[:, c]]
        out[i] = acc.sum() * 2.0 ** -K
    return out


def grad(subs, tensors, n_qubits: int, n_cuts: int, G: np.ndarray):
    """dL/dT_c for L = sum_x G(x) p(x), by the chain rule applied to the plain
    sum: dL/dT_c[row][x_c] = 2^-K sum_{e: e|c = row} sum_{x: x|c = x_c}
    G(x) prod_{c' != c} T_c'[e|c'][x|c']."""
    K = n_cuts
    Ts = [_flat(T, s) for T, s in zip(tensors, subs)]
    grads = [np.zeros_like(T) for T in Ts]
    positions = [list(s.out_qubit) for s in subs]
    Gt = np.asarray(G, np.float64).reshape([2] * n_qubits)
    for e in range(4 ** K):
        dg = _digits(e, K)
        rows = [row_of(s, dg) for s in subs]
        for c, s in enumerate(subs):
            vecs = [Ts[j][rows[j]] if j != c else np.ones(2 ** s.n_eff) for j in range(len(subs))]
            w = _place(vecs, subs, positions, n_qubits).reshape([2] * n_qubits) * Gt
            other = tuple(q for q in range(n_qubits) if q not in set(s.out_qubit))
            gc = w.sum(axis=other) if other else w
            # remaining axes are subcircuit c's qubits in increasing order = local order
            grads[c][rows[c]] += gc.reshape(-1)
    return [g * 2.0 ** -K for g in grads]


def grad_entry(subs, tensors, n_qubits: int, n_cuts: int, c: int, row: int, xc: int, G_of) -> float:
    """One entry dL/dT_c[row][xc] of the chain rule above, for large n: the
    sum over the cut assignments e with e|c = row and over the outputs x with
    x|c = xc, G given as a function of an array of global indices."""
    K = n_cuts
    Ts = [_flat(T, s) for T, s in zip(tensors, subs)]
    others = [j for j in range(len(subs)) if j != c]
    # global index contribution of subcircuit c's fixed bits
    base = 0
    sc = subs[c]
    for i, q in enumerate(sc.out_qubit):
        if (xc >> (sc.n_eff - 1 - i)) & 1:
            base |= 1 << (n_qubits - 1 - q)
    total = 0.0
    for e in range(4 ** K):
        dg = _digits(e, K)
        if row_of(sc, dg) != row:
            continue
        # Kronecker product of the other subcircuits' vectors over their bits
        vals = np.ones(1)
        gidx = np.full(1, base, dtype=np.int64)
        for j in others:
            s = subs[j]
            v = Ts[j][row_of(s, dg)]
            loc = np.arange(2 ** s.n_eff, dtype=np.int64)
            off = np.zeros(2 ** s.n_eff, dtype=np.int64)
            for i, q in enumerate(s.out_qubit):
                off |= ((loc >> (s.n_eff - 1 - i)) & 1) << (n_qubits - 1 - q)
            vals = np.multiply.outer(vals, v).reshape(-1)
            gidx = np.add.outer(gidx, off).reshape(-1)
        total += float(np.dot(vals, G_of(gidx)))
    return total * 2.0 ** -K


def maxcut_of(n_qubits: int, edges):
    """G_of for the MaxCut cost: the cut count of each global index."""
    def f(x):
        x = np.asarray(x, dtype=np.int64)
        c = np.zeros(x.shape)
        for (i, j) in edges:
            c += ((x >> (n_qubits - 1 - i)) & 1) != ((x >> (n_qubits - 1 - j)) & 1)
        return c
    return f


def maxcut_values(n_qubits: int, edges) -> np.ndarray:
    """C(x) = number of edges whose endpoints differ in x, for all 2^n x."""
    x = np.arange(2 ** n_qubits, dtype=np.int64)
    c = np.zeros(2 ** n_qubits)
    for (i, j) in edges:
        bi = (x >> (n_qubits - 1 - i)) & 1
        bj = (x >> (n_qubits - 1 - j)) & 1
        c += (bi != bj)
    return c
