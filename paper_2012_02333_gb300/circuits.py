"""Seeded circuit generators and the wire cutter: the structural inputs of the path.

This module is shared by the CUDA path (its GPU subcircuit simulator takes the
gate lists built here) and by the FP64 oracle.  It holds no arithmetic of the
method: gates are names with parameters (each simulator owns its own matrices),
and the cutter only decides which gates land in which subcircuit, where the
wire cuts fall, and how slots and output bits are numbered.

Conventions (paper Sec. 3.2: a circuit C(|q_0..q_{n-1}>; M_0..M_{n-1})):
  * qubit q0 is the most significant bit of every output index;
  * Pauli digits are I=0, X=1, Y=2, Z=3;
  * cut ids are numbered by (qubit, position along the wire); the joint Pauli
    assignment e over K cuts is the base-4 number with cut 0 most significant;
  * a subcircuit's init slots and measurement slots are each sorted by cut id,
    slot 0 is the most significant base-4 digit of its row index;
  * a subcircuit's effective output bits are sorted by global qubit, bit 0 is
    the most significant bit of its local output index x_c.

The benchmark families follow the paper's Sec. 5.3 (supremacy grid, AQFT, BV,
HWEA) plus QAOA MaxCut.  Every generator is seeded (numpy PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

# Gate names understood by both simulators.  Single-qubit: h x y z s sdg t
# sx sy sw rx ry rz.  Two-qubit: cz cx cp (controlled phase, param = angle).
ONE_QUBIT = ("h", "x", "y", "z", "s", "sdg", "t", "sx", "sy", "sw", "rx", "ry", "rz")
TWO_QUBIT = ("cz", "cx", "cp")


@dataclass(frozen=True)
class Gate:
    name: str
    qubits: Tuple[int, ...]
    params: Tuple[float, ...] = ()


@dataclass
class Circuit:
    n: int
    gates: List[Gate] = field(default_factory=list)
    family: str = ""

    def add(self, name: str, *qubits: int, params: Sequence[float] = ()) -> None:
        if name not in ONE_QUBIT + TWO_QUBIT:
            raise ValueError(f"unknown gate {name}")
        self.gates.append(Gate(name, tuple(int(q) for q in qubits), tuple(float(p) for p in params)))


# ---------------------------------------------------------------------------
# circuit families
# ---------------------------------------------------------------------------

def hwea(n: int, seed: int) -> Circuit:
    """Hardware-efficient ansatz on a linear chain: Ry(t)Rz(p) on every qubit,
    a CNOT chain q0->q1->...->q_{n-1}, then a second Ry Rz layer; angles U[0,2pi)."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, family="hwea")
    for q in range(n):
        c.add("ry", q, params=[rng.uniform(0, 2 * np.pi)])
        c.add("rz", q, params=[rng.uniform(0, 2 * np.pi)])
    for q in range(n - 1):
        c.add("cx", q, q + 1)
    for q in range(n):
        c.add("ry", q, params=[rng.uniform(0, 2 * np.pi)])
        c.add("rz", q, params=[rng.uniform(0, 2 * np.pi)])
    return c


def grid_cz_patterns(rows: int, cols: int) -> List[List[Tuple[int, int]]]:
    """Eight coupler layers that together activate every nearest-neighbour
    coupler of a rows x cols grid exactly once (horizontal and vertical
    couplers, four parity offsets each), in the alternating order used by
    Google-style random circuits."""
    def q(r, c):
        return r * cols + c
    pats = []
    for (pr, pc) in ((0, 0), (1, 1), (1, 0), (0, 1)):
        h = [(q(r, c), q(r, c + 1)) for r in range(rows) for c in range(cols - 1)
             if c % 2 == pc and r % 2 == pr]
        v = [(q(r, c), q(r + 1, c)) for r in range(rows - 1) for c in range(cols)
             if r % 2 == pr and c % 2 == pc]
        pats.append(h)
        pats.append(v)
    return pats


def supremacy_grid(rows: int, cols: int, depth: int, seed: int) -> Circuit:
    """Supremacy-style random circuit: H on all qubits, then `depth` cycles of
    (CZ layer from the 8-pattern cycle, then a random single-qubit gate from
    {sqrt X, sqrt Y, sqrt W} on every qubit, never the same gate twice in a row
    on one qubit)."""
    rng = np.random.default_rng(seed)
    n = rows * cols
    c = Circuit(n, family="supremacy")
    for q in range(n):
        c.add("h", q)
    pats = grid_cz_patterns(rows, cols)
    last = [-1] * n
    for d in range(depth):
        for (a, b) in pats[d % 8]:
            c.add("cz", a, b)
        for q in range(n):
            choices = [g for g in range(3) if g != last[q]]
            g = int(choices[rng.integers(len(choices))])
            last[q] = g
            c.add(("sx", "sy", "sw")[g], q)
    return c


def aqft(n: int, seed: int, max_order: int = 4) -> Circuit:
    """Approximate QFT on a seeded product input: Ry(t) on each qubit, then the
    QFT ladder keeping only controlled phases pi/2^m with m <= max_order."""
    rng = np.random.default_rng(seed)
    c = Circuit(n, family="aqft")
    for q in range(n):
        c.add("ry", q, params=[rng.uniform(0, np.pi)])
    for j in range(n):
        c.add("h", j)
        for k in range(j + 1, n):
            m = k - j
            if m <= max_order:
                c.add("cp", k, j, params=[np.pi / 2 ** m])
    return c


def bv(n: int, seed: int, secret: Optional[Sequence[int]] = None) -> Circuit:
    """Bernstein-Vazirani on n qubits: n-1 data qubits and the ancilla q_{n-1}.
    The output is the secret string on the data qubits and 1 on the ancilla."""
    rng = np.random.default_rng(seed)
    if secret is None:
        secret = [int(b) for b in rng.integers(0, 2, size=n - 1)]
    c = Circuit(n, family="bv")
    anc = n - 1
    c.add("x", anc)
    for q in range(n):
        c.add("h", q)
    for q, s in enumerate(secret):
        if s:
            c.add("cx", q, anc)
    for q in range(n):
        c.add("h", q)
    c.secret = list(secret)  # type: ignore[attr-defined]
    return c


def random_regular_graph(nodes: Sequence[int], degree: int, rng) -> List[Tuple[int, int]]:
    """A random simple graph on `nodes` in which every node has degree
    `degree`, by the pairing model retried until simple.  When len(nodes) *
    degree is odd no such graph exists; the last node then gets degree-1."""
    nodes = list(nodes)
    degs = [degree] * len(nodes)
    if (degree * len(nodes)) % 2:
        degs[-1] -= 1
    for _ in range(100000):
        stubs = [v for v, d in zip(nodes, degs) for _ in range(d)]
        rng.shuffle(stubs)
        edges = set()
        ok = True
        for i in range(0, len(stubs), 2):
            a, b = stubs[i], stubs[i + 1]
            if a == b or (min(a, b), max(a, b)) in edges:
                ok = False
                break
            edges.add((min(a, b), max(a, b)))
        if ok:
            return sorted(edges)
    raise RuntimeError("no simple graph with that degree sequence found")


def two_cluster_graph(n_per: int, seed: int, bridges: int = 2) -> Tuple[List[Tuple[int, int]], List[Tuple[int, int]], List[Tuple[int, int]]]:
    """Two random 3-regular clusters of n_per nodes (0..n_per-1 and
    n_per..2n_per-1) joined by `bridges` edges.  Returns (edges0, edges1, bridge)."""
    rng = np.random.default_rng(seed)
    e0 = random_regular_graph(range(n_per), 3, rng)
    e1 = random_regular_graph(range(n_per, 2 * n_per), 3, rng)
    h1 = len(e1) // 2
    first = {v for e in e1[:h1] for v in e}
    second = {v for e in e1[h1:] for v in e}
    both = sorted(first & second)      # cluster-1 nodes with ZZs before and after the bridges
    br = []
    used = set()
    while len(br) < bridges:
        a = int(rng.integers(n_per))
        b = int(both[rng.integers(len(both))])
        if a in used or b in used:
            continue
        used.update((a, b))
        br.append((a, b))
    return e0, e1, br


def qaoa_maxcut(n_per: int, seed: int, bridges: int = 2) -> Circuit:
    """QAOA p=1 for MaxCut on a two-cluster graph.  H on all, then per edge
    ZZ(gamma) = CX(i,j) Rz(2 gamma)(j) CX(i,j), then Rx(2 beta) on all;
    gamma, beta ~ U[0, pi].  Bridge edges sit mid-way through the cost layer so
    that each bridge ZZ cuts its qubit's wire twice."""
    rng = np.random.default_rng(seed)
    e0, e1, br = two_cluster_graph(n_per, seed, bridges)
    gamma = rng.uniform(0, np.pi)
    beta = rng.uniform(0, np.pi)
    n = 2 * n_per
    c = Circuit(n, family="qaoa")
    for q in range(n):
        c.add("h", q)
    h0, h1 = len(e0) // 2, len(e1) // 2
    order = e0[:h0] + e1[:h1] + br + e0[h0:] + e1[h1:]
    for (i, j) in order:
        c.add("cx", i, j)
        c.add("rz", j, params=[2 * gamma])
        c.add("cx", i, j)
    for q in range(n):
        c.add("rx", q, params=[2 * beta])
    c.edges = e0 + e1 + br  # type: ignore[attr-defined]
    c.bridges = br  # type: ignore[attr-defined]
    c.gamma, c.beta = gamma, beta  # type: ignore[attr-defined]
    return c


# ---------------------------------------------------------------------------
# cutting (Sec. 3.1 / 4.1: vertices = multi-qubit gates, edges = wires)
# ---------------------------------------------------------------------------

@dataclass
class Subcircuit:
    """One subcircuit: d local qubits (one per wire segment), its gates on local
    qubits, init slots (local qubit, cut id), measurement slots (local qubit,
    cut id) and effective outputs (local qubit, global qubit)."""
    d: int
    gates: List[Gate]
    in_slots: List[Tuple[int, int]]
    out_slots: List[Tuple[int, int]]
    outputs: List[Tuple[int, int]]

    @property
    def k_in(self) -> int:
        return len(self.in_slots)

    @property
    def k_out(self) -> int:
        return len(self.out_slots)

    @property
    def n_eff(self) -> int:
        return len(self.outputs)

    @property
    def in_cut(self) -> List[int]:
        return [c for _, c in self.in_slots]

    @property
    def out_cut(self) -> List[int]:
        return [c for _, c in self.out_slots]

    @property
    def out_qubit(self) -> List[int]:
        return [g for _, g in self.outputs]


@dataclass
class CutCircuit:
    circuit: Circuit          # the (possibly thinned) uncut circuit
    subs: List[Subcircuit]
    n_cuts: int
    cut_wires: List[Tuple[int, int]]   # cut id -> (qubit, position along the wire)

    @property
    def n(self) -> int:
        return self.circuit.n


def _wire_blocks(circ: Circuit, gate_block: Dict[int, int], home: Sequence[int]):
    """Per qubit: list of (gate index, block) for its gates, blocks resolved for
    single-qubit gates (they follow the preceding multi-qubit gate on the wire,
    else the following one, else the qubit's home block)."""
    per_q: List[List[int]] = [[] for _ in range(circ.n)]
    for gi, g in enumerate(circ.gates):
        for q in g.qubits:
            per_q[q].append(gi)
    out = []
    for q in range(circ.n):
        seq = per_q[q]
        blocks: List[Optional[int]] = [gate_block.get(gi) if len(circ.gates[gi].qubits) > 1 else None for gi in seq]
        prev = None
        for i, b in enumerate(blocks):
            if b is not None:
                prev = b
            elif prev is not None:
                blocks[i] = prev
        nxt = None
        for i in range(len(blocks) - 1, -1, -1):
            if blocks[i] is not None and len(circ.gates[seq[i]].qubits) > 1:
                nxt = blocks[i]
            elif blocks[i] is None:
                blocks[i] = nxt if nxt is not None else home[q]
        out.append(list(zip(seq, blocks)))
    return out


def _count_cuts(wires) -> int:
    k = 0
    for w in wires:
        for i in range(1, len(w)):
            if w[i][1] != w[i - 1][1]:
                k += 1
    return k


def cut_circuit(circ: Circuit, home: Sequence[int], max_cuts: Optional[int] = None,
                max_width: Optional[int] = None, policy: str = "min") -> CutCircuit:
    """Cut `circ` into the blocks given by `home` (qubit -> block).

    Multi-qubit gates whose qubits share a home block go there.  A crossing
    gate is tried in each of its qubits' blocks and placed where the total cut
    count K is smallest (ties: block of its first qubit); if that K exceeds
    `max_cuts`, or a subcircuit would exceed `max_width` qubits, the gate is
    dropped from the circuit.  With policy="first" a crossing gate is only
    tried in the block of its first qubit.  Either way it is (cut-by-construction: the returned circuit is the
    thinned one, so the cut is exact for it)."""
    gates = list(circ.gates)
    keep = [True] * len(gates)
    gate_block: Dict[int, int] = {}
    crossing = []
    for gi, g in enumerate(gates):
        if len(g.qubits) > 1:
            bs = {home[q] for q in g.qubits}
            if len(bs) == 1:
                gate_block[gi] = home[g.qubits[0]]
            else:
                crossing.append(gi)

    def thinned():
        c2 = Circuit(circ.n, [g for gi, g in enumerate(gates) if keep[gi]], circ.family)
        remap = {}
        j = 0
        for gi in range(len(gates)):
            if keep[gi]:
                remap[gi] = j
                j += 1
        gb = {remap[gi]: b for gi, b in gate_block.items() if keep[gi]}
        return c2, gb

    for gi in crossing:
        keep[gi] = False
    n_blocks = max(home) + 1
    for gi in crossing:
        best = None
        keep[gi] = True
        cand = gates[gi].qubits if policy == "min" else gates[gi].qubits[:1]
        for q in cand:
            b = home[q]
            gate_block[gi] = b
            c2, gb = thinned()
            wires = _wire_blocks(c2, gb, home)
            k = _count_cuts(wires)
            ok = max_cuts is None or k <= max_cuts
            if ok and max_width is not None:
                widths = [0] * n_blocks
                for qq, w in enumerate(wires):
                    prevb = None
                    for (_, bb) in w:
                        if bb != prevb:
                            widths[bb] += 1
                            prevb = bb
                    if not w:
                        widths[home[qq]] += 1
                ok = max(widths) <= max_width
            if ok and (best is None or k < best[0]):
                best = (k, b)
        if best is None:
            keep[gi] = False
            del gate_block[gi]
        else:
            gate_block[gi] = best[1]
    c2, gb = thinned()
    return build_cut(c2, gb, home)


def build_cut(circ: Circuit, gate_block: Dict[int, int], home: Sequence[int]) -> CutCircuit:
    """Turn a gate -> block assignment into subcircuits, slots and cut ids."""
    wires = _wire_blocks(circ, gate_block, home)
    n_blocks = max(max(home), max(gate_block.values(), default=0)) + 1
    # segments per qubit: list of (block, first pos, last pos)
    cut_wires: List[Tuple[int, int]] = []
    seg_of_gate: Dict[Tuple[int, int], Tuple[int, int]] = {}  # (gate, qubit) -> (qubit, seg idx)
    segs_per_q = []
    for q in range(circ.n):
        w = wires[q]
        segs = []
        if not w:
            segs.append(home[q])
        for i, (gi, b) in enumerate(w):
            if i == 0 or b != w[i - 1][1]:
                if i > 0:
                    cut_wires.append((q, i))
                segs.append(b)
            seg_of_gate[(gi, q)] = (q, len(segs) - 1)
        segs_per_q.append(segs)
    cut_id = {cw: k for k, cw in enumerate(sorted(cut_wires))}
    # cut k sits on qubit q between segment s and s+1
    cut_of_seg_boundary: Dict[Tuple[int, int], int] = {}
    for (q, pos), k in cut_id.items():
        w = wires[q]
        s = sum(1 for i in range(1, pos + 1) if w[i][1] != w[i - 1][1]) - 1
        cut_of_seg_boundary[(q, s)] = k
    # local qubits: per block ordered by (global qubit, segment)
    local: Dict[Tuple[int, int], Tuple[int, int]] = {}
    block_d = [0] * n_blocks
    for q in range(circ.n):
        for s, b in enumerate(segs_per_q[q]):
            local[(q, s)] = (b, block_d[b])
            block_d[b] += 1
    subs = []
    for b in range(n_blocks):
        gl = []
        for gi, g in enumerate(circ.gates):
            qs = []
            blk = None
            for q in g.qubits:
                bb, lq = local[seg_of_gate[(gi, q)]]
                blk = bb
                qs.append(lq)
            if blk == b:
                gl.append(Gate(g.name, tuple(qs), g.params))
        ins, outs, effs = [], [], []
        for q in range(circ.n):
            segs = segs_per_q[q]
            for s, bb in enumerate(segs):
                if bb != b:
                    continue
                lq = local[(q, s)][1]
                if s > 0:
                    ins.append((lq, cut_of_seg_boundary[(q, s - 1)]))
                if s < len(segs) - 1:
                    outs.append((lq, cut_of_seg_boundary[(q, s)]))
                else:
                    effs.append((lq, q))
        ins.sort(key=lambda t: t[1])
        outs.sort(key=lambda t: t[1])
        effs.sort(key=lambda t: t[1])
        subs.append(Subcircuit(block_d[b], gl, ins, outs, effs))
    cw = sorted(cut_wires)
    return CutCircuit(circ, subs, len(cw), cw)


# ---------------------------------------------------------------------------
# the benchmark workloads (seeded), sized as in the paper's families
# ---------------------------------------------------------------------------

def hwea_10q_k1(seed: int = 0) -> CutCircuit:
    """10-qubit HWEA cut once on q5 between CX(4,5) and CX(5,6): 2 subcircuits
    of 6 and 5 qubits, K=1."""
    c = hwea(10, seed)
    home = [0] * 5 + [1] * 5
    return cut_circuit(c, home)


def supremacy_4x6(seed: int = 0, depth: int = 8, max_cuts: int = 6, max_width: int = 15) -> CutCircuit:
    """4x6 supremacy-style grid cut into its left and right 4x3 halves (two
    subcircuits of <= 15 qubits, K <= 6).  Each kept crossing CZ lives in the
    left half, so the right qubit's wire visits the left subcircuit."""
    c = supremacy_grid(4, 6, depth, seed)
    home = [0 if (q % 6) < 3 else 1 for q in range(24)]
    return cut_circuit(c, home, max_cuts=max_cuts, max_width=max_width, policy="first")


def grid_blocks(rows: int, cols: int, depth: int, seed: int, brows: int, bcols: int,
                max_cuts: int, max_width: int) -> CutCircuit:
    """A rows x cols supremacy-style grid cut into brows x bcols rectangular
    blocks, under a cut budget and a subcircuit width limit."""
    c = supremacy_grid(rows, cols, depth, seed)
    rh, ch = rows // brows, cols // bcols
    home = [min(r // rh, brows - 1) * bcols + min(cc // ch, bcols - 1)
            for r in range(rows) for cc in range(cols)]
    return cut_circuit(c, home, max_cuts=max_cuts, max_width=max_width)


def cut_from_clusters(circ: Circuit, gate_cluster: Dict[int, int], max_width: Optional[int] = None) -> CutCircuit:
    """Subcircuits from an assignment of every multi-qubit gate (by gate index)
    to a subcircuit, as the cut searcher returns it (Sec. 4.1: the cuts are the
    wires whose consecutive multi-qubit gates lie in different subcircuits).
    Subcircuits are renumbered in order of first use.  A qubit that no
    multi-qubit gate touches is outside the search's graph (Sec. 4.1 takes the
    circuit to be connected); such qubits join the narrowest subcircuit that
    stays within max_width, else new subcircuits without cuts."""
    order: Dict[int, int] = {}
    for gi in sorted(gate_cluster):
        order.setdefault(gate_cluster[gi], len(order))
    gb = {gi: order[c] for gi, c in gate_cluster.items()}
    home = [-1] * circ.n
    for gi, g in enumerate(circ.gates):
        if len(g.qubits) > 1:
            for q in g.qubits:
                if home[q] < 0:
                    home[q] = gb[gi]
    n_blocks = max(len(order), 1)
    # widths of the connected part: wire segments per block
    width = [0] * n_blocks
    for w in _wire_blocks(circ, gb, [max(h, 0) for h in home]):
        prev = None
        for _, b in w:
            if b != prev:
                width[b] += 1
                prev = b
    for q in range(circ.n):
        if home[q] >= 0:
            continue
        b = min(range(n_blocks), key=lambda i: (width[i], i))
        if max_width is not None and width[b] >= max_width:
            b = n_blocks
            n_blocks += 1
            width.append(0)
        home[q] = b
        width[b] += 1
    return build_cut(circ, gb, home)


def chain_blocks(circ: Circuit, n_sub: int, max_cuts: Optional[int] = None,
                 max_width: Optional[int] = None, policy: str = "first") -> CutCircuit:
    """Cut a circuit on a chain of qubits into n_sub contiguous blocks."""
    n = circ.n
    home = [min(q * n_sub // n, n_sub - 1) for q in range(n)]
    return cut_circuit(circ, home, max_cuts=max_cuts, max_width=max_width, policy=policy)


def qaoa_2cluster(n_per: int = 15, seed: int = 0) -> CutCircuit:
    """QAOA MaxCut on two 3-regular clusters joined by 2 bridges, cut at the
    bridge ZZs into one subcircuit per cluster (K=4)."""
    c = qaoa_maxcut(n_per, seed)
    home = [0] * n_per + [1] * n_per
    cc = cut_circuit(c, home, policy="first")
    cc.edges = c.edges  # type: ignore[attr-defined]
    return cc


def bv_chain(n: int, seed: int, n_sub: int = 2) -> CutCircuit:
    """BV whose CNOTs all target the last qubit, cut into n_sub chain blocks."""
    return chain_blocks(bv(n, seed), n_sub)


def batch_instances(count: int = 64, seed: int = 0, max_width: int = 16) -> List[CutCircuit]:
    """A batch of cut circuits of uneven shape (the batched workload): each
    instance draws its family from {HWEA, AQFT (rotations below pi/2^4
    dropped), BV with a random secret}, an even width of 16..28 qubits and 2..4
    chain blocks of at most `max_width` qubits, with a cut budget K <= 8 and
    4^K * 2^n <= 2^40 (cut by construction: crossing gates beyond the budget
    are dropped).  Draws whose cut has fewer than 2 wires (a single crossing,
    as an HWEA chain in two blocks has) are drawn again, so every instance has
    2 <= K <= 8."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        fam = ("hwea", "aqft", "bv")[int(rng.integers(3))]
        n = int(rng.integers(8, 15)) * 2
        s = int(rng.integers(2, 5))
        while n / s > max_width - 2:
            s += 1
        kmax = min(8, (40 - n) // 2)
        cs = int(rng.integers(1 << 30))
        c = hwea(n, cs) if fam == "hwea" else aqft(n, cs) if fam == "aqft" else bv(n, cs)
        cc = chain_blocks(c, s, max_cuts=kmax, max_width=max_width)
        if cc.n_cuts < 2:
            continue
        cc.family = fam  # type: ignore[attr-defined]
        out.append(cc)
    return out
