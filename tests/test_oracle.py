"""Pins of the FP64 oracle against facts that do not come from the oracle:
textbook states, the paper's worked formulas (Sec. 3.2.2-3.2.3), brute-force
simulation of the uncut circuit (the exactness claim of Sec. 3.2.3), the
Figure 7 dynamic-definition example, closed forms and invariants."""
import json
import os

import numpy as np
import pytest

from paper_2012_02333_gb300 import circuits as C
from oracle import attribution as at
from oracle import reconstruct as rc
from oracle import statevector as sv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- simulator

def test_gate_matrices_unitary():
    for name in C.ONE_QUBIT + C.TWO_QUBIT:
        U = sv.gate_matrix(name, (0.7,))
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-14), name


def test_square_roots_square_to_paulis():
    X, Y = sv.gate_matrix("x"), sv.gate_matrix("y")
    W = (X + Y) / np.sqrt(2)
    for r, P in (("sx", X), ("sy", Y), ("sw", W)):
        R = sv.gate_matrix(r)
        assert np.allclose(R @ R, P, atol=1e-14)


def test_bell_and_ghz_textbook():
    c = C.Circuit(2)
    c.add("h", 0)
    c.add("cx", 0, 1)
    assert np.allclose(sv.probabilities(c), [0.5, 0, 0, 0.5], atol=1e-15)
    c = C.Circuit(3)
    c.add("h", 0)
    c.add("cx", 0, 1)
    c.add("cx", 1, 2)
    p = sv.probabilities(c)
    assert np.allclose(p[[0, 7]], 0.5) and np.allclose(np.delete(p, [0, 7]), 0)


def test_qubit0_is_msb_and_rotation():
    c = C.Circuit(3)
    c.add("x", 0)
    assert sv.probabilities(c)[4] == pytest.approx(1.0)
    c = C.Circuit(1)
    c.add("ry", 0, params=[0.9])
    assert np.allclose(sv.probabilities(c), [np.cos(0.45) ** 2, np.sin(0.45) ** 2])


def test_cx_control_is_first_qubit():
    c = C.Circuit(2)
    c.add("x", 1)
    c.add("cx", 1, 0)
    assert sv.probabilities(c)[3] == pytest.approx(1.0)


# ------------------------------------------------------------- attribution

def test_init_states_prepare_eigenstates():
    # |+i> measured in the Y basis gives outcome 0 (eigenvalue +1) with certainty
    sub = C.Subcircuit(1, [], [(0, 0)], [], [(0, 0)])
    p = at.variant_probabilities(sub)   # no measurement slot: Z basis only
    assert np.allclose(p[:, 0, :], [[1, 0], [0, 1], [0.5, 0.5], [0.5, 0.5]])
    # a measured cut qubit prepared |+i> by gates: S H |0> = |+i>
    sub = C.Subcircuit(1, [C.Gate("h", (0,)), C.Gate("s", (0,))], [], [(0, 0)], [])
    p = at.variant_probabilities(sub)[0]   # bases Z, X, Y
    assert np.allclose(p, [[0.5, 0.5], [0.5, 0.5], [1.0, 0.0]], atol=1e-15)


def test_pauli_expectations_of_a_known_state():
    # Ry(t) Rz(f) |0>: Bloch vector (sin t cos f, sin t sin f, cos t)
    t, f = 1.1, 0.4
    sub = C.Subcircuit(1, [C.Gate("ry", (0,), (t,)), C.Gate("rz", (0,), (f,))], [], [(0, 0)], [])
    T = at.subcircuit_tensor(sub)[0, :, 0]     # b over I, X, Y, Z
    assert np.allclose(T, [1, np.sin(t) * np.cos(f), np.sin(t) * np.sin(f), np.cos(t)], atol=1e-14)


def test_downstream_trace_identity():
    # Sum_x T[a] = 2^k_in for a = I...I and 0 otherwise (circuits preserve trace)
    cc = C.qaoa_2cluster(4, 3)
    for sub in cc.subs:
        T = at.subcircuit_tensor(sub)
        s = T.sum(axis=2)     # [a][b]
        b_I = 0               # b = I..I keeps the trace
        want = np.zeros(4 ** sub.k_in)
        want[0] = 2 ** sub.k_in
        assert np.allclose(s[:, b_I], want, atol=1e-12)


def test_upstream_bloch_ball():
    cc = C.hwea_10q_k1()
    up = [s for s in cc.subs if s.k_out == 1 and s.k_in == 0][0]
    T = at.subcircuit_tensor(up)[0]   # [b][x]
    ev = T.sum(axis=1)                # <I>, <X>, <Y>, <Z> of the cut qubit
    assert ev[0] == pytest.approx(1.0)
    assert ev[1] ** 2 + ev[2] ** 2 + ev[3] ** 2 <= 1 + 1e-12
    # outcome sums: p(x, m=0 | M) + p(x, m=1 | M) is the same for every basis
    p = at.variant_probabilities(up)[0].reshape(3, -1, 2)
    assert np.allclose(p.sum(axis=2)[0], p.sum(axis=2)[1]) and np.allclose(p.sum(axis=2)[0], p.sum(axis=2)[2])


def test_paper_worked_single_cut_formulas():
    """Sec. 3.2.2-3.2.3 written out as printed: p_{1,1..4} from the upstream
    variants, p_{2,1..4} from the downstream variants, p = 1/2 sum p_1i p_2i,
    against brute force of the uncut circuit (Figure 4 shape: 5 qubits, one
    cut on q2 between the first two CZs, two 3-qubit subcircuits)."""
    rng = np.random.default_rng(5)
    c = C.Circuit(5)
    for q in range(5):
        c.add("ry", q, params=[rng.uniform(0, 6.28)])
        c.add("rz", q, params=[rng.uniform(0, 6.28)])
    c.add("cz", 0, 2)
    c.add("cz", 1, 2)
    c.add("ry", 2, params=[0.3])
    c.add("cz", 2, 3)
    c.add("cz", 3, 4)
    c.add("cz", 2, 4)
    for q in range(5):
        c.add("sx", q)
    # cut q2 between the first two CZs that touch it and the rest (Figure 4)
    blocks = {}
    for gi, g in enumerate(c.gates):
        if len(g.qubits) == 2:
            blocks[gi] = 0 if g.qubits in ((0, 2), (1, 2)) else 1
    cc = C.build_cut(c, blocks, [0, 0, 0, 1, 1])
    assert cc.n_cuts == 1
    up, down = cc.subs
    assert up.d == 3 and down.d == 3 and up.k_out == 1 and down.k_in == 1
    pu = at.variant_probabilities(up)[0]   # [basis Z,X,Y][local state], local 2 = cut qubit
    pd = at.variant_probabilities(down)[:, 0, :]   # [init 0,1,+,+i][local state]
    ref = sv.probabilities(cc.circuit)
    lq_cut = up.out_slots[0][0]
    assert lq_cut == 2
    for x in range(32):
        bits = [(x >> (4 - q)) & 1 for q in range(5)]
        xx = 4 * bits[0] + 2 * bits[1]          # |xx0> in subcircuit 1's local order
        y2 = sum(bits[q] << (2 - i) for i, q in enumerate([2, 3, 4]))
        # downstream local order: (q2 segment = init qubit 0), q3, q4
        pI0, pI1 = pu[0, xx], pu[0, xx + 1]     # I and Z share the Z-basis circuit
        pX0, pX1 = pu[1, xx], pu[1, xx + 1]
        pY0, pY1 = pu[2, xx], pu[2, xx + 1]
        p11 = pI0 + pI1 + pI0 - pI1
        p12 = pI0 + pI1 - pI0 + pI1
        p13 = pX0 - pX1
        p14 = pY0 - pY1
        q0, q1, qp, qi = pd[0, y2], pd[1, y2], pd[2, y2], pd[3, y2]
        p21, p22 = q0, q1
        p23 = 2 * qp - q0 - q1
        p24 = 2 * qi - q0 - q1
        p = 0.5 * (p11 * p21 + p12 * p22 + p13 * p23 + p14 * p24)
        assert p == pytest.approx(ref[x], abs=1e-14)


def test_pauli_pairing_equals_paper_pairing():
    """Eq. 2 pairs (I+Z) with |0> and (I-Z) with |1>; the oracle pairs I with I
    and Z with Z.  The two sums agree for every x (R2 reading)."""
    cc = C.hwea_10q_k1(3)
    Tu, Td = at.tensors(cc)
    up, down = cc.subs
    a = Tu[0]      # [b][x_up]
    b = Td[:, 0]   # [a][x_down]
    pauli = 0.5 * np.einsum("ex,ey->xy", a, b)
    paper = 0.5 * (np.outer(a[0] + a[3], (b[0] + b[3]) / 2) + np.outer(a[0] - a[3], (b[0] - b[3]) / 2)
                   + np.outer(a[1], b[1]) + np.outer(a[2], b[2]))
    assert np.allclose(pauli, paper, atol=1e-15)


# ------------------------------------------------------------ full definition

CASES = [
    ("hwea10_k1", lambda: C.hwea_10q_k1(0)),
    ("bv6", lambda: C.chain_blocks(C.bv(6, 1), 2, max_width=4)),
    ("grid3x4", lambda: C.grid_blocks(3, 4, 8, 1, 1, 2, 6, 9)),
    ("qaoa8", lambda: C.qaoa_2cluster(4, 1)),
    ("aqft8", lambda: C.chain_blocks(C.aqft(8, 0), 2, max_cuts=6)),
    ("hwea9_s3", lambda: C.chain_blocks(C.hwea(9, 2), 3)),
    ("grid4x4_s4", lambda: C.grid_blocks(4, 4, 6, 3, 2, 2, 8, 7)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fd_equals_brute_force(name, make):
    """Sec. 3.2.3: the reconstruction strictly equals the uncut output."""
    cc = make()
    Ts = at.tensors(cc)
    p = rc.fd_full(cc.subs, Ts, cc.n, cc.n_cuts)
    ref = sv.probabilities(cc.circuit)
    assert np.abs(p - ref).max() < 1e-13
    assert p.sum() == pytest.approx(1.0, abs=1e-12)
    xs = [0, 1, 2 ** cc.n - 1, 5 % 2 ** cc.n]
    assert np.allclose(rc.fd_entries(cc.subs, Ts, cc.n, cc.n_cuts, xs), ref[xs], atol=1e-13)


def test_fd_no_cut_is_statevector():
    c = C.hwea(6, 4)
    cc = C.cut_circuit(c, [0] * 6)
    assert cc.n_cuts == 0 and len(cc.subs) == 1
    Ts = at.tensors(cc)
    assert np.allclose(rc.fd_full(cc.subs, Ts, 6, 0), sv.probabilities(c), atol=1e-15)


def test_fig12_term_count():
    """Figure 12: the 4x6 supremacy grid on a 15-qubit device takes 4 cuts,
    4^4 = 256 Kronecker products."""
    g = json.load(open(os.path.join(GOLDEN, "fig12_supremacy_4x6.json")))
    cc = C.supremacy_4x6(0)
    assert cc.n == g["n_qubits"] and cc.n_cuts == g["n_cuts"]
    assert max(s.d for s in cc.subs) <= g["max_width"]
    assert 4 ** cc.n_cuts == g["kronecker_products"]
    assert sum(s.n_eff for s in cc.subs) == cc.n


def test_cut_model_constraints():
    """Eqs. 5-7 and 13: f_c = alpha_c + rho_c - O_c sums to n, and every cut
    has exactly one upstream and one downstream slot."""
    for _, make in CASES:
        cc = make()
        assert sum(s.n_eff for s in cc.subs) == cc.n
        ins = sorted(c for s in cc.subs for c in s.in_cut)
        outs = sorted(c for s in cc.subs for c in s.out_cut)
        assert ins == outs == list(range(cc.n_cuts))
        for s in cc.subs:
            alpha = s.d - s.k_in
            assert s.n_eff == alpha + s.k_in - s.k_out


def test_planted_mistakes_are_caught():
    """A dropped Y term, a flipped sign or a transposed operand in the sum must
    break the brute-force pin."""
    cc = C.grid_blocks(3, 4, 8, 1, 1, 2, 6, 9)
    Ts = at.tensors(cc)
    ref = sv.probabilities(cc.circuit)
    bad = [T.copy() for T in Ts]
    bad[0][:, :, :] *= np.where(np.arange(bad[0].shape[0] * bad[0].shape[1]) % 4 == 2, 0, 1).reshape(bad[0].shape[0], bad[0].shape[1], 1)
    assert np.abs(rc.fd_full(cc.subs, bad, cc.n, cc.n_cuts) - ref).max() > 1e-6
    bad = [T.copy() for T in Ts]
    bad[1] = -bad[1]
    assert np.abs(rc.fd_full(cc.subs, bad, cc.n, cc.n_cuts) - ref).max() > 1e-6


# ------------------------------------------------------- dynamic definition

def test_fig7_bv_dd_golden():
    g = json.load(open(os.path.join(GOLDEN, "fig7_bv4_dd.json")))
    c = C.bv(g["n_qubits"], 0, g["secret"])
    cc = C.chain_blocks(c, 2, max_width=3)
    assert max(s.d for s in cc.subs) <= 3 and cc.n_cuts >= 1
    Ts = at.tensors(cc)
    for strategy in ("dfs", "bfs"):
        recs = rc.dd_run(cc.subs, Ts, cc.n, cc.n_cuts, g["n_active"], 4, strategy)
        for rec, want in zip(recs, g["bins_per_recursion"]):
            assert np.allclose(rec["bins"], want, atol=1e-13)
        # recursion 2 holds qubit 0 at |1> (the first qubit of the paper's 1-based count)
        assert recs[1]["roles"][0] == 3
        last = recs[-1]
        hot = int(np.argmax(last["bins"]))        # the one active qubit's heavier value
        bits = [1 if r == 3 else 0 if r == 2 else hot for r in last["roles"]]
        sol = sum(b << (3 - q) for q, b in enumerate(bits))
        assert sol == g["solution"] and last["bins"][hot] == pytest.approx(g["solution_probability"])


@pytest.mark.parametrize("name,make", CASES[1:5], ids=[c[0] for c in CASES[1:5]])
def test_dd_bins_are_brute_force_marginals(name, make):
    cc = make()
    Ts = at.tensors(cc)
    ref = sv.probabilities(cc.circuit).reshape([2] * cc.n)
    recs = rc.dd_run(cc.subs, Ts, cc.n, cc.n_cuts, 3, 4, "bfs")
    assert recs[0]["bins"].sum() == pytest.approx(1.0, abs=1e-12)
    for rec in recs:
        roles = rec["roles"]
        idx = tuple(0 if r == 2 else 1 if r == 3 else slice(None) for r in roles)
        sub = ref[idx]
        kept = [r for r in roles if r in (0, 1)]
        merged_axes = tuple(i for i, r in enumerate(kept) if r == 1)
        want = sub.sum(axis=merged_axes).reshape(-1) if merged_axes else sub.reshape(-1)
        assert np.allclose(rec["bins"], want, atol=1e-13)
        if rec["parent"] is not None:
            ri, bi = rec["parent"]
            assert rec["bins"].sum() == pytest.approx(recs[ri]["bins"][bi], abs=1e-13)


def _slab_of(cc, Ts, roles):
    """slab(c, a) for dd_entries over host tensors: the entries of subcircuit
    c's rows whose active outputs read `a` and zoomed outputs their fixed
    bits, handed over in two row pieces, each split into two column pieces
    in reverse column order (the oracle must not depend on how they come)."""
    def slab(c, a):
        s = cc.subs[c]
        T = Ts[c].reshape(4 ** s.k_in * 4 ** s.k_out, -1)
        act = [i for i, q in enumerate(s.out_qubit) if roles[q] == 0]
        cols = []
        for x in range(2 ** s.n_eff):
            ok = True
            for i, q in enumerate(s.out_qubit):
                bit = (x >> (s.n_eff - 1 - i)) & 1
                r = roles[q]
                if (r == 2 and bit) or (r == 3 and not bit):
                    ok = False
                elif r == 0 and bit != (a >> (len(act) - 1 - act.index(i))) & 1:
                    ok = False
            if ok:
                cols.append(x)
        cols = cols[::-1]
        h, w = T.shape[0] // 2, len(cols) // 2
        for r0, r1 in ((0, h), (h, T.shape[0])):
            for part in (cols[:w], cols[w:]):
                yield r0, T[r0:r1][:, part] if part else np.zeros((r1 - r0, 0))
    return slab


@pytest.mark.parametrize("name,make", CASES[1:5], ids=[c[0] for c in CASES[1:5]])
def test_dd_entries_are_brute_force_marginals(name, make):
    """Selected bins from merged slabs (the form used where the merged tensors
    cannot be formed whole) equal the uncut circuit's marginals, for every bin
    of several recursions."""
    cc = make()
    Ts = at.tensors(cc)
    ref = sv.probabilities(cc.circuit).reshape([2] * cc.n)
    recs = rc.dd_run(cc.subs, Ts, cc.n, cc.n_cuts, 3, 4, "bfs")
    for rec in recs:
        roles = rec["roles"]
        idx = tuple(0 if r == 2 else 1 if r == 3 else slice(None) for r in roles)
        sub = ref[idx]
        kept = [r for r in roles if r in (0, 1)]
        merged_axes = tuple(i for i, r in enumerate(kept) if r == 1)
        want = sub.sum(axis=merged_axes).reshape(-1) if merged_axes else sub.reshape(-1)
        bins = list(range(len(want)))
        got = rc.dd_entries(cc.subs, _slab_of(cc, Ts, roles), cc.n, cc.n_cuts, roles, bins)
        assert np.allclose(got, want, atol=1e-13)


def test_dd_run_follows_only_near_ties():
    """The follow option of dd_run takes another run's zoom choice only when
    that bin is eligible and within the given distance of the heaviest one."""
    cc = CASES[2][1]()
    Ts = at.tensors(cc)
    plain = rc.dd_run(cc.subs, Ts, cc.n, cc.n_cuts, 3, 3, "bfs")
    same = rc.dd_run(cc.subs, Ts, cc.n, cc.n_cuts, 3, 3, "bfs", follow=[r["parent"] for r in plain], follow_tol=1.0)
    assert [r["roles"] for r in same] == [r["roles"] for r in plain]
    assert not any(r["followed"] for r in same)
    b = plain[0]["bins"]
    order = sorted(range(len(b)), key=lambda i: (-b[i], i))
    best, second = order[0], order[1]
    assert plain[1]["parent"] == (0, best)
    gap = b[best] - b[second]
    assert gap > 0
    far = rc.dd_run(cc.subs, Ts, cc.n, cc.n_cuts, 3, 2, "bfs", follow=[None, (0, second)], follow_tol=gap / 2)
    assert far[1]["parent"] == (0, best) and not far[1]["followed"]
    near = rc.dd_run(cc.subs, Ts, cc.n, cc.n_cuts, 3, 2, "bfs", follow=[None, (0, second)], follow_tol=gap * 2)
    assert near[1]["parent"] == (0, second) and near[1]["followed"]
    assert near[1]["bins"].sum() == pytest.approx(b[second], abs=1e-13)


def _roles_cycle(cc, pattern):
    """Roles over the global qubits: the pattern repeated over the qubit order."""
    return [pattern[q % len(pattern)] for q in range(cc.n)]


@pytest.mark.parametrize("pattern", [(0, 1, 2, 3), (1, 0, 1, 3, 0), (1, 1, 1, 2), (0, 0, 0, 0)])
def test_attribute_merged_is_attribution_of_merged_variants(pattern):
    """Merging (Algorithm 1) sums over output qubits and fixes zoomed ones,
    while Eq. 3 and Eq. 2 act only on the cut qubits' outcomes and the init
    variants, so attributing then merging equals attributing the variant
    distributions already summed over the merged outputs.  Checked with
    random, non-physical distributions (nothing cancels by accident) against
    that second route, built here from plain axis sums and a reduced
    subcircuit with the merged and zoomed qubits removed."""
    cc = C.qaoa_2cluster(4, 1)
    rng = np.random.default_rng(5)
    roles = _roles_cycle(cc, pattern)
    for sub in cc.subs:
        V = (4 ** sub.k_in) * (3 ** sub.k_out)
        p = rng.random((V, 2 ** sub.d))
        got = at.attribute_merged(sub, p, roles)
        role_of = {lq: roles[gq] for lq, gq in sub.outputs}
        arr = p.reshape([V] + [2] * sub.d)
        idx = [slice(None)] + [({2: 0, 3: 1}.get(role_of.get(lq), slice(None))) for lq in range(sub.d)]
        red = arr[tuple(idx)]
        remaining = [lq for lq in range(sub.d) if role_of.get(lq) not in (2, 3)]
        red = red.sum(axis=tuple(1 + remaining.index(lq) for lq in remaining if role_of.get(lq) == 1))
        kept = [lq for lq in remaining if role_of.get(lq) != 1]
        pos = {lq: i for i, lq in enumerate(kept)}
        reduced = C.Subcircuit(d=len(kept), gates=[], in_slots=[(0, c) for _, c in sub.in_slots],
                               out_slots=[(pos[lq], c) for lq, c in sub.out_slots],
                               outputs=[(pos[lq], gq) for lq, gq in sub.outputs if roles[gq] == 0])
        want = at.attribute(reduced, red.reshape(V, -1)).reshape(got.shape)
        assert got.shape == (4 ** (sub.k_in + sub.k_out), 2 ** sum(1 for _, g in sub.outputs if roles[g] == 0))
        assert np.allclose(got, want, atol=1e-12, rtol=0)
        assert np.abs(got).max() > 0.1


def test_attribute_merged_bins_are_brute_force_marginals():
    """A recursion's bins contracted from the fused merged tensors of the
    physical variants equal the uncut circuit's marginal over the merged
    qubits with the zoomed ones fixed."""
    cc = C.grid_blocks(3, 4, 8, 1, 1, 2, 6, 9)
    roles = _roles_cycle(cc, (0, 1, 3, 0, 1, 2))
    Ms = [at.attribute_merged(s, at.variant_probabilities(s), roles) for s in cc.subs]
    active = [q for q in range(cc.n) if roles[q] == 0]
    rank = {q: i for i, q in enumerate(active)}
    na = len(active)
    bins = np.zeros(2 ** na)
    for e in range(4 ** cc.n_cuts):
        dg = [(e >> (2 * (cc.n_cuts - 1 - k))) & 3 for k in range(cc.n_cuts)]
        term = np.ones(2 ** na)
        for s, M in zip(cc.subs, Ms):
            qs = [g for _, g in s.outputs if roles[g] == 0]
            vals = M[rc.row_of(s, dg)]
            for b in range(2 ** na):
                j = 0
                for q in qs:
                    j = 2 * j + ((b >> (na - 1 - rank[q])) & 1)
                term[b] *= vals[j]
        bins += term
    bins *= 2.0 ** -cc.n_cuts
    ref = sv.probabilities(cc.circuit).reshape([2] * cc.n)
    ref = ref[tuple(0 if r == 2 else 1 if r == 3 else slice(None) for r in roles)]
    kept = [r for r in roles if r in (0, 1)]
    want = ref.sum(axis=tuple(i for i, r in enumerate(kept) if r == 1)).reshape(-1)
    assert np.allclose(bins, want, atol=1e-13)


def test_dd_zoom_roles_reading():
    roles = rc.initial_roles(6, 2)
    assert roles == [0, 0, 1, 1, 1, 1]
    r2 = rc.zoom_roles(roles, 2, 2)        # bin 0b10: q0 = 1, q1 = 0
    assert r2 == [3, 2, 0, 0, 1, 1]
    r3 = rc.zoom_roles(r2, 1, 2)
    assert r3 == [3, 2, 2, 3, 0, 0]


# ----------------------------------------------------------------- gradient

def test_gradient_central_differences():
    """L = sum_x G(x) p(x) is linear in each tensor, so central differences
    with h = 1e-6 are exact up to rounding."""
    cc = C.qaoa_2cluster(4, 2)
    Ts = at.tensors(cc)
    rng = np.random.default_rng(0)
    G = rng.standard_normal(2 ** cc.n)
    grads = rc.grad(cc.subs, Ts, cc.n, cc.n_cuts, G)
    h = 1e-6
    for c in range(len(Ts)):
        flat = Ts[c].reshape(-1)
        for i in rng.choice(flat.size, 12, replace=False):
            tp = [T.copy() for T in Ts]
            tm = [T.copy() for T in Ts]
            tp[c].reshape(-1)[i] += h
            tm[c].reshape(-1)[i] -= h
            lp = G @ rc.fd_full(cc.subs, tp, cc.n, cc.n_cuts)
            lm = G @ rc.fd_full(cc.subs, tm, cc.n, cc.n_cuts)
            assert grads[c].reshape(-1)[i] == pytest.approx((lp - lm) / (2 * h), abs=1e-8)


def test_maxcut_expectation_matches_brute_force():
    cc = C.qaoa_2cluster(4, 2)
    edges = cc.edges
    Cx = rc.maxcut_values(cc.n, edges)
    # brute C(x) by direct bit loops
    for x in (0, 7, 200, 255):
        bits = [(x >> (cc.n - 1 - q)) & 1 for q in range(cc.n)]
        assert Cx[x] == sum(bits[i] != bits[j] for i, j in edges)
    Ts = at.tensors(cc)
    p = rc.fd_full(cc.subs, Ts, cc.n, cc.n_cuts)
    assert Cx @ p == pytest.approx(Cx @ sv.probabilities(cc.circuit), abs=1e-12)


def test_grad_entry_central_differences():
    """The one-entry gradient used at full size, against central differences
    of the plain sum for a MaxCut loss."""
    cc = C.qaoa_2cluster(4, 2)
    Ts = at.tensors(cc)
    G = rc.maxcut_values(cc.n, cc.edges)
    f = rc.maxcut_of(cc.n, cc.edges)
    h = 1e-6
    for c, r, x in [(0, 0, 0), (0, 7, 3), (1, 12, 9), (1, 255, 15)]:
        tp = [T.copy() for T in Ts]
        tm = [T.copy() for T in Ts]
        tp[c].reshape(tp[c].shape[0] * tp[c].shape[1], -1)[r, x] += h
        tm[c].reshape(tm[c].shape[0] * tm[c].shape[1], -1)[r, x] -= h
        fd = (G @ rc.fd_full(cc.subs, tp, cc.n, cc.n_cuts) - G @ rc.fd_full(cc.subs, tm, cc.n, cc.n_cuts)) / (2 * h)
        assert rc.grad_entry(cc.subs, Ts, cc.n, cc.n_cuts, c, r, x, f) == pytest.approx(fd, abs=1e-8)


# ---- Eq. 16 chi^2 loss, total variation, inverse-transform sampling --------

def test_chi_square_closed_forms():
    from oracle import metrics as mt
    # identical distributions: 0
    p = np.random.default_rng(1).random(64)
    p /= p.sum()
    assert mt.chi_square(p, p) == 0.0
    # a point mass against a fair coin: (1 - 1/2)^2 / (3/2) + (0 - 1/2)^2 / (1/2) = 1/6 + 1/2
    assert mt.chi_square([1.0, 0.0], [0.5, 0.5]) == pytest.approx(2.0 / 3.0, abs=1e-15)
    # disjoint supports: every term is (a + b)^2 / (a + b) = a + b, so chi^2 = 2
    assert mt.chi_square([0.5, 0.5, 0, 0], [0, 0, 0.25, 0.75]) == pytest.approx(2.0, abs=1e-15)
    # zero-weight outcomes on both sides contribute nothing (the reading for a_i + b_i = 0)
    assert mt.chi_square([1.0, 0.0, 0.0], [0.5, 0.5, 0.0]) == pytest.approx(2.0 / 3.0, abs=1e-15)
    # symmetric in its arguments
    q = np.random.default_rng(2).random(64)
    q /= q.sum()
    assert mt.chi_square(p, q) == pytest.approx(mt.chi_square(q, p), rel=1e-14)


def test_chi_square_small_differences_match_the_expansion():
    """For b = a + d with small d, (d_i)^2 / (2 a_i + d_i) ~ d_i^2 / (2 a_i):
    the leading term of the expansion, checked to relative O(|d|/a)."""
    from oracle import metrics as mt
    rng = np.random.default_rng(3)
    a = rng.random(256) + 0.5
    a /= a.sum()
    d = 1e-6 * rng.standard_normal(256)
    d -= d.mean()
    approx = float(np.sum(d ** 2 / (2 * a)))
    assert mt.chi_square(a, a + d) == pytest.approx(approx, rel=1e-3)


def test_total_variation_closed_forms():
    from oracle import metrics as mt
    assert mt.total_variation([0.5, 0.5, 0, 0], [0, 0, 0.25, 0.75]) == pytest.approx(1.0)
    assert mt.total_variation([1.0, 0.0], [0.5, 0.5]) == pytest.approx(0.5)
    p = np.full(8, 1 / 8)
    assert mt.total_variation(p, p) == 0.0


def test_sampling_special_cases():
    from oracle import metrics as mt
    # a point mass is always drawn
    p = np.zeros(16)
    p[11] = 1.0
    assert (mt.sample(p, [0.0, 0.3, 0.999999]) == 11).all()
    # uniform over 4: u in [k/4, (k+1)/4) draws k
    assert list(mt.sample([0.25] * 4, [0.0, 0.2499, 0.25, 0.5, 0.74, 0.999])) == [0, 0, 1, 2, 2, 3]
    # negative entries (rounding residue) carry no weight and are never drawn
    q = np.array([0.5, -1e-9, 0.0, 0.5])
    xs = mt.sample(q, np.linspace(0, 0.999, 200))
    assert set(xs.tolist()) == {0, 3}
    # unnormalised weights: drawn in proportion
    assert list(mt.sample([1.0, 3.0], [0.24, 0.26])) == [0, 1]
    # nothing carries weight: nothing can be drawn
    assert list(mt.sample([0.0, -1e-12, 0.0], [0.1, 0.9])) == [-1, -1]


def test_sampling_frequencies_follow_the_distribution():
    """Law of large numbers on a seeded stream: 200k draws from a 16-outcome
    distribution, Pearson statistic below the 0.999 quantile of chi^2 with 15
    degrees of freedom (37.7)."""
    from oracle import metrics as mt
    rng = np.random.default_rng(5)
    p = rng.random(16) ** 3
    p /= p.sum()
    n = 200_000
    xs = mt.sample(p, rng.random(n))
    counts = np.bincount(xs, minlength=16)
    stat = float(np.sum((counts - n * p) ** 2 / (n * p)))
    assert stat < 37.7


# ---- exact cut search (Sec. 4.1, Eqs. 4-15) --------------------------------

def _chain(n):
    from paper_2012_02333_gb300.circuits import Circuit
    c = Circuit(n)
    for q in range(n):
        c.add("h", q)
    for q in range(n - 1):
        c.add("cx", q, q + 1)
    return c


def test_cut_search_worked_chain():
    """A CNOT chain on 4 qubits: v0 = CX(0,1), v1 = CX(1,2), v2 = CX(2,3);
    edges v0->v1 (qubit 1) and v1->v2 (qubit 2); w = (2, 1, 1).  With D = 3 the
    uncut circuit (d = 4) is infeasible; cutting either edge gives K = 1 and
    subcircuits of f = (2, 2) or (1, 3): L = 4 * 2^4 = 64 both ways, and the
    first in vertex order is {v0, v1 | v2}."""
    from oracle import cutsearch as cs
    c = _chain(4)
    verts, edges, w = cs.graph(4, c.gates)
    assert edges == [(0, 1), (1, 2)] and w == [2, 1, 1]
    r = cs.search(4, c.gates, 3, 2)
    assert r["L"] == 64 and r["K"] == 1 and r["assign"] == [0, 0, 1]
    assert r["f"] == [2, 2] and r["d"] == [3, 2]
    # the other cut of the same cost
    other = cs.cost([0, 1, 1], edges, w, 2)
    assert other["L"] == 64 and other["f"] == [1, 3] and other["d"] == [2, 3]
    # with room for the whole circuit nothing is cut: f = (4, 0), L = 2^4
    r = cs.search(4, c.gates, 4, 2)
    assert r["K"] == 0 and r["L"] == 16
    # too small a device: no assignment satisfies Eq. 9
    assert cs.search(4, c.gates, 1, 2) is None


def test_cut_search_invariants():
    """For every assignment: sum_c f_c = n (each qubit's final segment is
    measured in exactly one subcircuit), sum_c rho_c = sum_c O_c = K, and
    sum_c alpha_c = n; L of the three-subcircuit sum written out by hand."""
    import itertools
    from oracle import cutsearch as cs
    from paper_2012_02333_gb300 import circuits as C
    circ = C.hwea(5, 3)
    verts, edges, w = cs.graph(5, circ.gates)
    for assign in itertools.product(*[range(min(k + 1, 3)) for k in range(len(verts))]):
        r = cs.cost(assign, edges, w, 3)
        assert sum(r["f"]) == 5 and sum(r["alpha"]) == 5
        assert sum(r["rho"]) == sum(r["O"]) == r["K"]
        f1, f2, f3 = r["f"]
        assert r["L"] == 4 ** r["K"] * (2 ** (f1 + f2) + 2 ** (f1 + f2 + f3))
