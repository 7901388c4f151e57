"""The exact cut searcher (Sec. 4.1, Eqs. 4-15) against the oracle's
enumeration: same least cost (exactly), same cut count, same assignment (both
take the first of least cost in vertex order), on small circuits of the
paper's benchmark families; errors come back as statuses.  Host code only."""
import pytest

from oracle import cutsearch as cs
from paper_2012_02333_gb300 import circuits as C


@pytest.fixture(scope="module")
def cq():
    from paper_2012_02333_gb300 import cutqc
    return cutqc


def chain(n):
    c = C.Circuit(n)
    for q in range(n):
        c.add("h", q)
    for q in range(n - 1):
        c.add("cx", q, q + 1)
    return c


def qaoa_ring(n, seed):
    """QAOA p=1 MaxCut layer on an n-ring: H, ZZ = CX Rz CX per edge, Rx."""
    import numpy as np
    rng = np.random.default_rng(seed)
    g, b = rng.uniform(0, np.pi, 2)
    c = C.Circuit(n)
    for q in range(n):
        c.add("h", q)
    for i in range(n):
        j = (i + 1) % n
        c.add("cx", i, j)
        c.add("rz", j, params=[2 * g])
        c.add("cx", i, j)
    for q in range(n):
        c.add("rx", q, params=[2 * b])
    return c


CASES = [
    ("chain4", lambda: chain(4), [(3, 2), (4, 2), (2, 3)]),
    ("hwea6", lambda: C.hwea(6, 1), [(3, 2), (4, 2), (4, 3), (2, 3)]),
    ("bv5", lambda: C.bv(5, 2), [(3, 2), (4, 2), (3, 3)]),
    ("aqft5", lambda: C.aqft(5, 0), [(4, 2), (3, 3)]),
    ("qaoa_ring4", lambda: qaoa_ring(4, 1), [(3, 2), (4, 2), (3, 3)]),
    ("grid2x3", lambda: C.supremacy_grid(2, 3, 3, 0), [(4, 2), (5, 2), (3, 3)]),
]


@pytest.mark.parametrize("name,make,shapes", CASES, ids=[c[0] for c in CASES])
def test_cut_search_matches_enumeration(cq, name, make, shapes):
    circ = make()
    verts, _, _ = cs.graph(circ.n, circ.gates)
    assert len(verts) <= 11, "keep the enumeration small"
    for D, nC in shapes:
        want = cs.search(circ.n, circ.gates, D, nC)
        if want is None:
            with pytest.raises(cq.CutQCError) as ei:
                cq.cut_search(circ, D, nC)
            assert ei.value.status == cq.CUTQC_ERR_UNSUPPORTED
            continue
        got = cq.cut_search(circ, D, nC)
        assert got["cost"] == float(want["L"]) and got["K"] == want["K"], (D, nC)
        assert got["assign"] == want["assign"], (D, nC)


def test_cut_search_errors(cq):
    circ = C.hwea(6, 1)
    with pytest.raises(cq.CutQCError) as ei:
        cq.cut_search(circ, 1, 2)                 # nothing fits a 1-qubit device
    assert ei.value.status == cq.CUTQC_ERR_UNSUPPORTED
    with pytest.raises(cq.CutQCError) as ei:
        cq.cut_search(circ, 3, 2, max_nodes=1)    # node budget
    assert ei.value.status == cq.CUTQC_ERR_UNSUPPORTED
    with pytest.raises(cq.CutQCError) as ei:
        cq.cut_search(circ, 3, 17)
    assert ei.value.status == cq.CUTQC_ERR_UNSUPPORTED


def test_searched_cut_builds_valid_subcircuits(cq):
    """The subcircuits built from a searched assignment have the widths and
    cut count the search reports (d_c <= D, K cuts, outputs partition the
    qubits)."""
    circ = C.hwea(8, 2)
    r = cq.cut_search(circ, 5, 2)
    cc = C.cut_from_clusters(circ, r["gate_cluster"], max_width=5)
    assert cc.n_cuts == r["K"]
    assert max(s.d for s in cc.subs) <= 5
    assert sorted(q for s in cc.subs for _, q in s.outputs) == list(range(circ.n))


def test_free_qubits_join_subcircuits_within_the_width(cq):
    """Bernstein-Vazirani leaves the qubits of 0 secret bits without
    multi-qubit gates; they are packed into subcircuits within the width."""
    circ = C.bv(8, 3)
    r = cq.cut_search(circ, 5, 2)
    cc = C.cut_from_clusters(circ, r["gate_cluster"], max_width=5)
    assert cc.n_cuts == r["K"] and max(s.d for s in cc.subs) <= 5
    assert sorted(q for s in cc.subs for _, q in s.outputs) == list(range(circ.n))
