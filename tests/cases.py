"""Seeded workloads shared by the GPU parity tests (structure only; the
tensors come from the FP64 oracle in the tests themselves)."""
from paper_2012_02333_gb300 import circuits as C

# small cases: span several 128-wide tiles and a ragged tail in at least one
# operand, several group merges, and the degenerate shapes
SMALL = {
    "hwea10_k1": lambda: C.hwea_10q_k1(0),                                  # config 1 shape
    "bv6_k1": lambda: C.chain_blocks(C.bv(6, 1), 2, max_width=4),           # sparse, zero rows
    "grid3x4_k3": lambda: C.grid_blocks(3, 4, 8, 1, 1, 2, 6, 9),
    "qaoa8_k4": lambda: C.qaoa_2cluster(4, 1),
    "aqft8_k4": lambda: C.chain_blocks(C.aqft(8, 0), 2, max_cuts=6),         # a subcircuit with n_eff = 0
    "hwea9_s3": lambda: C.chain_blocks(C.hwea(9, 2), 3),                     # one merge
    "grid4x4_s4": lambda: C.grid_blocks(4, 4, 6, 3, 2, 2, 8, 7),             # three merges
    "grid4x5_k5": lambda: C.grid_blocks(4, 5, 8, 2, 1, 2, 5, 13),            # multi-tile, 2 subcircuits
    "hwea16_s2": lambda: C.chain_blocks(C.hwea(16, 4), 2),                   # 2^8 x 2^8 tiles
    "nocut6": lambda: C.cut_circuit(C.hwea(6, 4), [0] * 6),                  # S = 1, K = 0
    "hwea14_skinny": lambda: C.cut_circuit(C.hwea(14, 6), [0] * 11 + [1] * 3),  # 2^11 x 2^3 outputs
}


def hwea22_chain():
    """22-qubit HWEA cut once between qubits 10 and 11 (2 subcircuits, K = 1)."""
    return C.chain_blocks(C.hwea(22, 5), 2)


def supremacy_4x6():
    """4x6 supremacy grid, depth 8, 2 subcircuits of <= 15 qubits (K = 4)."""
    return C.supremacy_4x6(0)


def dd_twin():
    """Scaled twin of the 80-qubit dynamic-definition workload: a 4x5 grid of
    depth 10 cut into 2x2 blocks (4 subcircuits), K <= 8."""
    return C.grid_blocks(4, 5, 10, 0, 2, 2, 8, 10)


def hwea26_chain():
    """26-qubit HWEA cut once between qubits 12 and 13: 2^13 x 2^13 outputs."""
    return C.chain_blocks(C.hwea(26, 7), 2)


def k8_pair():
    """A 6-qubit circuit whose middle wires cross between two 3-qubit halves
    nine times: two subcircuits (8 and 6 qubits) joined by K = 8 cuts, so
    4^8 = 65536 Kronecker terms over 2^6 outputs."""
    c = C.Circuit(6, [], "k8")
    for q in range(6):
        c.add("h", q)
    for layer in range(4):
        for q in range(6):
            c.add("ry", q, params=[0.3 + 0.1 * q + 0.2 * layer])
        c.add("cz", 2, 3)
        c.add("rz", 3, params=[0.7 + 0.1 * layer])
        c.add("cx", 3, 4)
        c.add("cz", 0, 1)
        c.add("cx", 1, 2)
        c.add("cz", 4, 5)
    c.add("ry", 3, params=[0.4])
    c.add("cz", 2, 3)
    cc = C.cut_circuit(c, [0, 0, 0, 1, 1, 1], policy="first")
    assert cc.n_cuts == 8 and len(cc.subs) == 2
    return cc
