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
