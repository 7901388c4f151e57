"""Subcircuit variants and shot attribution into Pauli-indexed tensors.
TEST INFRASTRUCTURE ONLY.

Sec. 3.1 (Eq. 1, Eq. 2, Fig. 3): cutting a wire decomposes the state on it as
  rho = 1/2 sum_{M in {I,X,Y,Z}} Tr(rho M) M .
Upstream of a cut the trace Tr(rho M) is a measurement of the cut qubit in the
M basis (I and Z share one circuit, so there are 3 physical variants); downstream
the operator M is prepared as a combination of eigenstate initialisations
(Eq. 2): I = |0><0| + |1><1|, Z = |0><0| - |1><1|, X = 2|+><+| - I,
Y = 2|+i><+i| - I (4 physical variants).

For one subcircuit with k_in init slots and k_out measurement slots this module
 1. simulates the 4^k_in x 3^k_out physical variants (Fig. 3, Fig. 4);
 2. attributes each measured cut qubit's outcome with the +-1 factor of Eq. 3
    (basis I: both outcomes count +1; otherwise outcome 0 -> +1, 1 -> -1);
 3. combines the init variants as in Eq. 2 (the p_{2,i} formulas of
    Sec. 3.2.2), giving T[a][b][x] with a, b in {I,X,Y,Z}^k (digit order
    I=0, X=1, Y=2, Z=3; slot 0 most significant) and x the effective outputs
    (bit 0 = lowest global qubit = most significant).

The paper pairs the I and Z terms as (I+Z) with |0> and (I-Z) with |1>
(Eq. 2, A1 and A2); since (I+Z)(x)|0><0| + (I-Z)(x)|1><1| = I(x)I + Z(x)Z this is
the same sum as the plain Pauli pairing used here; a test checks both.
"""
from __future__ import annotations

import itertools
import string

import numpy as np

from . import statevector as sv

_S2 = 1.0 / np.sqrt(2.0)
# physical initial states of an init qubit: |0>, |1>, |+>, |+i>
INIT_STATES = np.array([[1, 0], [0, 1], [_S2, _S2], [_S2, 1j * _S2]], complex)
# physical measurement bases of a measured cut qubit: Z (also serves I), X, Y
MEAS_BASES = ("Z", "X", "Y")

# Eq. 2: coefficient of physical init s in Pauli operator a (rows I, X, Y, Z)
INIT_COEF = np.array([
    [1.0, 1.0, 0.0, 0.0],    # I = |0><0| + |1><1|
    [-1.0, -1.0, 2.0, 0.0],  # X = 2|+><+| - |0><0| - |1><1|
    [-1.0, -1.0, 0.0, 2.0],  # Y = 2|+i><+i| - |0><0| - |1><1|
    [1.0, -1.0, 0.0, 0.0],   # Z = |0><0| - |1><1|
])

# Eq. 3: weight of (physical basis mb, outcome m) for Pauli b (rows I, X, Y, Z)
MEAS_WEIGHT = np.zeros((4, 3, 2))
MEAS_WEIGHT[0, 0] = (1.0, 1.0)    # I: Z-basis circuit, both outcomes +
MEAS_WEIGHT[1, 1] = (1.0, -1.0)   # X: X-basis circuit, 0 -> +, 1 -> -
MEAS_WEIGHT[2, 2] = (1.0, -1.0)   # Y: Y-basis circuit
MEAS_WEIGHT[3, 0] = (1.0, -1.0)   # Z: Z-basis circuit


def variant_probabilities(sub) -> np.ndarray:
    """Output distribution of every physical variant of a subcircuit.

    Returns p[s][mb][y] of shape (4^k_in, 3^k_out, 2^d): s enumerates the
    init states of the init slots (slot 0 most significant, INIT_STATES
    order), mb the measurement bases of the measurement slots (MEAS_BASES
    order), y the subcircuit's d local qubits (local qubit 0 most significant).
    Original inputs start in |0>.  The X basis is measured after H, the Y
    basis after S^dagger then H (outcome 0 <-> eigenvalue +1)."""
    d, kin, kout = sub.d, sub.k_in, sub.k_out
    B = 4 ** kin
    psi = np.zeros([B] + [2] * d, complex)
    init_q = {lq: j for j, (lq, _) in enumerate(sub.in_slots)}
    for s, digits in enumerate(itertools.product(range(4), repeat=kin)):
        v = np.ones(1, complex)
        for q in range(d):
            vec = INIT_STATES[digits[init_q[q]]] if q in init_q else INIT_STATES[0]
            v = np.kron(v, vec)
        psi[s] = v.reshape([2] * d)
    psi = sv.run(psi, sub.gates)
    out = np.empty((B, 3 ** kout, 2 ** d))
    H = sv.gate_matrix("h")
    SDG = sv.gate_matrix("sdg")
    for mi, bases in enumerate(itertools.product(range(3), repeat=kout)):
        phi = psi
        for j, basis in enumerate(bases):
            lq = sub.out_slots[j][0]
            if MEAS_BASES[basis] == "X":
                phi = sv.apply_gate(phi, H, (lq,))
            elif MEAS_BASES[basis] == "Y":
                phi = sv.apply_gate(phi, H @ SDG, (lq,))
        out[:, mi, :] = (np.abs(phi) ** 2).reshape(B, -1)
    return out


def _letters(k, start):
    return string.ascii_letters[start:start + k]


def attribute(sub, p: np.ndarray, snap: float = 2.0 ** -40) -> np.ndarray:
    """Attributed tensor T[a][b][x] of shape (4^k_in, 4^k_out, 2^n_eff) from
    the variant distributions of `variant_probabilities` (Eq. 3 then Eq. 2).
    Entries with |T| < snap become exactly 0 (they are rounding residue of
    terms that vanish exactly; the early-termination test of Sec. 4.2 then sees
    true zeros)."""
    d, kin, kout, f = sub.d, sub.k_in, sub.k_out, sub.n_eff
    arr = p.reshape([4] * kin + [3] * kout + [2] * d)
    # local qubit axes -> (measured cut qubits in slot order, outputs in order)
    q0 = kin + kout
    meas_axes = [q0 + lq for lq, _ in sub.out_slots]
    out_axes = [q0 + lq for lq, _ in sub.outputs]
    arr = arr.transpose(list(range(q0)) + meas_axes + out_axes)
    S = _letters(kin, 0)            # physical inits
    MB = _letters(kout, 10)         # physical measurement bases
    M = _letters(kout, 20)          # measured outcomes
    Bp = _letters(kout, 30)         # Pauli b digits
    A = _letters(kin, 40)           # Pauli a digits
    X = "Z"                          # flattened outputs
    arr = arr.reshape([4] * kin + [3] * kout + [2] * kout + [2 ** f])
    # Step 1, Eq. 3: sign-weighted sums over each measured cut qubit's outcome
    ops = [arr] + [MEAS_WEIGHT] * kout
    subs = [S + MB + M + X] + [Bp[j] + MB[j] + M[j] for j in range(kout)]
    P = np.einsum(",".join(subs) + "->" + S + Bp + X, *ops, optimize=True) if kout else arr
    # Step 2, Eq. 2: combine the physical inits into Pauli operators
    ops = [P] + [INIT_COEF] * kin
    subs = [S + Bp + X] + [A[j] + S[j] for j in range(kin)]
    T = np.einsum(",".join(subs) + "->" + A + Bp + X, *ops, optimize=True) if kin else P
    T = np.ascontiguousarray(T).reshape(4 ** kin, 4 ** kout, 2 ** f)
    T[np.abs(T) < snap] = 0.0
    return T


def attribute_merged(sub, p: np.ndarray, roles, snap: float = 2.0 ** -40) -> np.ndarray:
    """The merged tensor one recursion of Algorithm 1 contracts, taken from the
    variant distributions: the attributed tensor (Eq. 3 then Eq. 2,
    `attribute`) merged over the recursion's roles (`reconstruct.merge`:
    zoomed outputs fixed at their bit, merged outputs summed, active outputs
    kept in output order).  roles[q] is indexed by global qubit (0 active,
    1 merged, 2 zoomed at 0, 3 zoomed at 1).  Shape (4^k_in * 4^k_out,
    2^#active outputs)."""
    from .reconstruct import merge
    return merge(sub, attribute(sub, p, snap), roles)


def subcircuit_tensor(sub) -> np.ndarray:
    """T_c for one subcircuit, in float64."""
    return attribute(sub, variant_probabilities(sub))


def tensors(cc):
    """FP64 tensors of every subcircuit of a cut circuit."""
    return [subcircuit_tensor(s) for s in cc.subs]
