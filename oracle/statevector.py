"""Textbook statevector simulation in complex128 (the ground-truth mode of the
paper's Sec. 2 / Fig. 2a).  TEST INFRASTRUCTURE ONLY.

A state of d qubits is an ndarray of shape [B, 2, 2, ..., 2] (a batch of B
states); axis 1+q holds qubit q, so the row-major flattening puts qubit 0 in
the most significant bit (the paper's |q_0 ... q_{n-1}> order, Sec. 3.2).
"""
from __future__ import annotations

import numpy as np

_S2 = 1.0 / np.sqrt(2.0)


def gate_matrix(name: str, params=()) -> np.ndarray:
    """Unitary of a named gate (2x2 or 4x4; for two-qubit gates the first
    listed qubit is the more significant index bit)."""
    i = 1j
    if name == "h":
        return np.array([[1, 1], [1, -1]], complex) * _S2
    if name == "x":
        return np.array([[0, 1], [1, 0]], complex)
    if name == "y":
        return np.array([[0, -i], [i, 0]], complex)
    if name == "z":
        return np.array([[1, 0], [0, -1]], complex)
    if name == "s":
        return np.array([[1, 0], [0, i]], complex)
    if name == "sdg":
        return np.array([[1, 0], [0, -i]], complex)
    if name == "t":
        return np.array([[1, 0], [0, np.exp(i * np.pi / 4)]], complex)
    if name in ("sx", "sy", "sw"):
        # square root of a Hermitian involution P: ((1+i) I + (1-i) P) / 2
        P = {"sx": gate_matrix("x"), "sy": gate_matrix("y"),
             "sw": (gate_matrix("x") + gate_matrix("y")) * _S2}[name]
        return ((1 + i) * np.eye(2) + (1 - i) * P) / 2
    if name == "rx":
        t = params[0] / 2
        return np.array([[np.cos(t), -i * np.sin(t)], [-i * np.sin(t), np.cos(t)]], complex)
    if name == "ry":
        t = params[0] / 2
        return np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]], complex)
    if name == "rz":
        t = params[0] / 2
        return np.array([[np.exp(-i * t), 0], [0, np.exp(i * t)]], complex)
    if name == "cz":
        return np.diag([1, 1, 1, -1]).astype(complex)
    if name == "cx":
        return np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], complex)
    if name == "cp":
        return np.diag([1, 1, 1, np.exp(i * params[0])]).astype(complex)
    raise ValueError(f"unknown gate {name}")


def apply_gate(psi: np.ndarray, U: np.ndarray, qubits) -> np.ndarray:
    """Apply a k-qubit unitary to the given qubit axes of a batched state."""
    k = len(qubits)
    axes = [1 + q for q in qubits]
    Ut = U.reshape([2] * (2 * k))
    # contract U's input indices with the state's qubit axes
    out = np.tensordot(Ut, psi, axes=(list(range(k, 2 * k)), axes))
    # tensordot puts U's output indices first: move them back into place
    return np.moveaxis(out, list(range(k)), axes)


def run(psi: np.ndarray, gates) -> np.ndarray:
    for g in gates:
        psi = apply_gate(psi, gate_matrix(g.name, g.params), g.qubits)
    return psi


def zero_state(d: int, batch: int = 1) -> np.ndarray:
    psi = np.zeros([batch] + [2] * d, complex)
    psi.reshape(batch, -1)[:, 0] = 1.0
    return psi


def probabilities(circuit) -> np.ndarray:
    """Brute-force output distribution of an uncut circuit: |<x|U|0>|^2 over
    all 2^n x, qubit 0 = most significant bit."""
    psi = run(zero_state(circuit.n), circuit.gates)
    return (np.abs(psi) ** 2).reshape(-1)
