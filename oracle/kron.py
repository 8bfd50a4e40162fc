"""The paper's gate application written literally (QCLAB Sec. 3.2):
U = I_l (x) U' (x) I_r, with dense numpy Kronecker products (test infrastructure,
n <= 10).

For a gate on qubits spanning [a, b] (qubit 0 leftmost), I_l has dimension 2^a and
I_r has dimension 2^(n-1-b).  When the gate's qubits are not the whole span, or are
given out of order, U' is the 2^(b-a+1) operator on the span that acts as U on the
gate's qubits (first listed qubit = most significant row bit) and as the identity on
the span's other qubits; it is built entry by entry from that statement.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import gates
from . import op_matrix


def span_operator(U: np.ndarray, qubits: Sequence[int]) -> tuple:
    a, b = min(qubits), max(qubits)
    w = b - a + 1
    k = len(qubits)
    D = 1 << w
    Up = np.zeros((D, D), dtype=np.complex128)
    others = [q for q in range(a, b + 1) if q not in qubits]

    def bit(x, q):  # bit of qubit q inside the span index x (qubit a is the MSB)
        return (x >> (b - q)) & 1

    for r in range(D):
        for c in range(D):
            if any(bit(r, q) != bit(c, q) for q in others):
                continue
            rr = sum(bit(r, q) << (k - 1 - j) for j, q in enumerate(qubits))
            cc = sum(bit(c, q) << (k - 1 - j) for j, q in enumerate(qubits))
            Up[r, c] = U[rr, cc]
    return Up, a, b


def register_operator(n: int, U: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    Up, a, b = span_operator(U, qubits)
    return np.kron(np.kron(np.eye(1 << a), Up), np.eye(1 << (n - 1 - b)))


def controlled_operator(U: np.ndarray, nctrl: int, states: Sequence[int]) -> np.ndarray:
    """Operator on (controls..., target) that applies U iff the controls read
    ``states`` and the identity otherwise."""
    D = 1 << (nctrl + 1)
    M = np.eye(D, dtype=np.complex128)
    pat = 0
    for s in states:
        pat = (pat << 1) | int(s)
    base = pat << 1
    M[base:base + 2, base:base + 2] = U
    return M


def op_register_matrix(n: int, op, params=None) -> np.ndarray:
    form, U = op_matrix(op, params)
    if form == "ctrl":
        nctrl = len(op.qubits) - 1
        states = op.ctrl_states if op.ctrl_states is not None else (1,) * nctrl
        return register_operator(n, controlled_operator(U, nctrl, states), op.qubits)
    return register_operator(n, U, op.qubits)


def apply(psi: np.ndarray, n: int, ops, params=None) -> np.ndarray:
    out = np.array(psi, dtype=np.complex128)
    for op in ops:
        out = op_register_matrix(n, op, params) @ out
    return out


def circuit_unitary(n: int, ops, params=None) -> np.ndarray:
    M = np.eye(1 << n, dtype=np.complex128)
    for op in ops:
        M = op_register_matrix(n, op, params) @ M
    return M


def pauli_matrix(s: str) -> np.ndarray:
    M = np.eye(1, dtype=np.complex128)
    for c in s:
        M = np.kron(M, gates.PAULI[c])
    return M
