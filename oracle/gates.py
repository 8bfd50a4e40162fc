"""Gate matrices of the oracle (test infrastructure only).

The paper uses Hadamard, CNOT, CZ, Pauli X/Z and multi-controlled X (Sec. 2,
Sec. 5.3, Sec. 5.4) and supports custom gates.  Gates the workloads need beyond
those follow the OpenQASM 2 definitions, which QCLAB's QASM export (Sec. 4)
targets:

* U3(theta, phi, lam) = [[cos(theta/2), -e^{i lam} sin(theta/2)],
                         [e^{i phi} sin(theta/2), e^{i(phi+lam)} cos(theta/2)]]
* RX(t) = exp(-i t X/2), RY(t) = exp(-i t Y/2), RZ(t) = exp(-i t Z/2) = diag(e^{-it/2}, e^{it/2})
* CP(phi) = diag(1, 1, 1, e^{i phi})
* Y-basis change: S^dagger then H (so that |+i> measures as outcome 0).
"""
from __future__ import annotations

import numpy as np

SQ2 = 1.0 / np.sqrt(2.0)
I2 = np.eye(2, dtype=np.complex128)
H = np.array([[SQ2, SQ2], [SQ2, -SQ2]], dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
T = np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
PAULI = {"I": I2, "X": X, "Y": Y, "Z": Z}


def rx(t):
    c, s = np.cos(t / 2), np.sin(t / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def ry(t):
    c, s = np.cos(t / 2), np.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(t):
    return np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]], dtype=np.complex128)


def u3(theta, phi, lam):
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def phase(phi):
    return np.array([[1, 0], [0, np.exp(1j * phi)]], dtype=np.complex128)


def controlled(U: np.ndarray) -> np.ndarray:
    """|0><0| (x) I + |1><1| (x) U for a 2x2 U (control is the first factor)."""
    out = np.eye(4, dtype=np.complex128)
    out[2:, 2:] = U
    return out


def generator(kind: str) -> np.ndarray:
    """G in U(t) = exp(-i t G / 2) for the rotation kinds."""
    return {"rx": X, "ry": Y, "rz": Z}[kind]


def one_qubit(kind: str, params) -> np.ndarray:
    if kind == "h":
        return H
    if kind == "x":
        return X
    if kind == "y":
        return Y
    if kind == "z":
        return Z
    if kind == "s":
        return S
    if kind == "sdg":
        return S.conj().T
    if kind == "t":
        return T
    if kind == "tdg":
        return T.conj().T
    if kind == "rx":
        return rx(params[0])
    if kind == "ry":
        return ry(params[0])
    if kind == "rz":
        return rz(params[0])
    if kind == "u3":
        return u3(*params)
    raise ValueError(kind)
