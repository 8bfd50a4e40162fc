"""Reader for the small text fixtures under tests/golden (paper worked examples)."""
from __future__ import annotations

import os

import numpy as np

from workloads import Op

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            out[k.strip()] = v.strip()
    return out


def cvec(s: str) -> np.ndarray:
    return np.array([complex(t) for t in s.split()], dtype=np.complex128)


def fvec(s: str) -> np.ndarray:
    return np.array([float(t) for t in s.split()])


def ops(s: str) -> list:
    """'h 0; cnot 0 1; mcx 3 4 2 /01; measure 0' -> list of Op."""
    out = []
    for item in s.split(";"):
        tok = item.split()
        kind = tok[0]
        states = None
        if tok[-1].startswith("/"):
            states = tuple(int(c) for c in tok[-1][1:])
            tok = tok[:-1]
        out.append(Op(kind, tuple(int(t) for t in tok[1:]), ctrl_states=states))
    return out


def init_state(s: str, n: int):
    v = np.array([1, 1j]) / np.sqrt(2)
    if s == "kron_v_bell":
        return np.kron(v, np.array([1, 0, 0, 1]) / np.sqrt(2))
    if s == "kron_v_e0":
        e = np.zeros(1 << (n - 1))
        e[0] = 1
        return np.kron(v, e)
    return s  # bitstring
