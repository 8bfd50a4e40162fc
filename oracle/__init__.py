"""CPU oracle for the QCLAB state-vector method (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

Two independent forms of the paper's gate application (QCLAB Sec. 3.2,
U = I_l (x) U' (x) I_r):

* :mod:`oracle.kron` -- the formula literally: dense Kronecker products, n <= 10.
* this module -- the same map without forming the matrix, in plain C
  (``qc_oracle.c``), complex128, one gate per pass, usable up to 32 qubits.

Parity status of every function is listed in the header of ``qc_oracle.c`` and in
``tests/test_oracle_pins.py``; the printed tomography estimate of Sec. 5.2 and
MATLAB's ``rng(1)`` shot counts are *parity unpinned* (they depend on MATLAB's
generator and are internally inconsistent in the paper).
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import gates
from .build import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        U64 = ctypes.POINTER(ctypes.c_uint64)
        i64, c_int, c_double, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        sig = {
            "orc_apply_1q": (None, [D, c_int, c_int, D]),
            "orc_apply_kq": (None, [D, c_int, I, c_int, D]),
            "orc_apply_2q": (None, [D, c_int, c_int, c_int, D]),
            "orc_apply_ctrl": (None, [D, c_int, I, I, c_int, c_int, D]),
            "orc_probs": (None, [D, c_int, D]),
            "orc_outcome_prob": (c_double, [D, c_int, c_int, c_int]),
            "orc_collapse": (None, [D, c_int, c_int, c_int, c_double]),
            "orc_cdf": (None, [D, i64, D]),
            "orc_sample": (None, [D, i64, D, i64, U64]),
            "orc_inner": (None, [D, D, i64, D]),
            "orc_expect_masks": (None, [D, c_int, u64, u64, D]),
            "orc_gaussian_amplitudes": (None, [u64, i64, i64, D]),
            "orc_gaussian_norm2": (c_double, [u64, c_int]),
            "orc_dft_gaussian": (None, [u64, c_int, c_double, c_int, U64, c_int, D]),
            "orc_num_threads": (c_int, []),
            "orc_set_threads": (None, [c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(seq) -> Tuple[ctypes.Array, int]:
    arr = (ctypes.c_int * max(1, len(seq)))(*[int(x) for x in seq])
    return arr, len(seq)


def _mat(U: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(U, dtype=np.complex128)).view(np.float64).ravel().copy()


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(t: int) -> None:
    """Thread count of the oracle's parallel loops (for timing)."""
    lib().orc_set_threads(int(t))


# ---------------------------------------------------------------------------
# primitive maps (QCLAB Sec. 3.2 and Sec. 3.3)
# ---------------------------------------------------------------------------

def _n_of(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    assert psi.dtype == np.complex128 and psi.size == 1 << n
    return n


def apply_1q(psi: np.ndarray, q: int, U: np.ndarray) -> None:
    m = _mat(U)
    lib().orc_apply_1q(_dp(psi.view(np.float64)), _n_of(psi), int(q), _dp(m))


def apply_2q(psi: np.ndarray, qa: int, qb: int, U: np.ndarray) -> None:
    m = _mat(U)
    lib().orc_apply_2q(_dp(psi.view(np.float64)), _n_of(psi), int(qa), int(qb), _dp(m))


def apply_kq(psi: np.ndarray, qubits: Sequence[int], U: np.ndarray) -> None:
    m = _mat(U)
    qs, k = _ip(qubits)
    lib().orc_apply_kq(_dp(psi.view(np.float64)), _n_of(psi), qs, k, _dp(m))


def apply_ctrl(psi: np.ndarray, ctrls: Sequence[int], states: Sequence[int], target: int, U: np.ndarray) -> None:
    m = _mat(U)
    cs, nc = _ip(ctrls)
    ss, _ = _ip(states)
    lib().orc_apply_ctrl(_dp(psi.view(np.float64)), _n_of(psi), cs, ss, nc, int(target), _dp(m))


def probs(psi: np.ndarray) -> np.ndarray:
    out = np.empty(psi.size, dtype=np.float64)
    lib().orc_probs(_dp(psi.view(np.float64)), _n_of(psi), _dp(out))
    return out


def outcome_prob(psi: np.ndarray, q: int, outcome: int) -> float:
    return float(lib().orc_outcome_prob(_dp(psi.view(np.float64)), _n_of(psi), int(q), int(outcome)))


def collapse(psi: np.ndarray, q: int, outcome: int, P: float) -> None:
    lib().orc_collapse(_dp(psi.view(np.float64)), _n_of(psi), int(q), int(outcome), float(P))


def cdf(p: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty_like(p)
    lib().orc_cdf(_dp(p), p.size, _dp(out))
    return out


def sample(c: np.ndarray, u: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(c, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(u.size, dtype=np.uint64)
    lib().orc_sample(_dp(c), c.size, _dp(u), u.size, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    out = np.zeros(2)
    lib().orc_inner(_dp(a.view(np.float64)), _dp(b.view(np.float64)), a.size, _dp(out))
    return complex(out[0], out[1])


def gaussian_state(n: int, seed: int) -> np.ndarray:
    """The workloads' SplitMix64/Box-Muller start state, generated by the oracle's own
    C code (used where the state is too large to hand over from the host)."""
    out = np.empty(1 << n, dtype=np.complex128)
    lib().orc_gaussian_amplitudes(ctypes.c_uint64(seed), 0, 1 << n, _dp(out.view(np.float64)))
    nrm2 = float(lib().orc_gaussian_norm2(ctypes.c_uint64(seed), n))
    out /= np.sqrt(nrm2)
    return out


def dft_gaussian_samples(n: int, seed: int, ks: Sequence[int], round_c64: bool) -> np.ndarray:
    """y_k = N^{-1/2} sum_j x_j e^{+2 pi i jk/N} of the normalised Gaussian state."""
    ks_arr = np.ascontiguousarray(np.asarray(ks, dtype=np.uint64))
    out = np.empty(2 * ks_arr.size)
    nrm2 = float(lib().orc_gaussian_norm2(ctypes.c_uint64(seed), n))
    lib().orc_dft_gaussian(ctypes.c_uint64(seed), n, nrm2, 1 if round_c64 else 0,
                           ks_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), ks_arr.size, _dp(out))
    return out[0::2] + 1j * out[1::2]


# ---------------------------------------------------------------------------
# circuits
# ---------------------------------------------------------------------------

def _params_of(op, params):
    if op.param_index is not None:
        k = {"cp": 1, "u3": 3}.get(op.kind.replace("_dag", ""), 1)
        return tuple(float(params[op.param_index + i]) for i in range(k))
    return op.params


def op_matrix(op, params=None) -> Tuple[str, np.ndarray]:
    """('1q'|'2q'|'ctrl'|'kq', matrix) for a description op; '_dag' kinds give U^dagger."""
    kind = op.kind
    dag = kind.endswith("_dag")
    if dag:
        kind = kind[:-4]
    p = _params_of(op, params)
    if kind in ("u1q", "u2q", "ukq", "ctrl"):
        U = np.asarray(op.matrix, dtype=np.complex128)
        form = {"u1q": "1q", "u2q": "2q", "ukq": "kq", "ctrl": "ctrl"}[kind]
    elif kind == "cnot":
        U, form = gates.X, "ctrl"
    elif kind == "cz":
        U, form = gates.Z, "ctrl"
    elif kind == "cp":
        U, form = gates.phase(p[0]), "ctrl"
    elif kind == "mcx":
        U, form = gates.X, "ctrl"
    elif kind == "swap":
        U, form = gates.SWAP, "2q"
    else:
        U, form = gates.one_qubit(kind, p), "1q"
    if dag:
        U = U.conj().T
    return form, U


def apply_op(psi: np.ndarray, op, params=None) -> None:
    form, U = op_matrix(op, params)
    if form == "1q":
        apply_1q(psi, op.qubits[0], U)
    elif form == "2q":
        apply_2q(psi, op.qubits[0], op.qubits[1], U)
    elif form == "kq":
        apply_kq(psi, op.qubits, U)
    else:
        ctrls = op.qubits[:-1]
        states = op.ctrl_states if op.ctrl_states is not None else (1,) * len(ctrls)
        apply_ctrl(psi, ctrls, states, op.qubits[-1], U)


def run(psi: np.ndarray, ops, params=None) -> np.ndarray:
    """Applies every gate of ``ops`` to ``psi`` in place, one pass per gate."""
    for op in ops:
        apply_op(psi, op, params)
    return psi


def basis_state(n: int, bits) -> np.ndarray:
    """Start state from a bitstring (character j is qubit j) or an integer index
    (QCLAB Sec. 3.1: ``simulate('00')`` equals ``simulate([1;0;0;0])``)."""
    if isinstance(bits, str):
        assert len(bits) == n
        idx = int(bits, 2)
    else:
        idx = int(bits)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[idx] = 1.0
    return psi


# ---------------------------------------------------------------------------
# measurement with outcome branching (QCLAB Sec. 3.3)
# ---------------------------------------------------------------------------

ZERO_PROB = 1e-12  # a branch whose probability is at most this is dropped


def simulate(n: int, ops, init, params=None, zero_prob: float = ZERO_PROB):
    """QCLAB's ``simulate``: runs ``ops`` (gates and 'measure' / 'measure_x' /
    'measure_y' / 'reset' ops) from ``init`` (bitstring or vector).  Every measurement
    with two possible outcomes splits the run into branches, outcome 0 first.  Returns
    (results, probabilities, states) with results the measured bits in measurement
    order.

    Reset (mentioned in Sec. 3.3, not defined there) is read as a Z measurement whose
    outcome-1 branch is then flipped by X, so the qubit ends in |0> on every branch;
    its outcome is part of the branch label like any measurement's."""
    psi = basis_state(n, init) if isinstance(init, (str, int)) else np.array(init, dtype=np.complex128)
    branches = [("", 1.0, psi)]
    for op in ops:
        if op.kind.startswith("measure") or op.kind == "reset":
            q = op.qubits[0]
            basis = "z" if op.kind == "reset" else op.kind[len("measure"):].lstrip("_") or "z"
            new = []
            for res, pr, st in branches:
                pre, post = _basis_change(basis)
                for U in pre:
                    apply_1q(st, q, U)
                for o in (0, 1):
                    P = outcome_prob(st, q, o)
                    if P <= zero_prob:
                        continue
                    s2 = st.copy()
                    collapse(s2, q, o, P)
                    for U in post:
                        apply_1q(s2, q, U)
                    if op.kind == "reset" and o == 1:
                        apply_1q(s2, q, gates.X)
                    new.append((res + str(o), pr * P, s2))
            branches = new
        else:
            for _, _, st in branches:
                apply_op(st, op, params)
    return [b[0] for b in branches], [b[1] for b in branches], [b[2] for b in branches]


def _basis_change(basis: str):
    """Gates before and after a Z measurement that realise a measurement in
    ``basis`` (Sec. 3.3: X is H, measure, H^dagger; Y is S^dagger H, measure, H S)."""
    if basis == "z":
        return [], []
    if basis == "x":
        return [gates.H], [gates.H.conj().T]
    if basis == "y":
        return [gates.S.conj().T, gates.H], [gates.H.conj().T, gates.S]
    raise ValueError(basis)


def reduced_statevector(psi: np.ndarray, known: Sequence[int], bits: str) -> np.ndarray:
    """QCLAB's ``reducedStatevector``: the amplitudes whose known qubits carry
    ``bits``, in the order of the remaining qubits (Sec. 5.1)."""
    n = _n_of(psi)
    rest = [q for q in range(n) if q not in known]
    out = np.empty(1 << len(rest), dtype=np.complex128)
    base = 0
    for q, b in zip(known, bits):
        if b == "1":
            base |= 1 << (n - 1 - q)
    for r in range(out.size):
        idx = base
        for j, q in enumerate(rest):
            if (r >> (len(rest) - 1 - j)) & 1:
                idx |= 1 << (n - 1 - q)
        out[r] = psi[idx]
    return out


# ---------------------------------------------------------------------------
# Pauli expectations and gradients
# ---------------------------------------------------------------------------

def expect_pauli(psi: np.ndarray, strings: Sequence[str], coeffs=None) -> np.ndarray:
    """<psi| P_t |psi> for every string (character j is the Pauli on qubit j),
    evaluated by applying each single-qubit Pauli to a copy and taking the inner
    product; multiplied by ``coeffs`` when given."""
    n = _n_of(psi)
    out = np.empty(len(strings))
    for t, s in enumerate(strings):
        assert len(s) == n
        phi = psi.copy()
        for q, c in enumerate(s):
            if c != "I":
                apply_1q(phi, q, gates.PAULI[c])
        out[t] = inner(psi, phi).real
    if coeffs is not None:
        out = out * np.asarray(coeffs, dtype=np.float64)
    return out


def expect_masks(psi: np.ndarray, terms) -> np.ndarray:
    """coeff * <psi| P |psi> for Pauli terms (xmask, zmask, coeff) on index bits:
    bit b set in x only is X on the qubit of index bit b (qubit n-1-b), in z only Z,
    in both Y.  Written from the definition P|j> = i^{|x&z|} (-1)^{|j&z|} |j^x>
    (``orc_expect_masks``); real part returned."""
    n = _n_of(psi)
    out = np.empty(len(terms))
    buf = np.zeros(2)
    for t, (x, z, c) in enumerate(terms):
        lib().orc_expect_masks(_dp(psi.view(np.float64)), n, ctypes.c_uint64(int(x)), ctypes.c_uint64(int(z)),
                               _dp(buf))
        out[t] = float(c) * buf[0]
    return out


def energy_masks(n: int, ops, params, terms) -> float:
    """<H> of the circuit's output from |0...0> for H given as mask terms."""
    psi = basis_state(n, 0)
    run(psi, ops, params)
    return float(np.sum(expect_masks(psi, terms)))


def energy(n: int, ops, params, strings, coeffs) -> float:
    psi = basis_state(n, 0)
    run(psi, ops, params)
    return float(np.sum(expect_pauli(psi, strings, coeffs)))


def param_shift_grad(n: int, ops, params, strings, coeffs, which=None) -> np.ndarray:
    """Exact gradient of <H> for rotations exp(-i t G/2) with G^2 = I.  For one gate,
    d<H>/dt = (<H>(t + pi/2) - <H>(t - pi/2)) / 2.  A parameter used by several gates
    gets the sum of the per-gate rules (chain rule): each occurrence is shifted on
    its own, through a private copy of the parameter."""
    from dataclasses import replace
    params = np.asarray(params, dtype=np.float64)
    idx = range(params.size) if which is None else which
    g = []
    for p in idx:
        total = 0.0
        for k, op in enumerate(ops):
            if op.param_index != p:
                continue
            own = list(ops)
            own[k] = replace(op, param_index=params.size)
            for sgn in (1.0, -1.0):
                ext = np.append(params, params[p] + sgn * np.pi / 2)
                total += 0.5 * sgn * energy(n, own, ext, strings, coeffs)
        g.append(total)
    return np.array(g)


def central_diff_grad(n: int, ops, params, strings, coeffs, h: float, which) -> np.ndarray:
    params = np.asarray(params, dtype=np.float64)
    g = []
    for p in which:
        a = params.copy()
        a[p] += h
        b = params.copy()
        b[p] -= h
        g.append((energy(n, ops, a, strings, coeffs) - energy(n, ops, b, strings, coeffs)) / (2 * h))
    return np.array(g)
