"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module holds circuit *descriptions* (which gate kind acts on which qubits,
with which angles or which caller-supplied matrix) and random input data.  It
holds none of the simulation arithmetic: no gate matrix is built here from a
gate name, no amplitude is updated, no probability is formed.  Both sides turn
the descriptions below into matrices with their own code.

Conventions (QCLAB, Sec. 3.2 and the teleportation example of Sec. 5.1):
qubit 0 is the leftmost Kronecker factor, i.e. the most significant bit of the
amplitude index, so ``i = sum_q b_q * 2**(n-1-q)``.

Random sources
--------------
* numpy ``default_rng(seed)`` (PCG64) for angles, Haar matrices, circuit sizes and
  sampling uniforms.
* A counter-based SplitMix64 stream (Steele, Lea and Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014) for Gaussian start states, so that
  an amplitude can be regenerated from its index alone.  The CUDA path and the
  oracle each implement the same published generator for states too large to
  pass through host memory; :func:`gaussian_state` is the host version used for
  everything that fits.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence, Tuple

import numpy as np

TWO_PI = 2.0 * np.pi

# ---------------------------------------------------------------------------
# Circuit description
# ---------------------------------------------------------------------------

#: gate kinds understood by both sides.  Single-qubit kinds take ``qubits=(q,)``;
#: two-qubit kinds take ``qubits=(a, b)``; ``mcx``/``ctrl`` take
#: ``qubits=(c_0, ..., c_{m-1}, target)`` plus ``ctrl_states``.
KINDS_1Q = ("h", "x", "y", "z", "s", "sdg", "t", "tdg", "rx", "ry", "rz", "u3", "u1q")
KINDS_2Q = ("cnot", "cz", "cp", "swap", "u2q")
KINDS_MC = ("mcx", "ctrl")
KINDS_K = ("ukq",)
PARAM_COUNT = {"rx": 1, "ry": 1, "rz": 1, "u3": 3, "cp": 1}


@dataclass(frozen=True)
class Op:
    """One circuit operation.

    kind        gate kind (see ``KINDS_*``)
    qubits      qubit indices; for controlled kinds the target is last
    params      inline angles (radians), used when ``param_index`` is None
    matrix      complex matrix for ``u1q``/``u2q``/``ukq``/``ctrl`` (row index
                uses ``qubits[0]`` as the most significant bit)
    ctrl_states required control values for ``mcx``/``ctrl`` (default all 1)
    param_index index into an external parameter vector (parameterised
                circuits, e.g. the adjoint-gradient ansatz)
    """

    kind: str
    qubits: Tuple[int, ...]
    params: Tuple[float, ...] = ()
    matrix: Optional[np.ndarray] = field(default=None, compare=False)
    ctrl_states: Optional[Tuple[int, ...]] = None
    param_index: Optional[int] = None


# ---------------------------------------------------------------------------
# Random data
# ---------------------------------------------------------------------------

def haar_unitaries(count: int, dim: int, seed: int) -> np.ndarray:
    """``count`` Haar-random ``dim x dim`` unitaries (Mezzadri, "How to generate
    random matrices from the classical compact groups", Notices AMS 2007):
    Z = (A + iB)/sqrt(2) with A, B standard normal, Q R = qr(Z), U = Q diag(R_jj/|R_jj|).
    Draws ``standard_normal((count, 2, dim, dim))`` from ``default_rng(seed)``."""
    g = np.random.default_rng(seed).standard_normal((count, 2, dim, dim))
    z = (g[:, 0] + 1j * g[:, 1]) / np.sqrt(2.0)
    out = np.empty((count, dim, dim), dtype=np.complex128)
    for c in range(count):
        q, r = np.linalg.qr(z[c])
        d = np.diag(r)
        out[c] = q * (d / np.abs(d))[None, :]
    return out


def uniforms(count: int, seed: int) -> np.ndarray:
    """``count`` FP64 uniforms in [0, 1) from ``default_rng(seed)``."""
    return np.random.default_rng(seed).random(count)


_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_SM_M1 = np.uint64(0xBF58476D1CE4E5B9)
_SM_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64: output ``c`` of the stream seeded with ``seed`` is
    mix(seed + (c + 1) * 0x9E3779B97F4A7C15) with the published finaliser
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
    z ^= z >> 31 (all arithmetic modulo 2**64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * _SM_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _SM_M1
        z = (z ^ (z >> np.uint64(27))) * _SM_M2
        return z ^ (z >> np.uint64(31))


def splitmix_uniform(seed: int, counters: np.ndarray) -> np.ndarray:
    """53-bit uniforms in [0, 1): (output >> 11) * 2**-53."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian_amplitudes(seed: int, start: int, count: int) -> np.ndarray:
    """Unnormalised complex Gaussian amplitudes ``start .. start+count-1``.

    Amplitude j uses uniforms u1 = U(2j), u2 = U(2j+1) of the SplitMix64 stream and the
    Box-Muller transform (Box and Muller, Ann. Math. Stat. 1958):
    r = sqrt(-2 ln(1 - u1)), re = r cos(2 pi u2), im = r sin(2 pi u2)."""
    j = np.arange(start, start + count, dtype=np.uint64)
    u1 = splitmix_uniform(seed, 2 * j)
    u2 = splitmix_uniform(seed, 2 * j + np.uint64(1))
    r = np.sqrt(-2.0 * np.log1p(-u1))
    t = TWO_PI * u2
    return r * np.cos(t) + 1j * (r * np.sin(t))


def gaussian_state(n: int, seed: int) -> np.ndarray:
    """Normalised complex Gaussian state on n qubits (complex128)."""
    x = gaussian_amplitudes(seed, 0, 1 << n)
    return x / np.sqrt(np.sum(x.real * x.real + x.imag * x.imag))


def random_state(n: int, seed: int) -> np.ndarray:
    """Small normalised random state from ``default_rng(seed)`` for unit tests."""
    g = np.random.default_rng(seed).standard_normal((2, 1 << n))
    x = g[0] + 1j * g[1]
    return x / np.linalg.norm(x)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def u3_ladder(n: int = 10, layers: int = 20, seed: int = 1) -> list:
    """U3 on every qubit then a CNOT ladder q_i -> q_{i+1}, ``layers`` times.
    Angles ``default_rng(seed).uniform(0, 2pi, (layers, n, 3))`` in the order
    layer -> qubit -> (theta, phi, lambda)."""
    ang = np.random.default_rng(seed).uniform(0.0, TWO_PI, (layers, n, 3))
    ops = []
    for l in range(layers):
        for q in range(n):
            ops.append(Op("u3", (q,), tuple(float(a) for a in ang[l, q])))
        for q in range(n - 1):
            ops.append(Op("cnot", (q, q + 1)))
    return ops


def brickwork(n: int = 28, depth: int = 40, seed: int = 2) -> list:
    """Brickwork of Haar-random two-qubit unitaries: even layers act on pairs
    (0,1), (2,3), ...; odd layers on (1,2), (3,4), ...; layer 0 is even.  The
    unitaries are drawn once, in circuit order, by :func:`haar_unitaries`."""
    pairs = []
    for l in range(depth):
        start = 0 if l % 2 == 0 else 1
        pairs.extend((a, a + 1) for a in range(start, n - 1, 2))
    mats = haar_unitaries(len(pairs), 4, seed)
    return [Op("u2q", p, matrix=mats[i]) for i, p in enumerate(pairs)]


def window_chain(n: int, first: int, width: int, count: int, seed: int) -> list:
    """`count` Haar-random two-qubit unitaries in brickwork order on the neighbouring
    pairs of qubits first .. first+width-1 only (a deep circuit on a window of the
    register); drawn by :func:`haar_unitaries`."""
    pairs = []
    layer = 0
    while len(pairs) < count:
        start = 0 if layer % 2 == 0 else 1
        pairs.extend((first + a, first + a + 1) for a in range(start, width - 1, 2))
        layer += 1
    pairs = pairs[:count]
    mats = haar_unitaries(len(pairs), 4, seed)
    return [Op("u2q", p, matrix=mats[i]) for i, p in enumerate(pairs)]


def qft(n: int) -> list:
    """Textbook quantum Fourier transform with qubit 0 as the most significant
    bit: for j = 0..n-1, H(q_j) then CP(2 pi / 2**k) on (q_{j+k-1}, q_j) for
    k = 2..n-j; then SWAP(q_j, q_{n-1-j}) for j < n/2."""
    ops = []
    for j in range(n):
        ops.append(Op("h", (j,)))
        for k in range(2, n - j + 1):
            ops.append(Op("cp", (j + k - 1, j), (TWO_PI / float(2 ** k),)))
    for j in range(n // 2):
        ops.append(Op("swap", (j, n - 1 - j)))
    return ops


def ansatz(n: int, layers: int, ring: bool) -> list:
    """Hardware-efficient ansatz: per layer RY(theta) then RZ(theta) on every
    qubit, then CZ(i, i+1) for i = 0..n-2 in ascending order (plus CZ(n-1, 0)
    when ``ring``).  Parameter index = layer*2n + 2q + {0: RY, 1: RZ}."""
    ops = []
    for l in range(layers):
        for q in range(n):
            ops.append(Op("ry", (q,), param_index=l * 2 * n + 2 * q))
            ops.append(Op("rz", (q,), param_index=l * 2 * n + 2 * q + 1))
        for q in range(n - 1):
            ops.append(Op("cz", (q, q + 1)))
        if ring and n > 2:
            ops.append(Op("cz", (n - 1, 0)))
    return ops


def ansatz_params(n: int, layers: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, TWO_PI, layers * 2 * n)


def zz_terms(n: int, ring: bool) -> list:
    """Pauli strings of sum_i Z_i Z_{i+1} (chain, or ring with Z_{n-1} Z_0)."""
    out = []
    last = n if ring else n - 1
    for i in range(last):
        s = ["I"] * n
        s[i] = "Z"
        s[(i + 1) % n] = "Z"
        out.append("".join(s))
    return out


def x_terms(n: int) -> list:
    out = []
    for i in range(n):
        s = ["I"] * n
        s[i] = "X"
        out.append("".join(s))
    return out


def adjoint_workload(n: int = 24, layers: int = 10, seed: int = 5):
    """Ansatz with a CZ ring; H = sum_ring Z_i Z_{i+1} + 1.0 * sum_i X_i."""
    ops = ansatz(n, layers, ring=True)
    params = ansatz_params(n, layers, seed)
    terms = zz_terms(n, ring=True) + x_terms(n)
    coeffs = np.ones(len(terms))
    return ops, params, terms, coeffs


def batch_workload(count: int = 4096, layers: int = 8, nmin: int = 12, nmax: int = 20, seed: int = 4):
    """``count`` ansatz circuits (CZ chain) with qubit counts uniform in
    [nmin, nmax]; returns (qubit counts, list of parameter vectors)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    params = [rng.uniform(0.0, TWO_PI, layers * 2 * int(m)) for m in ns]
    return ns.astype(np.int64), params


def circuit_inverse(ops: Sequence[Op]) -> list:
    """The inverse circuit as a description: reverse order, each op marked with
    ``kind + '_dag'`` handled by each side's own matrix code."""
    return [Op(o.kind + "_dag" if not o.kind.endswith("_dag") else o.kind[:-4],
               o.qubits, o.params, o.matrix, o.ctrl_states, o.param_index) for o in reversed(ops)]
