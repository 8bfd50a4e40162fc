"""Host-only check of the fused adjoint reverse sweep's plan (qc_adjoint_emulate; no GPU
needed): the passes, stages, op conditions and record positions the gradient launches,
applied on the host in FP64 to psi (the circuit's output) and lambda = H psi, give each
rotation's record Im <lambda|G|psi>, which is dE/dtheta; summed per parameter they must
equal the oracle's parameter-shift gradient.  The planner may move a record past gates
that commute with its generator; a move past one that does not changes the record by
order 1."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import gates
from workloads import Op

PAULI = {"X": gates.X, "Y": gates.Y, "Z": gates.Z}


def h_apply(psi, strings, coeffs):
    out = np.zeros_like(psi)
    for s, c in zip(strings, coeffs):
        x = psi.copy()
        for q, ch in enumerate(s):
            if ch != "I":
                oracle.apply_1q(x, q, PAULI[ch])
        out += c * x
    return out


def emulated_grad(n, ops, params, terms, coeffs, dtype):
    import paper_2503_03016_gb300 as P
    psi = oracle.run(oracle.basis_state(n, 0), ops, params)
    lam = h_apply(psi, terms, coeffs)
    rec = P.qc_adjoint_emulate(P.Circuit(n, ops), params, psi, lam, P.QC_C64 if dtype == "c64" else P.QC_C128)
    pidx = [o.param_index for o in ops if o.param_index is not None]
    g = np.zeros(len(params))
    for r, p in enumerate(pidx):
        g[p] += rec[r]
    return g


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [12, 15])
def test_ansatz_ring(dtype, n):
    ops, params, terms, coeffs = W.adjoint_workload(n, 3, 5)
    g = emulated_grad(n, ops, params, terms, coeffs, dtype)
    np.testing.assert_allclose(g, oracle.param_shift_grad(n, ops, params, terms, coeffs), atol=1e-12, rtol=0)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_mixed_generators_shared_parameters_and_fixed_gates(dtype):
    """RX, RY and RZ on random qubits sharing 12 parameters, among H, T, CNOT, CZ and
    controlled phases on random pairs; H = ZZ + X terms and a Y string."""
    n = 13
    rng = np.random.default_rng(3)
    ops = []
    for i in range(90):
        c = int(rng.integers(0, 7))
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        if c < 3:
            ops.append(Op(["rx", "ry", "rz"][c], (a,), param_index=int(rng.integers(0, 12))))
        elif c == 3:
            ops.append(Op("h", (a,)))
        elif c == 4:
            ops.append(Op("cnot", (a, b)))
        elif c == 5:
            ops.append(Op("cz", (a, b)))
        else:
            ops += [Op("t", (a,)), Op("cp", (a, b), (float(rng.uniform(0, 6.3)),))]
    params = rng.uniform(0, 2 * np.pi, 12)
    terms = W.zz_terms(n, ring=True) + W.x_terms(n) + ["Y" * 3 + "I" * (n - 3)]
    coeffs = np.linspace(0.5, 1.5, len(terms))
    g = emulated_grad(n, ops, params, terms, coeffs, dtype)
    np.testing.assert_allclose(g, oracle.param_shift_grad(n, ops, params, terms, coeffs), atol=1e-12, rtol=0)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_swaps_haar_gates_and_random_pauli_sums(dtype, seed):
    """Rotations between SWAPs, Haar two-qubit gates, CNOT, CZ and controlled phases on
    random qubits; H a sum of random 1- to 3-qubit X/Y/Z strings with signed weights."""
    n = 13
    rng = np.random.default_rng(seed)
    npar = 9
    ops = []
    for i in range(100):
        c = int(rng.integers(0, 9))
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        if c < 3:
            ops.append(Op(["rx", "ry", "rz"][c], (a,), param_index=int(rng.integers(0, npar))))
        elif c == 3:
            ops.append(Op("swap", (a, b)))
        elif c == 4:
            ops.append(Op("u2q", (a, b), matrix=W.haar_unitaries(1, 4, 100 * seed + i)[0]))
        elif c == 5:
            ops.append(Op("cnot", (a, b)))
        elif c == 6:
            ops.append(Op("cz", (a, b)))
        elif c == 7:
            ops.append(Op("cp", (a, b), (float(rng.uniform(0, 6.3)),)))
        else:
            ops.append(Op("h", (a,)))
    params = rng.uniform(0, 2 * np.pi, npar)
    terms = []
    for _ in range(5):
        s = ["I"] * n
        for q in rng.choice(n, int(rng.integers(1, 4)), replace=False):
            s[int(q)] = "XYZ"[int(rng.integers(0, 3))]
        terms.append("".join(s))
    coeffs = rng.uniform(-1, 1, len(terms))
    g = emulated_grad(n, ops, params, terms, coeffs, dtype)
    np.testing.assert_allclose(g, oracle.param_shift_grad(n, ops, params, terms, coeffs), atol=1e-12, rtol=0)
