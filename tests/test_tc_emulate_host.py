"""Host-only check of the tensor-core passes' plan logic (qc_tc_emulate; no GPU needed):
the planner's passes, stage blocks (their FP64 products), deferred phase factors (the
FP32 tables the kernel reads), SWAP relabelings and copy passes applied on the host in
the kernel's order, against the oracle.

Circuits whose deferred factors are all +-1 (CZ rings) or that have none come out at
FP64 rounding; circuits with deferred phases carry the tables' FP32 rounding (a few
units of 1e-8 per factor).  A planning mistake -- a factor moved past an op it does not
commute with, a wrong slot or row bit, a misread relabeling -- gives errors of order 1."""
import numpy as np
import pytest

import oracle
import workloads as W
from workloads import Op


def emulate(n, ops, psi, params=None):
    import paper_2503_03016_gb300 as P
    got = P.qc_tc_emulate(P.Circuit(n, ops), psi, params)
    want = oracle.run(psi.copy(), ops, params)
    return np.linalg.norm(got - want) / np.linalg.norm(want)


@pytest.mark.parametrize("n", [13, 14, 16, 17])
def test_qft_with_deferred_ladders(n):
    """(16 and 17 qubits: one and two passes that are only the final swaps' relabeling)"""
    import paper_2503_03016_gb300 as P
    if n >= 16:
        assert P.qc_tc_plan_info(P.Circuit(n, W.qft(n)))[3] == n - 15
    assert emulate(n, W.qft(n), W.gaussian_state(n, 3)) <= 1e-6


def test_inverse_qft_with_far_and_open_control_phases():
    n = 16
    ops = W.circuit_inverse(W.qft(n))
    rng = np.random.default_rng(8)
    for i in range(48):
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        ph = float(rng.uniform(0, 6.3))
        if i % 4 == 0:
            ops.append(Op("cp", (a, b), (ph,)))
        elif i % 4 == 1:
            ops.append(Op("ctrl", (a, b), matrix=np.diag([1.0, np.exp(1j * ph)]), ctrl_states=(0,)))
        elif i % 4 == 2:
            ops.append(Op("ctrl", (a, b), matrix=np.diag([np.exp(-0.5j * ph), np.exp(0.5j * ph)]),
                          ctrl_states=(0,)))
        else:
            ops += [Op("h", (a,)), Op("t", (b,))]
    assert emulate(n, ops, W.gaussian_state(n, 5)) <= 1e-6


@pytest.mark.parametrize("n", [13, 15])
def test_brickwork_and_ansatz_ring_exact(n):
    assert emulate(n, W.brickwork(n, 12, 7), W.random_state(n, 1)) <= 1e-12
    layers = 4
    params = np.random.default_rng(n).uniform(0, 2 * np.pi, layers * 2 * n)
    assert emulate(n, W.ansatz(n, layers, True), W.random_state(n, 2), params) <= 1e-12


def test_swaps_relabelings_and_copy_passes():
    n = 15
    rng = np.random.default_rng(n)
    U = W.haar_unitaries(60, 4, 3 * n)
    ops = []
    for i in range(60):
        a = int(rng.integers(0, n - 1))
        ops.append(Op("u2q", (a, a + 1), matrix=U[i]))
        if i % 4 == 3:
            b, c = (int(v) for v in rng.choice(n, 2, replace=False))
            ops.append(Op("swap", (b, c)))
    ops += [Op("swap", (j, n - 1 - j)) for j in range(n // 2)]  # a bit reversal at the end
    assert emulate(n, ops, W.random_state(n, 3)) <= 1e-12


def test_rejects_circuits_outside_the_stages_and_small_registers():
    import paper_2503_03016_gb300 as P
    n = 16
    ops = [Op("h", (q,)) for q in range(n)]
    ops.append(Op("ctrl", (0, n - 1, n // 2), matrix=np.diag([1.0, np.exp(0.7j)])))
    psi = W.random_state(n, 4)
    try:
        err = emulate(n, ops, psi)
        assert err <= 1e-6  # planned onto the stages after all: still exact
    except P.QCError as e:
        assert e.status == 4
    with pytest.raises(P.QCError):
        P.qc_tc_emulate(P.Circuit(10, W.qft(10)), W.random_state(10, 1))


def _mixed(n, seed, count=120):
    """Every gate kind: 1-qubit gates and rotations, CNOT, CZ, CP, SWAP, Haar and
    diagonal two-qubit matrices, multi-controlled X and controlled 2x2 gates with open
    and closed controls, on random qubits."""
    rng = np.random.default_rng(seed)
    ops = []
    kinds1 = ["h", "x", "y", "z", "s", "sdg", "t", "tdg"]
    for i in range(count):
        c = int(rng.integers(0, 11))
        qs = [int(x) for x in rng.permutation(n)[:4]]
        ang = float(rng.uniform(0, 6.3))
        if c == 0:
            ops.append(Op(kinds1[int(rng.integers(0, len(kinds1)))], (qs[0],)))
        elif c == 1:
            ops.append(Op(["rx", "ry", "rz"][int(rng.integers(0, 3))], (qs[0],), (ang,)))
        elif c == 2:
            ops.append(Op("u3", (qs[0],), tuple(float(a) for a in rng.uniform(0, 6.3, 3))))
        elif c == 3:
            ops.append(Op("cnot", (qs[0], qs[1])))
        elif c == 4:
            ops.append(Op("cz", (qs[0], qs[1])))
        elif c == 5:
            ops.append(Op("cp", (qs[0], qs[1]), (ang,)))
        elif c == 6:
            ops.append(Op("swap", (qs[0], qs[1])))
        elif c == 7:
            ops.append(Op("u2q", (qs[0], qs[1]), matrix=W.haar_unitaries(1, 4, seed * 1000 + i)[0]))
        elif c == 8:
            ops.append(Op("mcx", (qs[0], qs[1], qs[2]), ctrl_states=(int(rng.integers(0, 2)), int(rng.integers(0, 2)))))
        elif c == 9:
            ops.append(Op("ctrl", (qs[0], qs[1]), matrix=np.diag(np.exp(1j * rng.uniform(0, 6.3, 2))),
                          ctrl_states=(int(rng.integers(0, 2)),)))
        else:
            ops.append(Op("u2q", (qs[0], qs[1]), matrix=np.diag(np.exp(1j * rng.uniform(0, 6.3, 4)))))
    return ops


def test_random_mixed_circuits():
    """Seeded circuits of every gate kind on 12 to 15 qubits: where the tensor-core
    planner takes the circuit, its plan applied on the host equals the oracle (FP32
    phase tables: 1e-6); most of them fit the stages."""
    import paper_2503_03016_gb300 as P
    fit = 0
    cases = [(n, seed) for n in (12, 13, 15) for seed in range(1, 7)]
    for n, seed in cases:
        ops = _mixed(n, seed)
        try:
            err = emulate(n, ops, W.random_state(n, seed))
        except P.QCError as e:
            assert e.status == 4
            continue
        fit += 1
        assert err <= 1e-6, (n, seed, err)
    assert fit >= len(cases) // 2, fit


def test_plan_statistics_pinned():
    """The tensor-core plans behind the benchmark numbers (stage cuts searched two
    stages ahead): the 28-qubit brickwork in 30 passes of 102 stage blocks (no deferred
    factor), the 32-qubit QFT in 8 passes of 9 stage blocks with 30 deferred factors and 3
    relabeling-only passes, the 24-qubit ansatz of the gradient benchmark in 8 passes of
    38 stage blocks."""
    import paper_2503_03016_gb300 as P
    assert P.qc_tc_plan_info(P.Circuit(28, W.brickwork(28, 40, 2))) == (30, 102, 0, 0)
    assert P.qc_tc_plan_info(P.Circuit(32, W.qft(32))) == (8, 9, 30, 3)
    ops, params, _, _ = W.adjoint_workload(24, 10, 5)
    assert P.qc_tc_plan_info(P.Circuit(24, ops), params)[:2] == (8, 38)


def test_replanning_with_new_values_reuses_the_structure():
    """The same circuit with other rotation angles (a training loop) re-plans with the
    variants kept from the first plan (the same passes and stages for generic angles);
    the plan stays exact for every set of values, including angles that make rotations
    diagonal or the identity (a new structure: its own search)."""
    import paper_2503_03016_gb300 as P
    n, layers = 15, 4
    ops = W.ansatz(n, layers, True)
    psi = W.random_state(n, 6)
    rng = np.random.default_rng(11)
    info = None
    for trial in range(4):
        params = rng.uniform(0, 2 * np.pi, layers * 2 * n)
        if trial == 3:
            params[::3] = 0.0  # identity rotations
            params[1::3] = np.pi
        got = P.qc_tc_plan_info(P.Circuit(n, ops), params)
        info = got if info is None else info
        if trial < 3:
            assert got[:2] == info[:2]
        assert emulate(n, ops, psi, params) <= 1e-12, trial


def test_plans_do_not_carry_over_between_circuits():
    """The host plan's vectors are reused from one plan to the next on a thread: a plan
    made after a larger one (more passes, stage images and factor tables) and after a
    smaller one is the same plan, and the circuit still emulates exactly."""
    import paper_2503_03016_gb300 as P
    n = 16
    small = P.Circuit(13, W.brickwork(13, 6, 3))
    large = P.Circuit(18, W.qft(18))
    ops = W.circuit_inverse(W.qft(n))
    first = P.qc_tc_plan_info(P.Circuit(n, ops))
    for other in (large, small, large):
        P.qc_tc_plan_info(other)
        assert P.qc_tc_plan_info(P.Circuit(n, ops)) == first
    assert emulate(n, ops, W.gaussian_state(n, 9)) <= 1e-6


# gate-kind weights of _weighted: 1q fixed, rotation, U3, CNOT, CZ, CP, SWAP, Haar 2q on
# random qubits, MCX, controlled diagonal, diagonal 2q, controlled Haar 2x2, Haar 2q on
# neighbours
MIXES = {
    "phase_heavy": [1, 2, 0.5, 0.5, 3, 3, 0.5, 0.3, 0.2, 2, 2, 0.3, 0.5],
    "swap_heavy": [1, 1, 0.5, 1, 1, 1, 4, 1, 0.3, 0.5, 0.5, 0.5, 1],
    "dense": [1, 1, 1, 1, 0.2, 0.2, 0.2, 3, 0.3, 0.2, 0.2, 1, 3],
}


def _weighted(n, seed, count, weights):
    rng = np.random.default_rng(seed)
    w = np.asarray(weights, float) / np.sum(weights)
    kinds1 = ["h", "x", "y", "z", "s", "sdg", "t", "tdg"]
    ops = []
    for i in range(count):
        c = int(rng.choice(len(w), p=w))
        q = [int(x) for x in rng.permutation(n)[:3]]
        ang = float(rng.uniform(0, 6.3))
        if c == 0:
            ops.append(Op(kinds1[int(rng.integers(0, 8))], (q[0],)))
        elif c == 1:
            ops.append(Op(["rx", "ry", "rz"][int(rng.integers(0, 3))], (q[0],), (ang,)))
        elif c == 2:
            ops.append(Op("u3", (q[0],), tuple(float(a) for a in rng.uniform(0, 6.3, 3))))
        elif c in (3, 4, 6):
            ops.append(Op({3: "cnot", 4: "cz", 6: "swap"}[c], (q[0], q[1])))
        elif c == 5:
            ops.append(Op("cp", (q[0], q[1]), (ang,)))
        elif c == 7:
            ops.append(Op("u2q", (q[0], q[1]), matrix=W.haar_unitaries(1, 4, 1000 * seed + i)[0]))
        elif c == 8:
            ops.append(Op("mcx", tuple(q), ctrl_states=tuple(int(v) for v in rng.integers(0, 2, 2))))
        elif c == 9:
            ops.append(Op("ctrl", (q[0], q[1]), matrix=np.diag(np.exp(1j * rng.uniform(0, 6.3, 2))),
                          ctrl_states=(int(rng.integers(0, 2)),)))
        elif c == 10:
            ops.append(Op("u2q", (q[0], q[1]), matrix=np.diag(np.exp(1j * rng.uniform(0, 6.3, 4)))))
        elif c == 11:
            ops.append(Op("ctrl", (q[0], q[1]), matrix=W.haar_unitaries(1, 2, 7 * seed + i)[0],
                          ctrl_states=(int(rng.integers(0, 2)),)))
        else:
            a = int(rng.integers(0, n - 1))
            ops.append(Op("u2q", (a, a + 1), matrix=W.haar_unitaries(1, 4, 3 * seed + i)[0]))
    return ops


@pytest.mark.parametrize("mix", sorted(MIXES))
def test_weighted_random_circuits(mix):
    """Seeded circuits of 20-200 gates, weighted towards phases (deferred factors),
    SWAPs (relabelings) or dense gates, on 12 to 18 qubits; the planner's caches of
    stage cuts and variants are shared across them, as in one process of the library."""
    import paper_2503_03016_gb300 as P
    for n in (12, 14, 16, 18):
        for seed in range(2):
            count = int(np.random.default_rng(seed + 99).integers(20, 200))
            ops = _weighted(n, 1000 * n + seed, count, MIXES[mix])
            try:
                err = emulate(n, ops, W.random_state(n, seed + 5))
            except P.QCError as e:
                assert e.status == 4
                continue
            assert err <= 1e-6, (n, seed, err)
