"""GPU parity of the complex128 sweeps on states of 2^14 amplitudes or more, which run in
double-float arithmetic (FP32 pairs, 48-bit significands): every sweep kernel (dense,
diagonal, diagonal on the set half, anti-diagonal, two-qubit dense, with bit 0 among
the targets or the controls) against the oracle, a mixed per-gate circuit, and inputs
with zeros and with magnitudes outside the conversions' fast range.

Tolerance: relative L2 1e-13 for one gate (the double-float arithmetic keeps 48 bits;
its error per gate is a few units of 2^-48) and the complex128 target 1e-12 for
circuits."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import gates

from gpu_util import gpu_state, need_gpu, record, rel_l2

pytestmark = pytest.mark.gpu
GATE_TOL = 1e-13


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def rand_u(d, seed):
    return W.haar_unitaries(1, d, seed)[0]


@pytest.mark.parametrize("n", [14, 15])
def test_1q_every_kernel(n):
    import paper_2503_03016_gb300 as P
    mats = {"dense": rand_u(2, 3), "h": gates.H, "y": gates.Y, "z": gates.Z, "s": gates.S,
            "rz": gates.rz(0.7), "x": gates.X}
    worst = 0.0
    for q in (0, 1, n // 2, n - 2, n - 1):  # n - 1 is bit 0
        for name, U in mats.items():
            psi = W.random_state(n, 31 * q + len(name))
            st = gpu_state(psi, "c128")
            P.qc_apply_1q(st.handle, q, U)
            want = psi.copy()
            oracle.apply_1q(want, q, U)
            err = rel_l2(st.numpy(), want)
            worst = max(worst, err)
            assert err <= GATE_TOL, (q, name, err)
    record("c128_df_1q", n=n, worst_rel_l2=worst)


@pytest.mark.parametrize("n", [14, 16])
def test_controlled_with_bit0(n):
    """Controls on bit 0 (the sweeps without neighbour pairs) and targets on bit 0."""
    import paper_2503_03016_gb300 as P
    worst = 0.0
    cases = [([n - 1], [1], 3), ([n - 1], [0], 0), ([2, n - 1], [1, 0], 5), ([0], [1], n - 1),
             ([4, 7], [0, 1], n - 1), ([n - 3], [1], 1)]
    for ci, (ctrls, states, t) in enumerate(cases):
        for name, U in (("dense", rand_u(2, 40 + ci)), ("rz", gates.rz(1.1)), ("t", gates.T),
                        ("y", gates.Y)):
            psi = W.random_state(n, 500 + ci)
            st = gpu_state(psi, "c128")
            P.qc_apply_ctrl(st.handle, ctrls, states, t, U)
            want = psi.copy()
            oracle.apply_ctrl(want, ctrls, states, t, U)
            err = rel_l2(st.numpy(), want)
            worst = max(worst, err)
            assert err <= GATE_TOL, (ctrls, t, name, err)
    record("c128_df_ctrl", n=n, worst_rel_l2=worst)


@pytest.mark.parametrize("n", [14, 15])
def test_2q_pairs_including_bit0(n):
    import paper_2503_03016_gb300 as P
    worst = 0.0
    pairs = [(0, 1), (1, 0), (3, n - 1), (n - 1, 3), (n - 2, n - 1), (n - 1, 0), (5, 9)]
    for pi, (qa, qb) in enumerate(pairs):
        for U in (rand_u(4, 60 + pi), np.diag(np.exp(1j * np.arange(4) * 0.37))):
            psi = W.random_state(n, 700 + pi)
            st = gpu_state(psi, "c128")
            P.qc_apply_2q(st.handle, qa, qb, U)
            want = psi.copy()
            oracle.apply_2q(want, qa, qb, U)
            err = rel_l2(st.numpy(), want)
            worst = max(worst, err)
            assert err <= GATE_TOL, (qa, qb, err)
    record("c128_df_2q", n=n, worst_rel_l2=worst)


def test_per_gate_circuit_16q():
    """A 400-gate brickwork and a QFT, gate by gate: the complex128 target 1e-12."""
    import paper_2503_03016_gb300 as P
    n = 16
    psi = W.random_state(n, 9)
    ops = W.brickwork(n, 40, 5) + W.qft(n)
    st = gpu_state(psi, "c128")
    st.run(ops, mode=P.QC_RUN_PER_GATE)
    want = oracle.run(psi.copy(), ops)
    err = rel_l2(st.numpy(), want)
    record("c128_df_circuit", n=n, gates=len(ops), rel_l2=err)
    assert err <= 1e-12


def test_zeros_and_extreme_magnitudes():
    """Exact zeros stay zero; amplitudes far below 2^-126 (general conversions) and a
    basis state keep their values to the tolerance relative to the state's norm."""
    import paper_2503_03016_gb300 as P
    n = 14
    rng = np.random.default_rng(4)
    psi = W.random_state(n, 2)
    mags = 10.0 ** rng.uniform(-60, 0, psi.size)
    psi = psi / np.abs(psi) * mags
    psi[::7] = 0
    U = rand_u(2, 8)
    for q in (0, 6, n - 1):
        st = gpu_state(psi, "c128")
        P.qc_apply_1q(st.handle, q, U)
        want = psi.copy()
        oracle.apply_1q(want, q, U)
        got = st.numpy()
        assert rel_l2(got, want) <= GATE_TOL
        # zeros of both inputs of a pair give an exact zero
        both = (want == 0)
        assert np.all(got[both] == 0)
    e0 = oracle.basis_state(n, 5)
    st = gpu_state(e0, "c128")
    P.qc_apply_2q(st.handle, 3, n - 1, rand_u(4, 2))
    want = e0.copy()
    oracle.apply_2q(want, 3, n - 1, rand_u(4, 2))
    assert rel_l2(st.numpy(), want) <= GATE_TOL
    assert np.count_nonzero(st.numpy()) == np.count_nonzero(want)
