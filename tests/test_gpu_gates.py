"""GPU parity: per-gate sweeps, fused blocks and circuits against the CPU oracle
(through the C ABI).  Tolerance: relative L2 1e-12 for complex128, 1e-5 for complex64."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import gates, kron
from workloads import Op

from gpu_util import TOL, gpu_state, need_gpu, record, rel_l2

pytestmark = pytest.mark.gpu
DTYPES = ["c128", "c64"]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def rand_u(d, seed):
    return W.haar_unitaries(1, d, seed)[0]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 3, 6, 11])
def test_1q_all_positions_and_structures(dtype, n):
    import paper_2503_03016_gb300 as P
    mats = [rand_u(2, 1), gates.H, gates.X, gates.Y, gates.Z, gates.S, gates.rz(0.7), gates.T]
    for q in range(n):
        for mi, U in enumerate(mats):
            psi = W.random_state(n, 17 * q + mi)
            st = gpu_state(psi, dtype)
            P.qc_apply_1q(st.handle, q, U)
            want = psi.copy()
            oracle.apply_1q(want, q, U)
            assert rel_l2(st.numpy(), want) <= TOL[dtype], (q, mi)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_2q_all_ordered_pairs(dtype, n):
    import paper_2503_03016_gb300 as P
    for qa in range(n):
        for qb in range(n):
            if qa == qb:
                continue
            for U in (rand_u(4, 7 * qa + qb), gates.SWAP, np.diag([1, 1, 1, np.exp(0.3j)])):
                psi = W.random_state(n, 100 + qa * n + qb)
                st = gpu_state(psi, dtype)
                P.qc_apply_2q(st.handle, qa, qb, U)
                want = psi.copy()
                oracle.apply_2q(want, qa, qb, U)
                assert rel_l2(st.numpy(), want) <= TOL[dtype], (qa, qb)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("nctrl", [1, 2, 3])
def test_controlled_every_state(dtype, nctrl):
    import paper_2503_03016_gb300 as P
    n = 7
    rng = np.random.default_rng(nctrl)
    for trial in range(12):
        qs = [int(x) for x in rng.permutation(n)[: nctrl + 1]]
        ctrls, tgt = qs[:-1], qs[-1]
        states = [int(x) for x in rng.integers(0, 2, nctrl)]
        U = [rand_u(2, trial), gates.X, gates.Z, gates.phase(1.1)][trial % 4]
        psi = W.random_state(n, trial)
        st = gpu_state(psi, dtype)
        P.qc_apply_ctrl(st.handle, ctrls, states, tgt, U)
        want = psi.copy()
        oracle.apply_ctrl(want, ctrls, states, tgt, U)
        assert rel_l2(st.numpy(), want) <= TOL[dtype], (ctrls, states, tgt)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_fused_native_block(dtype, k):
    import paper_2503_03016_gb300 as P
    n = 10
    rng = np.random.default_rng(k)
    for trial in range(3):
        qs = [int(x) for x in rng.permutation(n)[:k]]
        U = rand_u(1 << k, 40 + trial)
        psi = W.random_state(n, trial)
        st = gpu_state(psi, dtype)
        P.qc_apply_fused_k(st.handle, qs, U, P.QC_PREC_NATIVE)
        want = psi.copy()
        oracle.apply_kq(want, qs, U)
        assert rel_l2(st.numpy(), want) <= TOL[dtype], qs


@pytest.mark.parametrize("dtype", DTYPES)
def test_u3_ladder_10q(dtype):
    """The 10-qubit workload: 20 layers of U3 on every qubit plus a CNOT ladder, from
    |0...0>, against the loop oracle and the dense Kronecker form."""
    import paper_2503_03016_gb300 as P
    n = 10
    ops = W.u3_ladder(n, 20, 1)
    st = P.State(n, dtype).init_basis(0)
    st.run(ops, mode=P.QC_RUN_PER_GATE)
    want = oracle.run(oracle.basis_state(n, 0), ops)
    got = st.numpy()
    assert rel_l2(got, want) <= TOL[dtype]
    want_k = kron.apply(oracle.basis_state(n, 0), n, ops)
    assert rel_l2(got, want_k) <= TOL[dtype]
    p = st.probs().cpu().numpy()
    if dtype == "c128":
        np.testing.assert_array_equal(p, oracle.probs(got.astype(np.complex128)))
    assert abs(p.sum() - 1) < (1e-12 if dtype == "c128" else 1e-5)


@pytest.mark.parametrize("dtype", DTYPES)
def test_circuits_and_inverse(dtype):
    import paper_2503_03016_gb300 as P
    n = 9
    ops = W.brickwork(n, 6, 3) + W.qft(n) + W.ansatz(n, 2, True) + [
        Op("mcx", (0, 3, 5), ctrl_states=(1, 0)), Op("swap", (1, 7)), Op("cp", (8, 2), (0.4,)),
        Op("u1q", (4,), matrix=rand_u(2, 3)), Op("t", (6,)), Op("sdg", (2,)), Op("rx", (1,), (0.9,))]
    params = W.ansatz_params(n, 2, 3)
    psi = W.random_state(n, 5)
    st = gpu_state(psi, dtype)
    st.run(ops, params)
    want = oracle.run(psi.copy(), ops, params)
    err = rel_l2(st.numpy(), want)
    st.run(W.circuit_inverse(ops), params)
    err_inv = rel_l2(st.numpy(), psi)
    record("per_gate_circuits_and_inverse", n=n, dtype=dtype, rel_l2=err, rel_l2_inverse=err_inv)
    assert err <= TOL[dtype]
    assert err_inv <= TOL[dtype]


def test_gaussian_init_matches_generator():
    """complex128: the FP64 construction to rounding; complex64: the transform in FP32,
    within a few FP32 roundings (the bound 1e-6 is 17x FP32 epsilon, 10x under the
    complex64 target)."""
    import paper_2503_03016_gb300 as P
    for n in (1, 5, 12, 16):
        st = P.State(n, "c128").init_gaussian(3)
        assert rel_l2(st.numpy(), W.gaussian_state(n, 3)) <= 1e-14
        st64 = P.State(n, "c64").init_gaussian(3)
        assert rel_l2(st64.numpy(), W.gaussian_state(n, 3)) <= 1e-6


def test_argument_errors():
    import paper_2503_03016_gb300 as P
    st = P.State(4, "c64").init_basis(0)
    with pytest.raises(P.QCError):
        P.qc_apply_1q(st.handle, 4, gates.H)
    with pytest.raises(P.QCError):
        P.qc_apply_2q(st.handle, 1, 1, gates.SWAP)
    with pytest.raises(P.QCError):
        P.qc_apply_ctrl(st.handle, [0], [2], 1, gates.X)
    with pytest.raises(P.QCError):
        P.qc_state_init_basis(st.handle, 16)
    with pytest.raises(P.QCError):
        st.run([Op("h", (5,))])
    # the state is untouched by rejected calls
    np.testing.assert_array_equal(st.numpy(), oracle.basis_state(4, 0).astype(np.complex64))
