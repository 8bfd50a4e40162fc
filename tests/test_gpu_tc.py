"""Tensor-core fused blocks (qc_apply_fused_k with QC_PREC_TF32X3, tcgen05 kind::tf32
with the three-product split) against the oracle's dense k-qubit block."""
import numpy as np
import pytest

import oracle
import workloads as W

from gpu_util import gpu_state, need_gpu, record, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def test_tc_identity_within_split_error():
    """With U = I the three products give a_hi + a_lo with a_lo truncated to TF32 by
    the tensor core: relative error per element below 2^-21."""
    import paper_2503_03016_gb300 as P
    n = 12
    psi = W.random_state(n, 1).astype(np.complex64)
    st = gpu_state(psi, "c64")
    P.qc_apply_fused_k(st.handle, [0, 3, 5, 7, 11], np.eye(32), P.QC_PREC_TF32X3)
    got = st.numpy()
    err = np.abs(got - psi) / np.maximum(np.abs(psi), 1e-30)
    assert err.max() < 2.0 ** -21, err.max()


@pytest.mark.parametrize("n,k", [(n, k) for n in (12, 14) for k in (2, 3, 4, 5)] + [(13, 6), (15, 6)])
def test_tc_block_vs_oracle(n, k):
    """k <= 5 run as 5-qubit blocks (padded with identity qubits); k = 6 through the
    six-qubit kernel (two K halves of A through one buffer)."""
    import paper_2503_03016_gb300 as P
    rng = np.random.default_rng(10 * n + k)
    for trial in range(3):
        qs = [int(x) for x in rng.permutation(n)[:k]]
        U = W.haar_unitaries(1, 1 << k, 100 * k + trial)[0]
        psi = W.random_state(n, trial)
        st = gpu_state(psi, "c64")
        P.qc_apply_fused_k(st.handle, qs, U, P.QC_PREC_TF32X3)
        want = psi.copy()
        oracle.apply_kq(want, qs, U)
        assert rel_l2(st.numpy(), want) <= 1e-5, (qs, rel_l2(st.numpy(), want))


def test_tc_six_qubit_identity_and_low_bits():
    """A six-qubit identity block returns the state within the split error, and a block
    on the six lowest index bits (whole rows contiguous) matches the oracle."""
    import paper_2503_03016_gb300 as P
    n = 14
    psi = W.random_state(n, 3).astype(np.complex64)
    st = gpu_state(psi, "c64")
    P.qc_apply_fused_k(st.handle, [1, 4, 6, 9, 12, 13], np.eye(64), P.QC_PREC_TF32X3)
    got = st.numpy()
    err = np.abs(got - psi) / np.maximum(np.abs(psi), 1e-30)
    assert err.max() < 2.0 ** -20, err.max()
    U = W.haar_unitaries(1, 64, 77)[0]
    qs = list(range(n - 6, n))
    psi = W.random_state(n, 4)
    st = gpu_state(psi, "c64")
    P.qc_apply_fused_k(st.handle, qs, U, P.QC_PREC_TF32X3)
    want = psi.copy()
    oracle.apply_kq(want, qs, U)
    assert rel_l2(st.numpy(), want) <= 1e-5


def test_tc_rejects_unsupported():
    import paper_2503_03016_gb300 as P
    st = gpu_state(W.random_state(12, 0), "c128")
    with pytest.raises(P.QCError):
        P.qc_apply_fused_k(st.handle, [0, 1], np.eye(4), P.QC_PREC_TF32X3)
    st = gpu_state(W.random_state(10, 0), "c64")
    with pytest.raises(P.QCError):
        P.qc_apply_fused_k(st.handle, [0, 1], np.eye(4), P.QC_PREC_TF32X3)
    st = gpu_state(W.random_state(12, 0), "c64")  # six-qubit blocks need n >= 13
    with pytest.raises(P.QCError):
        P.qc_apply_fused_k(st.handle, [0, 1, 2, 3, 4, 5], np.eye(64), P.QC_PREC_TF32X3)


@pytest.mark.parametrize("n,bits", [(20, (9, 10, 11, 12)), (20, (9, 10, 11, 12, 13)), (20, (2, 7, 12, 17)),
                                    (20, (1, 6, 11, 15, 18)), (22, (6, 9, 12, 15, 19))])
def test_tc_block_box_and_gather_layouts(n, bits):
    """Blocks on the given index bits, against the oracle: a tile (index bits 0..3, the
    block's bits, fillers) that is one box (bits 9..), one that is two boxes (the two
    spread layouts at 20 qubits: one tile bit is a box coordinate), and one with no box
    plan of at most two coordinate bits (22 qubits: the gathering block kernel)."""
    import paper_2503_03016_gb300 as P
    k = len(bits)
    qs = [n - 1 - b for b in bits]
    U = W.haar_unitaries(1, 1 << k, 40 + k + n)[0]
    psi = W.random_state(n, 5 + k)
    st = gpu_state(psi, "c64")
    P.qc_apply_fused_k(st.handle, qs, U, P.QC_PREC_TF32X3)
    want = psi.copy()
    oracle.apply_kq(want, qs, U)
    err = rel_l2(st.numpy(), want)
    record("tc_block_layout", n=n, bits=list(bits), rel_l2=err)
    assert err <= 1e-5, (bits, err)
