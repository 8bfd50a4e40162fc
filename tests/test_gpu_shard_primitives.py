"""The library entry points the sharded state builds on, on the GPU against the
oracle: <a|b> (qc_inner) and collapse with a caller-supplied normaliser
(qc_collapse_norm); and the sharded state's GPU engine in a one-process group (every
qubit local, the library doing every gate and readout)."""
import numpy as np
import pytest

import oracle
import workloads as W

from gpu_util import TOL, gpu_state, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 7, 20])
def test_inner_product(dtype, n):
    import paper_2503_03016_gb300 as P
    a, b = W.random_state(n, 1), W.random_state(n, 2)
    sa, sb = gpu_state(a, dtype), gpu_state(b, dtype)
    got = P.qc_inner(sa.handle, sb.handle)
    if dtype == "c64":
        a, b = a.astype(np.complex64).astype(np.complex128), b.astype(np.complex64).astype(np.complex128)
    want = oracle.inner(a, b)
    assert abs(got - want) <= (1e-14 if dtype == "c128" else 1e-6), (got, want)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_collapse_with_given_normaliser(dtype):
    import paper_2503_03016_gb300 as P
    n = 12
    psi = W.random_state(n, 3)
    for q, o, p in ((0, 1, 0.3), (n - 1, 0, 0.7), (5, 1, 0.0), (-1, 0, 0.25)):
        st = gpu_state(psi, dtype)
        P.qc_collapse_norm(st.handle, q, o, p)
        want = psi.copy()
        if q >= 0:
            oracle.collapse(want, q, o, p if p > 0 else 1.0)
        if p == 0:
            want[:] = 0
        elif q < 0:
            want = want / np.sqrt(p)
        got = st.numpy()
        if p == 0:
            assert not np.any(got)
        else:
            assert rel_l2(got, want) <= TOL[dtype] * 10 if dtype == "c64" else rel_l2(got, want) <= 1e-15


def test_sharded_engine_single_process():
    """A one-process group (no global qubits): the GPU engine runs the gates, the
    expectations, outcome probabilities and collapse of the sharded state."""
    import os

    import torch.distributed as dist

    from paper_2503_03016_gb300.sharded import CudaShard, ShardedState
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", "29533")
    own = not dist.is_initialized()
    if own:
        dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        n = 14
        ops = W.brickwork(n, 6, 2) + W.qft(n)
        st = ShardedState(n, CudaShard(n, "c128"))
        st.init_basis(3).run(ops)
        assert st.at != list(range(n))  # the QFT's final swaps only relabelled qubits
        want = oracle.run(oracle.basis_state(n, 3), ops)
        st.normalize()  # identity placement: the shard is then the state vector
        assert rel_l2(st.eng.download(), want) <= 1e-12
        strings = ["XYZ" + "I" * (n - 3), "Z" * n]
        np.testing.assert_allclose(st.expect(strings), oracle.expect_pauli(want, strings), atol=1e-12)
        p = st.collapse(2, 1)
        assert abs(p - oracle.outcome_prob(want, 2, 1)) < 1e-13
        oracle.collapse(want, 2, 1, oracle.outcome_prob(want, 2, 1))
        st.normalize()
        assert rel_l2(st.eng.download(), want) <= 1e-12
    finally:
        if own:
            dist.destroy_process_group()
