"""Degenerate inputs of the fused paths (tile passes on the CUDA cores and with
tensor-core stages) against the CPU oracle: the empty circuit, diagonal-only circuits,
single gates on the extreme qubits, and the smallest registers each path takes."""
import numpy as np
import pytest

import oracle
import workloads as W
from workloads import Op

from gpu_util import TOL, gpu_state, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def run(n, ops, dtype, prec, psi=None):
    import paper_2503_03016_gb300 as P
    psi = W.random_state(n, 11) if psi is None else psi
    st = gpu_state(psi, dtype)
    st.run(ops, mode=P.QC_RUN_FUSED, prec=P.QC_PREC_TF32X3 if prec == "tf32x3" else P.QC_PREC_NATIVE)
    return psi, st.numpy(), oracle.run(psi.copy(), ops)


@pytest.mark.parametrize("dtype,prec", [("c64", "native"), ("c128", "native"), ("c64", "tf32x3")])
def test_empty_circuit_leaves_the_state(dtype, prec):
    psi, got, _ = run(13, [], dtype, prec)
    want = psi.astype(np.complex64) if dtype == "c64" else psi
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_diagonal_only_circuit(dtype):
    """Phases only (RZ, S, T, CZ, CP, a diagonal 2-qubit gate): no dense target anywhere."""
    n = 14
    rng = np.random.default_rng(3)
    ops = []
    for i in range(40):
        a, b = (int(x) for x in rng.permutation(n)[:2])
        k = i % 6
        if k == 0:
            ops.append(Op("rz", (a,), (float(rng.uniform(0, 6.3)),)))
        elif k == 1:
            ops.append(Op("s", (a,)))
        elif k == 2:
            ops.append(Op("t", (a,)))
        elif k == 3:
            ops.append(Op("cz", (a, b)))
        elif k == 4:
            ops.append(Op("cp", (a, b), (float(rng.uniform(0, 6.3)),)))
        else:
            ops.append(Op("u2q", (a, b), matrix=np.diag(np.exp(1j * rng.uniform(0, 6.3, 4)))))
    _, got, want = run(n, ops, dtype, "native")
    assert rel_l2(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype,prec", [("c64", "native"), ("c128", "native"), ("c64", "tf32x3")])
@pytest.mark.parametrize("n", [12, 13])
def test_single_gates_on_the_extreme_qubits(dtype, prec, n):
    """One gate at a time on qubit 0 (the top index bit), on qubit n-1 (index bit 0),
    and on the pairs (0, n-1) and (n-2, n-1)."""
    U2 = W.haar_unitaries(2, 2, 4)
    U4 = W.haar_unitaries(2, 4, 5)
    for ops in ([Op("u1q", (0,), matrix=U2[0])], [Op("u1q", (n - 1,), matrix=U2[1])],
                [Op("u2q", (0, n - 1), matrix=U4[0])], [Op("u2q", (n - 2, n - 1), matrix=U4[1])]):
        _, got, want = run(n, ops, dtype, prec)
        assert rel_l2(got, want) <= TOL[dtype], ops[0].qubits


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_smallest_tile_register(dtype):
    """10 qubits, the smallest register the tile passes take (smaller ones run per gate)."""
    import paper_2503_03016_gb300 as P
    ops = W.brickwork(10, 10, 6)
    _, got, want = run(10, ops, dtype, "native")
    assert P.qc_last_fused_path() == 1
    assert rel_l2(got, want) <= TOL[dtype]
