"""GPU parity of the fused execution (QC_RUN_FUSED: shared-memory tile passes with
merged diagonal gates) against the CPU oracle, plus full-size properties."""
import numpy as np
import pytest

import oracle
import workloads as W
from workloads import Op

from gpu_util import TOL, gpu_state, need_gpu, record, rel_l2

pytestmark = pytest.mark.gpu
DTYPES = ["c128", "c64"]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def mixed_circuit(n, seed):
    """Every gate kind, controls inside and outside any tile, open controls,
    diagonal and non-diagonal two-qubit matrices."""
    rng = np.random.default_rng(seed)
    ops = []
    kinds1 = ["h", "x", "y", "z", "s", "sdg", "t", "tdg"]
    for i in range(160):
        c = rng.integers(0, 10)
        qs = [int(x) for x in rng.permutation(n)[:4]]
        if c == 0:
            ops.append(Op(kinds1[rng.integers(0, len(kinds1))], (qs[0],)))
        elif c == 1:
            ops.append(Op(["rx", "ry", "rz"][rng.integers(0, 3)], (qs[0],), (float(rng.uniform(0, 6.3)),)))
        elif c == 2:
            ops.append(Op("u3", (qs[0],), tuple(float(a) for a in rng.uniform(0, 6.3, 3))))
        elif c == 3:
            ops.append(Op("cnot", (qs[0], qs[1])))
        elif c == 4:
            ops.append(Op("cz", (qs[0], qs[1])))
        elif c == 5:
            ops.append(Op("cp", (qs[0], qs[1]), (float(rng.uniform(0, 6.3)),)))
        elif c == 6:
            ops.append(Op("swap", (qs[0], qs[1])))
        elif c == 7:
            ops.append(Op("u2q", (qs[0], qs[1]), matrix=W.haar_unitaries(1, 4, seed * 1000 + i)[0]))
        elif c == 8:
            ops.append(Op("mcx", (qs[0], qs[1], qs[2]), ctrl_states=(int(rng.integers(0, 2)), int(rng.integers(0, 2)))))
        else:
            ph = np.exp(1j * rng.uniform(0, 6.3, 4))
            ops.append(Op("u2q", (qs[0], qs[1]), matrix=np.diag(ph)))
    return ops


def run_both(n, ops, dtype, psi=None, params=None):
    import paper_2503_03016_gb300 as P
    psi = W.random_state(n, n) if psi is None else psi
    st = gpu_state(psi, dtype)
    st.run(ops, params, mode=P.QC_RUN_FUSED)
    passes = P.qc_last_pass_count()
    want = oracle.run(psi.copy(), ops, params)
    return st.numpy(), want, passes


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [10, 13, 16])
def test_fused_brickwork(dtype, n):
    ops = W.brickwork(n, 12, 7)
    got, want, passes = run_both(n, ops, dtype)
    assert rel_l2(got, want) <= TOL[dtype]
    assert passes < len(ops)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [10, 14, 17])
def test_fused_qft(dtype, n):
    ops = W.qft(n)
    x = W.gaussian_state(n, 3)
    got, want, passes = run_both(n, ops, dtype, psi=x)
    assert rel_l2(got, want) <= TOL[dtype]
    assert rel_l2(got, np.sqrt(2.0 ** n) * np.fft.ifft(x)) <= TOL[dtype]
    assert passes <= 8, passes


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [11, 15])
def test_fused_mixed(dtype, n):
    ops = mixed_circuit(n, n)
    got, want, _ = run_both(n, ops, dtype)
    err = rel_l2(got, want)
    record("fused_mixed", n=n, dtype=dtype, rel_l2=err)
    assert err <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_fused_ansatz_and_ladder(dtype):
    n = 12
    ops = W.ansatz(n, 3, ring=True) + W.u3_ladder(n, 3, 4)
    params = W.ansatz_params(n, 3, 9)
    got, want, _ = run_both(n, ops, dtype, params=params)
    assert rel_l2(got, want) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [12, 17])
def test_fused_cz_runs(dtype, n):
    """Runs of CZ gates (merged into sign ops) between dense layers: pairs between any
    two bit positions (register slots, lane bits, bits fixed by the tile number), the
    same pair twice, and interleaved gates that must not join a run (a CZ with an open
    control, a controlled phase other than pi, a diagonal two-qubit gate with the CZ's
    phases but a global phase)."""
    rng = np.random.default_rng(n)
    U = W.haar_unitaries(8, 4, 31)
    ops = []
    for layer in range(4):
        for q in range(0, n - 1, 2):
            ops.append(Op("u2q", (q, q + 1), matrix=U[(layer + q) % 8]))
        for _ in range(3 * n):
            a, b = (int(x) for x in rng.permutation(n)[:2])
            ops.append(Op("cz", (a, b)))
        ops.append(Op("cz", (ops[-1].qubits[0], ops[-1].qubits[1])))  # the same pair again
        a, b = (int(x) for x in rng.permutation(n)[:2])
        ops.append(Op("ctrl", (a, b), matrix=np.diag([1.0, -1.0]), ctrl_states=(0,)))
        ops.append(Op("cz", (b, a)))
        ops.append(Op("cp", (a, b), (3.0,)))
        ops.append(Op("u2q", (b, a), matrix=np.diag([1j, 1j, 1j, -1j])))
        ops.append(Op("cz", (a, (a + 1) % n)))
    got, want, _ = run_both(n, ops, dtype)
    err = rel_l2(got, want)
    record("fused_cz_runs", n=n, dtype=dtype, rel_l2=err)
    assert err <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [12, 15])
def test_fused_swaps_relabeled(dtype, n):
    """Exact SWAPs inside a tile move no data: the pass's later ops are renamed and the
    write-out reads the tile through the permutation.  Chains of swaps over low and
    high bits, the same pair twice, swaps followed by dense gates, controls and phases
    on the swapped qubits, and a circuit of swaps alone."""
    rng = np.random.default_rng(100 + n)
    U = W.haar_unitaries(16, 4, 5)
    ops = []
    for layer in range(6):
        for _ in range(6):
            a, b = (int(x) for x in rng.permutation(n)[:2])
            ops.append(Op("swap", (a, b)))
        ops += [Op("swap", (n - 1, n - 2)), Op("swap", (n - 1, 0)), Op("swap", (n - 1, 0))]
        a, b, c = (int(x) for x in rng.permutation(n)[:3])
        ops += [Op("u2q", (a, b), matrix=U[layer]), Op("cnot", (c, a)), Op("cp", (b, c), (0.7,)),
                Op("u3", (a,), (0.3, 1.2, 2.1)), Op("mcx", (a, b, c), ctrl_states=(1, 0)),
                Op("swap", (a, c)), Op("rz", (a,), (0.9,)), Op("cz", (c, b)), Op("h", (c,))]
    got, want, _ = run_both(n, ops, dtype)
    assert rel_l2(got, want) <= TOL[dtype]
    only = [Op("swap", (int(a), int(b))) for a, b in (rng.permutation(n)[:2] for _ in range(40))]
    got, want, _ = run_both(n, only, dtype)
    assert rel_l2(got, want) <= TOL[dtype]


def test_fused_small_n_uses_per_gate():
    ops = W.brickwork(6, 4, 1)
    got, want, _ = run_both(6, ops, "c128")
    assert rel_l2(got, want) <= 1e-12


@pytest.mark.slow
def test_fused_brickwork_28_inverse_property():
    """Full size, the benchmark's configuration: the 540-gate 28-qubit brickwork
    followed by its inverse returns |0...0> (complex64), and the fused result
    agrees with the per-gate sweeps."""
    import torch

    import paper_2503_03016_gb300 as P
    n = 28
    ops = W.brickwork(n, 40, 2)
    circ = P.Circuit(n, ops)
    inv = P.Circuit(n, W.circuit_inverse(ops))
    a = P.State(n, "c64").init_basis(0)
    P.qc_run_circuit(a.handle, circ, None, P.QC_RUN_FUSED)
    b = P.State(n, "c64").init_basis(0)
    P.qc_run_circuit(b.handle, circ, None, P.QC_RUN_PER_GATE)
    diff = torch.linalg.vector_norm(a.tensor - b.tensor).item()
    assert diff <= 1e-5, diff
    p = a.probs()
    assert abs(p.sum().item() - 1) < 1e-5
    P.qc_run_circuit(a.handle, inv, None, P.QC_RUN_FUSED)
    amp0 = a.tensor[0].item()
    assert abs(amp0 - 1) < 1e-5, amp0
    assert abs(torch.linalg.vector_norm(a.tensor).item() - 1) < 1e-5
