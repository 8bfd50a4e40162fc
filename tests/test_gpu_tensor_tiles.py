"""GPU parity of the tile passes whose stages run on the tensor cores (QC_RUN_FUSED
with QC_PREC_TF32X3, complex64): each stage's gates multiplied into one 32 x 32 block
and applied as a TF32x3 GEMM, against the CPU oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from workloads import Op

from gpu_util import TOL, gpu_state, need_gpu, record, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def run_tc(n, ops, psi=None, params=None):
    import paper_2503_03016_gb300 as P
    psi = W.random_state(n, n) if psi is None else psi
    st = gpu_state(psi, "c64")
    st.run(ops, params, mode=P.QC_RUN_FUSED, prec=P.QC_PREC_TF32X3)
    path = P.qc_last_fused_path()
    want = oracle.run(psi.copy(), ops, params)
    return st.numpy(), want, path


@pytest.mark.parametrize("n,depth", [(12, 8), (13, 12), (16, 12), (18, 40)])
def test_tc_brickwork(n, depth):
    ops = W.brickwork(n, depth, 7)
    got, want, path = run_tc(n, ops)
    assert path == 2
    assert rel_l2(got, want) <= TOL["c64"]


@pytest.mark.parametrize("n", [13, 15])
def test_tc_single_and_two_stage_passes(n):
    """Gates confined to the five lowest qubits (one stage per pass: the stage's block
    stays resident) and to two groups of five (two stages per pass)."""
    U = W.haar_unitaries(64, 4, n)
    lo = list(range(n - 5, n))
    ops = [Op("u2q", (lo[i % 4], lo[i % 4 + 1]), matrix=U[i]) for i in range(30)]
    got, want, path = run_tc(n, ops)
    assert path == 2
    assert rel_l2(got, want) <= TOL["c64"]
    hi = list(range(0, 5))
    ops = []
    for i in range(40):
        grp = lo if i % 2 else hi
        ops.append(Op("u2q", (grp[(i // 2) % 4], grp[(i // 2) % 4 + 1]), matrix=U[i % 64]))
    got, want, path = run_tc(n, ops)
    assert path == 2
    assert rel_l2(got, want) <= TOL["c64"]


def test_tc_whole_state_tile_takes_every_control():
    """With the whole state in one tile (12 qubits) every control is a tile bit: the
    QFT's ladders fold into stage blocks and run on the tensor cores."""
    n = 12
    ops = W.qft(n)
    x = W.gaussian_state(n, 4)
    got, want, path = run_tc(n, ops, psi=x)
    assert path == 2
    assert rel_l2(got, want) <= TOL["c64"]


def test_tc_one_qubit_controlled_and_diagonal_ops():
    """U3, RX/RY/RZ, H, S, T, CNOT and CZ between neighbours, open controls, a
    controlled phase and a diagonal two-qubit gate, all folded into stage blocks."""
    n = 14
    rng = np.random.default_rng(5)
    ops = []
    for layer in range(6):
        for q in range(n):
            ops.append(Op("u3", (q,), tuple(float(a) for a in rng.uniform(0, 6.3, 3))))
        for q in range(layer % 2, n - 1, 2):
            c = (q + layer) % 5
            if c == 0:
                ops.append(Op("cnot", (q, q + 1)))
            elif c == 1:
                ops.append(Op("cz", (q, q + 1)))
            elif c == 2:
                ops.append(Op("cp", (q + 1, q), (float(rng.uniform(0, 6.3)),)))
            elif c == 3:
                ops.append(Op("ctrl", (q, q + 1), matrix=W.haar_unitaries(1, 2, layer * 100 + q)[0], ctrl_states=(0,)))
            else:
                ops.append(Op("u2q", (q, q + 1), matrix=np.diag(np.exp(1j * rng.uniform(0, 6.3, 4)))))
        ops += [Op("h", (layer,)), Op("s", (layer + 1,)), Op("t", (layer + 2,)),
                Op("rx", (layer + 3,), (0.3,)), Op("ry", (layer + 4,), (1.1,)), Op("rz", (layer + 5,), (2.2,))]
    got, want, path = run_tc(n, ops)
    assert path in (1, 2)
    assert rel_l2(got, want) <= TOL["c64"]


@pytest.mark.parametrize("n", [14, 16, 20])
def test_tc_qft_defers_phase_bits(n):
    """QFT on more qubits than a tile holds: the controlled-phase ladders reach row bits
    and bits outside the tile.  Each ladder is keyed on its target (a stage slot); the
    part of its phases on the other bits commutes with the rest of the stage and is
    applied per output after the stage's product, so the circuit runs on the tensor
    cores."""
    ops = W.qft(n)
    x = W.gaussian_state(n, 3)
    got, want, path = run_tc(n, ops, psi=x)
    assert path == 2
    record("tc_qft_deferred", n=n, rel_l2=rel_l2(got, want))
    assert rel_l2(got, want) <= TOL["c64"]


def test_tc_inverse_qft_and_open_control_phases():
    """The inverse QFT (negative ladders, the swaps first) and controlled phases on far
    qubits with open and closed controls -- among them controlled Z rotations with an
    open control, whose deferred part is conditioned on the control reading 0 --
    interleaved with Hadamards and T gates, all on the tensor-core passes."""
    n = 18
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
    x = W.gaussian_state(n, 5)
    got, want, path = run_tc(n, ops, psi=x)
    assert path == 2
    record("tc_inverse_qft_phases", n=n, path=path, rel_l2=rel_l2(got, want))
    assert rel_l2(got, want) <= TOL["c64"]


def test_tc_falls_back_for_a_doubly_controlled_phase_outside_the_tile():
    """A phase conditioned on two far qubits whose phase bit lies elsewhere cannot be
    deferred (its condition spans two slots); the result is the same either way."""
    n = 16
    ops = [Op("h", (q,)) for q in range(n)]
    ops.append(Op("ctrl", (0, n - 1, n // 2), matrix=np.diag([1.0, np.exp(0.7j)])))
    ops += [Op("h", (q,)) for q in range(0, n, 3)]
    got, want, path = run_tc(n, ops)
    assert path in (1, 2)
    assert rel_l2(got, want) <= TOL["c64"]


@pytest.mark.slow
def test_tc_brickwork_28_inverse_property():
    """Full size, the benchmark's circuit: the 540-gate 28-qubit brickwork on the
    tensor-core passes, then its inverse, returns |0...0>; the forward state agrees
    with the complex64 per-gate sweeps."""
    import torch

    import paper_2503_03016_gb300 as P
    n = 28
    ops = W.brickwork(n, 40, 2)
    circ = P.Circuit(n, ops)
    inv = P.Circuit(n, W.circuit_inverse(ops))
    a = P.State(n, "c64").init_basis(0)
    P.qc_run_circuit(a.handle, circ, None, P.QC_RUN_FUSED, P.QC_PREC_TF32X3)
    assert P.qc_last_fused_path() == 2
    b = P.State(n, "c64").init_basis(0)
    P.qc_run_circuit(b.handle, circ, None, P.QC_RUN_PER_GATE)
    diff = torch.linalg.vector_norm(a.tensor - b.tensor).item()
    assert diff <= 1e-5, diff
    P.qc_run_circuit(a.handle, inv, None, P.QC_RUN_FUSED, P.QC_PREC_TF32X3)
    amp0 = a.tensor[0].item()
    assert abs(amp0 - 1) < 2e-5, amp0


def test_auto_precision_picks_and_caches_a_path(tmp_path, monkeypatch):
    """QC_PREC_AUTO times both kinds of fused pass once per circuit structure, keeps the
    faster (recorded in QC_AUTOTUNE_CACHE), and either way matches the oracle; a second
    run of the same structure with other matrices takes the same path without timing."""
    import paper_2503_03016_gb300 as P
    n = 16
    cache = tmp_path / "autotune.txt"
    monkeypatch.setenv("QC_AUTOTUNE_CACHE", str(cache))
    ops = W.brickwork(n, 10, 77)
    psi = W.random_state(n, 4)
    st = gpu_state(psi, "c64")
    st.run(ops, mode=P.QC_RUN_FUSED, prec=P.QC_PREC_AUTO)
    path = P.qc_last_fused_path()
    assert path in (1, 2)
    assert rel_l2(st.numpy(), oracle.run(psi.copy(), ops)) <= TOL["c64"]
    lines = cache.read_text().split("\n")
    assert any(l.endswith(" 0") or l.endswith(" 2") for l in lines)
    ops2 = W.brickwork(n, 10, 78)  # same structure, other unitaries
    st2 = gpu_state(psi, "c64")
    st2.run(ops2, mode=P.QC_RUN_FUSED, prec=P.QC_PREC_AUTO)
    assert P.qc_last_fused_path() == path
    assert len(cache.read_text().strip().split("\n")) == len([l for l in lines if l.strip()])
    assert rel_l2(st2.numpy(), oracle.run(psi.copy(), ops2)) <= TOL["c64"]


def test_bf16x3_is_rejected():
    import paper_2503_03016_gb300 as P
    st = gpu_state(W.random_state(12, 1), "c64")
    with pytest.raises(P.QCError) as e:
        st.run(W.brickwork(12, 2, 1), mode=P.QC_RUN_FUSED, prec=P.QC_PREC_BF16X3)
    assert e.value.status == 4


@pytest.mark.parametrize("n", [13, 17])
def test_tc_swaps_as_relabelings(n):
    """SWAPs between random qubits among dense two-qubit gates and a final bit
    reversal: a pass may take its SWAPs as a relabeling (the tile permuted before its
    write-back) instead of stage ops; the result matches the oracle either way."""
    rng = np.random.default_rng(n)
    U = W.haar_unitaries(60, 4, 3 * n)
    ops = []
    for i in range(60):
        a = int(rng.integers(0, n - 1))
        ops.append(Op("u2q", (a, a + 1), matrix=U[i]))
        if i % 4 == 3:
            b, c = (int(v) for v in rng.choice(n, 2, replace=False))
            ops.append(Op("swap", (b, c)))
    ops += [Op("swap", (j, n - 1 - j)) for j in range(n // 2)]
    got, want, path = run_tc(n, ops)
    assert path == 2
    record("tc_swaps_relabeled", n=n, rel_l2=rel_l2(got, want))
    assert rel_l2(got, want) <= TOL["c64"]


@pytest.mark.parametrize("n", [14, 18])
def test_tc_ansatz_ring(n):
    """The adjoint benchmark's ansatz (RY RZ on every qubit, a CZ ring) on the
    tensor-core passes: a CZ to a qubit outside the stage's slots is deferred, and the
    stage cut keeps the next layer's rotations of that qubit out of the stage."""
    layers = 4
    ops = W.ansatz(n, layers, True)
    params = np.random.default_rng(n).uniform(0, 2 * np.pi, layers * 2 * n)
    got, want, path = run_tc(n, ops, params=params)
    assert path == 2
    record("tc_ansatz_ring", n=n, rel_l2=rel_l2(got, want))
    assert rel_l2(got, want) <= TOL["c64"]
