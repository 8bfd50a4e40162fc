"""Host-only check of the CUDA-core tile-pass planner (qc_tile_emulate; no GPU needed): the
plan QC_RUN_FUSED builds -- passes, register stages, tile ops with their conditions on
slots, lanes and global bits, matrices, phase tables, CZ code words, relabeled SWAPs --
interpreted on the host in FP64 in the kernel's order, against the oracle.  Both plan
structures are checked: complex64's (dense SWAPs, no butterflies) and complex128's
(SWAPs as register permutations, butterflies, real matrices).  The interpretation is
exact up to FP64 rounding, so the bound is 1e-12: a planning mistake gives errors of
order 1."""
import numpy as np
import pytest

import oracle
import workloads as W
from workloads import Op

from test_tc_emulate_host import MIXES, _mixed, _weighted

DTYPES = ["c64", "c128"]


def emulate(n, ops, dtype, psi=None, params=None):
    import paper_2503_03016_gb300 as P
    psi = W.random_state(n, n) if psi is None else psi
    got = P.qc_tile_emulate(P.Circuit(n, ops), psi, params, P.QC_C64 if dtype == "c64" else P.QC_C128)
    want = oracle.run(psi.copy(), ops, params)
    return np.linalg.norm(got - want) / np.linalg.norm(want)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [12, 14, 17])
def test_qft(dtype, n):
    assert emulate(n, W.qft(n), dtype, psi=W.gaussian_state(n, 3)) <= 1e-12


@pytest.mark.parametrize("dtype", DTYPES)
def test_brickwork_and_ansatz_ring(dtype):
    assert emulate(13, W.brickwork(13, 16, 7), dtype) <= 1e-12
    n, layers = 15, 4
    params = np.random.default_rng(n).uniform(0, 2 * np.pi, layers * 2 * n)
    assert emulate(n, W.ansatz(n, layers, True), dtype, params=params) <= 1e-12


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [10, 12, 13, 16])
def test_mixed_circuits(dtype, n):
    """Every gate kind on random qubits, controls inside and outside the tile."""
    for seed in (1, 2, 3):
        assert emulate(n, _mixed(n, seed), dtype) <= 1e-12, (n, seed)


@pytest.mark.parametrize("dtype", DTYPES)
def test_cz_runs_and_swaps(dtype):
    """Runs of CZ gates (one sign op per run) across the register, and SWAPs between
    random qubits with a final bit reversal (relabelings)."""
    n = 14
    rng = np.random.default_rng(5)
    ops = [Op("h", (q,)) for q in range(n)]
    for _ in range(6):
        for _ in range(8):
            a, b = (int(v) for v in rng.choice(n, 2, replace=False))
            ops.append(Op("cz", (a, b)))
        for q in rng.choice(n, 4, replace=False):
            ops.append(Op("ry", (int(q),), (float(rng.uniform(0, 6.3)),)))
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        ops.append(Op("swap", (a, b)))
    ops += [Op("swap", (j, n - 1 - j)) for j in range(n // 2)]
    assert emulate(n, ops, dtype) <= 1e-12


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mix", sorted(MIXES))
def test_weighted_random_circuits(dtype, mix):
    """Seeded circuits weighted towards phases, SWAPs or dense gates (12 to 18 qubits)."""
    for n in (12, 15, 18):
        for seed in range(2):
            count = int(np.random.default_rng(seed + 7).integers(20, 200))
            ops = _weighted(n, 1000 * n + seed, count, MIXES[mix])
            assert emulate(n, ops, dtype) <= 1e-12, (n, seed)


def test_rejects_invalid_arguments():
    import paper_2503_03016_gb300 as P
    with pytest.raises(P.QCError):
        P.qc_tile_emulate(P.Circuit(9, W.qft(9)), W.random_state(9, 1))
