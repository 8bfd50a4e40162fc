"""Host-only planning (qc_plan_info, no GPU): tile passes, register stages and ops of
the fused path."""
import pytest

import workloads as W
from workloads import Op


def plan(n, ops, dtype):
    import paper_2503_03016_gb300 as P
    return P.qc_plan_info(P.Circuit(n, ops), None, dtype)


@pytest.mark.parametrize("n", [12, 16, 26])
def test_exact_swaps_are_relabelings(n):
    """An exact SWAP inside a tile applies no arithmetic (the pass's later ops name the
    exchanged bits and the write-out reads the tile through the permutation): the QFT
    plans the same ops as the QFT without its final swaps, for both precisions."""
    import paper_2503_03016_gb300 as P
    ops = W.qft(n)
    noswap = [o for o in ops if o.kind != "swap"]
    for dt in (P.QC_C64, P.QC_C128):
        assert plan(n, ops, dt)[2] == plan(n, noswap, dt)[2]


def test_controlled_swap_is_not_a_relabeling():
    """A SWAP with a control (a three-qubit gate built as CNOT-Toffoli-CNOT) keeps its
    arithmetic: only exact, unconditioned SWAPs are relabeled."""
    import paper_2503_03016_gb300 as P
    n = 12
    fredkin = [Op("cnot", (2, 1)), Op("mcx", (0, 1, 2)), Op("cnot", (2, 1))]
    assert plan(n, fredkin, P.QC_C64)[2] == 3
    assert plan(n, [Op("swap", (1, 2))] * 3, P.QC_C64)[2] == 0


def test_brickwork_plan_is_stable():
    """The 28-qubit Haar brickwork: 24 passes, 153 register stages of 4 bits, 540 ops
    (complex64)."""
    import paper_2503_03016_gb300 as P
    assert plan(28, W.brickwork(28, 40, 2), P.QC_C64) == (24, 153, 540)
