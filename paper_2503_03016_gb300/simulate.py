"""QCLAB's ``simulate`` (Sec. 3.1 - 3.3) on the GPU: start state, gates, and
measurements with outcome branching.

Host control flow only: every amplitude operation is a C-ABI call (qc_run_circuit,
qc_state_copy, qc_collapse).  A measurement in the X or Y basis applies the basis
change before and its inverse after the Z measurement (Sec. 3.3): X = H .. H, Y =
S^dagger H .. H S.  A reset (mentioned in Sec. 3.3, not defined there) is a Z
measurement whose outcome-1 branch is then flipped by X; its outcome labels the branch
like a measurement's.  A branch whose outcome probability is at most the zero threshold
of qc_collapse is dropped (1e-12 complex128, 1e-6 complex64)."""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from . import _binding as B
from .state import State

_BASIS_PRE = {"z": [], "x": ["h"], "y": ["sdg", "h"]}
_BASIS_POST = {"z": [], "x": ["h"], "y": ["h", "s"]}


class _Op:  # minimal op record for basis changes (same fields the binding reads)
    def __init__(self, kind, q):
        self.kind, self.qubits, self.params, self.matrix = kind, (q,), (), None
        self.ctrl_states, self.param_index = None, None


def _start(n: int, init, dtype: str) -> State:
    st = State(n, dtype)
    if isinstance(init, str):
        if len(init) != n or any(c not in "01" for c in init):
            raise ValueError("bitstring start must have n characters 0/1")
        st.init_basis(int(init, 2))
    elif isinstance(init, (int, np.integer)):
        st.init_basis(int(init))
    else:
        v = np.asarray(init, dtype=np.complex128 if dtype == "c128" else np.complex64)
        st.init_vector(v)
    return st


def _copy(st: State) -> State:
    out = State(st.n, "c64" if st.dtype == B.QC_C64 else "c128")
    B.qc_state_copy(out.handle, st.handle)
    return out


def simulate(n: int, ops: Sequence, init, dtype: str = "c128", params=None,
             mode: int = B.QC_RUN_PER_GATE) -> Tuple[List[str], List[float], List[State]]:
    """Returns (results, probabilities, states): one entry per branch with nonzero
    probability, outcome 0 before 1 at every measurement, results listing the measured
    bits in measurement order."""
    branches = [("", 1.0, _start(n, init, dtype))]
    pending: list = []

    def flush():
        if pending:
            circ = B.Circuit(n, list(pending))
            for _, _, st in branches:
                B.qc_run_circuit(st.handle, circ, params, mode, B.QC_PREC_NATIVE)
            pending.clear()

    for op in ops:
        reset = op.kind == "reset"
        if not (op.kind.startswith("measure") or reset):
            pending.append(op)
            continue
        flush()
        q = op.qubits[0]
        basis = "z" if reset else op.kind[len("measure"):].lstrip("_") or "z"
        pre = [_Op(k, q) for k in _BASIS_PRE[basis]]
        post = [_Op(k, q) for k in _BASIS_POST[basis]]
        new = []
        for res, pr, st in branches:
            if pre:
                B.qc_run_circuit(st.handle, B.Circuit(n, pre), None, B.QC_RUN_PER_GATE, B.QC_PREC_NATIVE)
            for o in (0, 1):
                s2 = _copy(st)
                try:
                    p = B.qc_collapse(s2.handle, q, o)
                except B.QCError as e:
                    if e.status == 5:  # QC_ERR_ZERO_PROB: no such branch
                        s2.free()
                        continue
                    raise
                after = post + ([_Op("x", q)] if reset and o == 1 else [])
                if after:
                    B.qc_run_circuit(s2.handle, B.Circuit(n, after), None, B.QC_RUN_PER_GATE, B.QC_PREC_NATIVE)
                new.append((res + str(o), pr * p, s2))
            st.free()
        branches = new
    flush()
    return [b[0] for b in branches], [b[1] for b in branches], [b[2] for b in branches]


def reduced_statevector(st: State, known: Sequence[int], bits: str):
    """QCLAB's reducedStatevector (Sec. 5.1) on the GPU: a torch tensor of the
    amplitudes whose known qubits carry `bits`."""
    import torch
    m = len(known)
    tdt = torch.complex64 if st.dtype == B.QC_C64 else torch.complex128
    out = torch.empty(1 << (st.n - m), dtype=tdt, device="cuda")
    B.qc_reduced_state(st.handle, list(known), [int(c) for c in bits], out)
    return out


def counts(st: State, qubits: Sequence[int], u) -> np.ndarray:
    """Frequencies of the outcomes of measuring `qubits` (qubits[0] most significant)
    for the caller's uniforms `u` (a CUDA float64 tensor): the marginal distribution
    (qc_marginal_probs) sampled by qc_sample_probs (Sec. 5.2 counts)."""
    import torch
    m = len(qubits)
    marg = torch.empty(max(2, 1 << m), dtype=torch.float64, device="cuda")
    B.qc_marginal_probs(st.handle, list(qubits), marg)
    out = torch.empty(u.numel(), dtype=torch.int64, device="cuda")
    B.qc_sample_probs(st.handle, marg, m, u, u.numel(), out)
    return np.bincount(out.cpu().numpy(), minlength=1 << m)
