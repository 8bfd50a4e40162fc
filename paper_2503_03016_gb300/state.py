"""A state whose amplitudes live in a torch CUDA tensor (torch allocates device
memory; the CUDA library does all the work)."""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import _binding as B


class State:
    def __init__(self, n: int, dtype: str = "c64", stream=None):
        import torch
        self.n = n
        self.dtype = B.QC_C64 if dtype in ("c64", "complex64", B.QC_C64) else B.QC_C128
        tdt = torch.complex64 if self.dtype == B.QC_C64 else torch.complex128
        self.tensor = torch.empty(1 << n, dtype=tdt, device="cuda")
        self.handle = B.qc_state_wrap(n, self.dtype, self.tensor, stream)

    def free(self) -> None:
        if self.handle:
            B.qc_state_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # initialisation
    def init_basis(self, index: int = 0) -> "State":
        B.qc_state_init_basis(self.handle, index)
        return self

    def init_vector(self, v) -> "State":
        v = np.ascontiguousarray(v)
        src = B.QC_C64 if v.dtype == np.complex64 else B.QC_C128
        if src == B.QC_C128:
            v = v.astype(np.complex128)
        B.qc_state_init_vector(self.handle, v, src, True)
        import torch
        torch.cuda.current_stream().synchronize()
        return self

    def init_gaussian(self, seed: int) -> "State":
        B.qc_state_init_gaussian(self.handle, seed)
        return self

    def numpy(self) -> np.ndarray:
        return B.qc_state_download(self.handle)

    # gates
    def apply_1q(self, q, U):
        B.qc_apply_1q(self.handle, q, U)

    def apply_2q(self, qa, qb, U):
        B.qc_apply_2q(self.handle, qa, qb, U)

    def apply_ctrl(self, ctrls, states, target, U):
        B.qc_apply_ctrl(self.handle, ctrls, states, target, U)

    def apply_fused_k(self, qubits, U, prec=B.QC_PREC_NATIVE):
        B.qc_apply_fused_k(self.handle, qubits, U, prec)

    def run(self, circuit, params=None, mode=B.QC_RUN_PER_GATE, prec=B.QC_PREC_NATIVE):
        if not isinstance(circuit, B.Circuit):
            circuit = B.Circuit(self.n, circuit)
        B.qc_run_circuit(self.handle, circuit, params, mode, prec)

    # readout
    def probs(self):
        import torch
        out = torch.empty(1 << self.n, dtype=torch.float64, device="cuda")
        B.qc_probs(self.handle, out)
        return out

    def sample(self, u):
        import torch
        out = torch.empty(u.numel(), dtype=torch.int64, device="cuda")
        B.qc_sample(self.handle, u, u.numel(), out)
        return out

    def expect(self, strings, coeffs=None):
        return B.qc_expect_pauli(self.handle, strings, coeffs)

    def measure(self, q, u):
        return B.qc_measure(self.handle, q, u)

    def collapse(self, q, outcome):
        return B.qc_collapse(self.handle, q, outcome)
