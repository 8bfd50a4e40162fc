"""torch.autograd binding of the adjoint gradient (qc_adjoint_grad_dev)."""
from __future__ import annotations

import numpy as np

from . import _binding as B


class AdjointExpectation:
    """E(theta) = <psi(theta)| H |psi(theta)> with psi(theta) = circuit(theta)|0...0>.

    ``AdjointExpectation.apply(params, circuit, strings, coeffs, dtype)`` returns a
    0-d tensor on the parameters' device; its gradient with respect to ``params`` comes
    from the library's reverse sweep (one forward sweep + one backward sweep, both on
    the GPU).  The angles go to the library as a device FP64 tensor and the energy and
    gradient come back in device tensors on the current stream: nothing of them passes
    through host memory here (the library reads the angles once to build its plan)."""

    _fn = None

    @classmethod
    def apply(cls, params, circuit, strings, coeffs=None, dtype=B.QC_C128):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, theta, circ, ham, dt):
                    th = theta.detach().to(device="cuda", dtype=torch.float64).contiguous()
                    e = torch.empty(1, dtype=torch.float64, device=th.device)
                    g = torch.empty(th.numel(), dtype=torch.float64, device=th.device)
                    B.qc_adjoint_grad_dev(circ, th, ham, dt, e, g)
                    ctx.save_for_backward(g.to(dtype=theta.dtype, device=theta.device))
                    return e[0].to(dtype=theta.dtype, device=theta.device)

                @staticmethod
                def backward(ctx, grad_out):
                    (g,) = ctx.saved_tensors
                    return grad_out * g, None, None, None

            cls._fn = _F
        if not isinstance(circuit, B.Circuit):
            raise TypeError("circuit must be a paper_2503_03016_gb300.Circuit")
        ham = B.Hamiltonian.from_strings(list(strings), None if coeffs is None else np.asarray(coeffs))
        return cls._fn.apply(params, circuit, ham, dtype)
