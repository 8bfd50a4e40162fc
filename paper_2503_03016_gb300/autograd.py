"""torch.autograd binding of the adjoint gradient (qc_adjoint_grad)."""
from __future__ import annotations

import numpy as np

from . import _binding as B


class AdjointExpectation:
    """E(theta) = <psi(theta)| H |psi(theta)> with psi(theta) = circuit(theta)|0...0>.

    ``AdjointExpectation.apply(params, circuit, strings, coeffs, dtype)`` returns a
    0-d tensor; its gradient with respect to ``params`` comes from the library's
    reverse sweep (one forward sweep + one backward sweep, both on the GPU)."""

    _fn = None

    @classmethod
    def apply(cls, params, circuit, strings, coeffs=None, dtype=B.QC_C128):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, theta, circ, terms, cf, dt):
                    host = theta.detach().to("cpu", torch.float64).numpy()
                    e, g = B.qc_adjoint_grad(circ, host, terms, cf, dt)
                    ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
                    return torch.tensor(e, dtype=theta.dtype, device=theta.device)

                @staticmethod
                def backward(ctx, grad_out):
                    (g,) = ctx.saved_tensors
                    return grad_out * g, None, None, None, None

            cls._fn = _F
        if not isinstance(circuit, B.Circuit):
            raise TypeError("circuit must be a paper_2503_03016_gb300.Circuit")
        return cls._fn.apply(params, circuit, list(strings), None if coeffs is None else np.asarray(coeffs), dtype)
