"""E(theta) = <0|U(theta)^dag H U(theta)|0> as a torch.autograd.Function.

When the gradient is needed, the forward pass makes ONE library call,
qs_adjoint_gradient, which runs the circuit once, forms E and walks the
gates backwards (re-deriving the intermediate states by applying inverse
gates instead of storing them); the gradient is kept for the backward pass,
which only scales it by the incoming gradient.  So a training step runs the
circuit once, not once for E and again inside the gradient.  Without a
gradient (no_grad, or theta not requiring one) the forward runs the fused
circuit and the expectation only.  E and dE/dtheta come back on theta's
device and in theta's dtype.
"""

from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class AdjointExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, circuit, hamiltonian, psi, lam, opts):
        th = np.ascontiguousarray(theta.detach().to("cpu", torch.float64).numpy())
        if ctx.needs_input_grad[0]:
            e, g = B.adjoint_gradient(circuit, th, hamiltonian, psi, lam)
            ctx.save_for_backward(torch.from_numpy(g).to(device=theta.device, dtype=theta.dtype))
        else:
            circuit.set_params(th)
            psi.init_basis(0)
            plan = B.Plan(circuit, psi.dtype, opts)
            plan.execute(psi)
            e = B.expectation(psi, hamiltonian)
            plan.close()
        return torch.tensor(e, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        if not ctx.needs_input_grad[0]:
            return None, None, None, None, None, None
        (g,) = ctx.saved_tensors
        return g * grad_out.to(g.dtype), None, None, None, None, None


class Expectation(torch.nn.Module):
    """Module wrapper: owns the circuit, Hamiltonian and two work states."""

    def __init__(self, circuit_spec, hamiltonian_terms, dtype="c64", k_max=4):
        super().__init__()
        self.circuit = B.circuit_from(circuit_spec)
        self.h = B.PauliSum(circuit_spec.n, hamiltonian_terms)
        self.psi = B.State(circuit_spec.n, dtype)
        self.lam = B.State(circuit_spec.n, dtype, init=None)
        self.opts = B.options(k_max=k_max)

    def forward(self, theta):
        return AdjointExpectation.apply(theta, self.circuit, self.h, self.psi, self.lam, self.opts)
