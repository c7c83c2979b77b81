"""E(theta) = <0|U(theta)^dag H U(theta)|0> as a torch.autograd.Function.

The forward pass runs the circuit and the Pauli-sum expectation on the GPU;
the backward pass calls the library's adjoint gradient, which re-derives the
intermediate states by applying inverse gates instead of storing them.
"""

from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class AdjointExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, circuit, hamiltonian, psi, lam, opts):
        th = theta.detach().to("cpu", torch.float64).numpy()
        circuit.set_params(th)
        psi.init_basis(0)
        plan = B.Plan(circuit, psi.dtype, opts)
        plan.execute(psi)
        e = B.expectation(psi, hamiltonian)
        plan.close()
        ctx.objs = (circuit, hamiltonian, psi, lam)
        ctx.theta = th
        return torch.tensor(e, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        if not ctx.needs_input_grad[0]:
            return None, None, None, None, None, None
        circuit, hamiltonian, psi, lam = ctx.objs
        _, g = B.adjoint_gradient(circuit, ctx.theta, hamiltonian, psi, lam)
        g = torch.from_numpy(np.asarray(g)) * grad_out.to(torch.float64)
        return g, None, None, None, None, None


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
