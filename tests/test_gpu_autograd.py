"""The torch.autograd.Function around the adjoint gradient: the ansatz (RY,
RZ on every qubit per layer, CZ ladder) at 12 qubits x 20 layers with the
transverse-field Ising H.  torch.autograd.grad of E(theta) against exact
parameter shift on the FP64 oracle (sampled parameters), for theta on the
CPU and on the GPU, complex64 and complex128 states; the gradient comes back
on theta's device in theta's dtype and is scaled by the incoming gradient."""

import numpy as np
import pytest
import torch

import oracle
from paper_2008_00216_gb300.autograd import Expectation
from workloads import circuits as C

pytestmark = pytest.mark.gpu

N, LAYERS = 12, 20
TOL = {"c64": 1e-4, "c128": 1e-10}
_REF = {}


def _reference():
    if not _REF:
        theta = C.ansatz_theta(N, LAYERS, seed=11)
        terms = C.ising_hamiltonian(N)
        build = lambda t: C.ansatz_circuit(N, LAYERS, t).gates
        rng = np.random.default_rng(4)
        params = np.sort(rng.choice(theta.size, 24, replace=False))
        _REF.update(theta=theta, params=params, terms=terms,
                    ps=oracle.parameter_shift_gradient(N, build, theta, terms, params=params),
                    energy=oracle.energy(N, build, theta, terms))
    return _REF


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("device", ["cpu", "cuda"])
def test_autograd_matches_parameter_shift(qs, dtype, device):
    ref = _reference()
    mod = Expectation(C.ansatz_circuit(N, LAYERS, ref["theta"]), ref["terms"], dtype=dtype)
    theta = torch.tensor(ref["theta"], dtype=torch.float64, device=device, requires_grad=True)
    e = mod(theta)
    assert e.device == theta.device and e.dtype == theta.dtype
    (g,) = torch.autograd.grad(e, theta)
    assert g.device == theta.device and g.dtype == theta.dtype
    g = g.detach().cpu().numpy()
    ps = ref["ps"]
    err = np.linalg.norm(g[ref["params"]] - ps) / np.linalg.norm(ps)
    assert err < TOL[dtype], err
    assert abs(e.item() - ref["energy"]) < (1e-4 if dtype == "c64" else 1e-10) * max(1.0, abs(ref["energy"]))


def test_autograd_chain_rule_and_no_grad(qs):
    """loss = 2E + E^2 gives (2 + 2E) dE/dtheta; a float32 theta gets a
    float32 gradient; under no_grad the forward gives the same E without a
    gradient call."""
    ref = _reference()
    mod = Expectation(C.ansatz_circuit(N, LAYERS, ref["theta"]), ref["terms"], dtype="c128")
    theta = torch.tensor(ref["theta"], dtype=torch.float64, device="cuda", requires_grad=True)
    e = mod(theta)
    (g,) = torch.autograd.grad(e, theta)
    theta2 = theta.detach().clone().requires_grad_(True)
    e2 = mod(theta2)
    (gl,) = torch.autograd.grad(2 * e2 + e2 * e2, theta2)
    assert torch.allclose(gl, (2 + 2 * e.detach()) * g, rtol=1e-12, atol=1e-14)
    with torch.no_grad():
        e3 = mod(theta.detach())
    assert abs(e3.item() - e.item()) < 1e-11
    t32 = torch.tensor(ref["theta"], dtype=torch.float32, device="cuda", requires_grad=True)
    (g32,) = torch.autograd.grad(mod(t32), t32)
    assert g32.dtype == torch.float32 and g32.device == t32.device
