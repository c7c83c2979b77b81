"""The FP64 oracle against facts that do not come from the oracle itself."""

import numpy as np
import pytest

import oracle
import pins
from workloads.circuits import ansatz_circuit, ansatz_theta, ising_hamiltonian


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(check):
    check()


@pytest.mark.parametrize("n,gates,k", [(4, 10, 1), (6, 30, 2), (8, 40, 3), (9, 20, 4)])
def test_brute_force_sizes(n, gates, k):
    pins.check_brute_force(n=n, num_gates=gates, seed=n * 7 + k, max_k=k)


def test_parameter_shift_matches_fd_on_ansatz():
    """On the full ansatz (with the CZ ladder) parameter shift and central
    differences agree to the FD truncation error O(h^2)."""
    n, layers = 4, 2
    theta = ansatz_theta(n, layers, seed=3)
    build = lambda t: ansatz_circuit(n, layers, t).gates
    H = ising_hamiltonian(n)
    ps = oracle.parameter_shift_gradient(n, build, theta, H)
    fd = oracle.central_fd_gradient(n, build, theta, H, h=1e-4)
    assert np.max(np.abs(ps - fd)) < 2e-8
