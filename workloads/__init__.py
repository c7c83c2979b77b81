"""Seeded synthetic inputs (circuits, parameters, Hamiltonians, states).

Shared by the tests, the benchmark and the oracle's callers.  It defines the
inputs only: it neither simulates nor fuses gates.
"""

from . import gates, rng, circuits  # noqa: F401
from .circuits import (Circuit, Gate, PauliTerm, ansatz_circuit, ansatz_theta,  # noqa: F401
                       batched_workload, grid_circuit, grid_shape, ising_hamiltonian,
                       random_circuit, scale_grid_circuit, small_grid_circuit)
