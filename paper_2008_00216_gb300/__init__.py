"""GB300 (sm_103a) Schroedinger-style state-vector simulator.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/qsgb.h``); this package is its binding.  Importing it does not
touch the GPU; ``load()`` loads (and if needed builds) the library and fails
loudly when it cannot.
"""

from .binding import (Circuit, Options, PauliSum, Plan, QsError, State, adjoint_gradient,  # noqa: F401
                      apply_circuit, apply_gate, apply_pauli_sum, circuit_from, expectation,
                      exported_symbols, fuse, load, options, version)


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)
