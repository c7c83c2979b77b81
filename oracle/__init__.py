"""FP64 CPU oracle: test infrastructure only.

Only tests, the package entry's smoke check and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never imports it, and it imports nothing from the product.

``statevector`` is the numpy oracle; ``omp`` is the same Section 3 update as
a plain C loop parallel over set ids (for the full-state checks at 26-28
qubits and the timed CPU baseline); ``metrics`` holds the error measures.
"""

from . import metrics, statevector  # noqa: F401
from .statevector import (apply_gate, apply_pauli_sum, basis_state, central_fd_gradient,  # noqa: F401
                          energy, expectation, full_unitary, gate_unitary, norm_sq,
                          parameter_shift_gradient, probabilities, simulate, zero_state)
