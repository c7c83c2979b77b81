"""FP64 CPU oracle: test infrastructure only.

Only tests, the package entry's smoke check and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never imports it, and it imports nothing from the product.
"""

from . import metrics, statevector  # noqa: F401
from .statevector import (apply_gate, apply_pauli_sum, basis_state, central_fd_gradient,  # noqa: F401
                          energy, expectation, full_unitary, gate_unitary, norm_sq,
                          parameter_shift_gradient, probabilities, simulate, zero_state)
