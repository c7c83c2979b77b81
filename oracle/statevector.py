"""Plain FP64 CPU state-vector oracle.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the package entry's smoke check and the
benchmark's CPU-baseline / reference leg use it.  It shares no code with the
CUDA library and imports nothing from it.

What it computes (all in complex128 / float64):

* ``apply_gate``: Section 3, "Fast Schroedinger simulation".  A q-qubit gate
  on qubits i_0..i_{q-1} splits the 2^n amplitudes into 2^(n-q) disjoint sets
  of 2^q amplitudes; the other n-q index bits form the set id; each set a is
  replaced by M a.  Index bit b of an amplitude is the value of qubit b
  (qubit 0 is the least significant bit); inside a set, qubits[0] is the most
  significant local bit (Kronecker order of Eq. 1).
* ``simulate``: psi_out = U_L ... U_1 psi_0, one gate at a time (Section 3).
* ``full_unitary``: the Kronecker-padded 2^n x 2^n evaluation of Section 3,
  built entry by entry (only for n <= 10).
* ``norm_sq``: sum of |alpha_j|^2 accumulated without rounding drift, the
  accuracy check of Section 4.1 (math.fsum returns the correctly rounded
  sum, stronger than the paper's double or sum-of-two accumulation).
* ``expectation``: <psi|H|psi> for a Pauli sum, by applying each Pauli
  string with ``apply_gate`` and taking the inner product.
* ``parameter_shift_gradient`` / ``central_fd_gradient``: dE/dtheta for
  gates exp(-i theta P / 2) with P^2 = I.

Every function above is pinned by tests that do not reuse it (brute force,
closed forms, invariants); none is "parity unpinned".
"""

from __future__ import annotations

import math
from typing import Callable, Iterable, Sequence, Tuple

import numpy as np

# Pauli matrices, written out here (the oracle keeps its own constants).
_PAULI = {
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def _check_gate(n: int, qubits: Sequence[int], m: np.ndarray) -> int:
    k = len(qubits)
    if k < 1 or k > n:
        raise ValueError("gate must act on 1..n qubits")
    if len(set(qubits)) != k or min(qubits) < 0 or max(qubits) >= n:
        raise ValueError(f"bad qubit list {qubits} for n={n}")
    if m.shape != (1 << k, 1 << k):
        raise ValueError("matrix shape does not match the qubit count")
    return k


def zero_state(n: int) -> np.ndarray:
    """|0...0>: the computation starts from the first basis vector (Section 2)."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def basis_state(n: int, j: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[j] = 1.0
    return psi


def apply_gate(psi: np.ndarray, n: int, qubits: Sequence[int], m) -> np.ndarray:
    """Return the state after applying matrix m on `qubits` (Section 3).

    The state is viewed as an n-axis 2 x ... x 2 array in which axis a holds
    index bit n-1-a.  The gate's axes are moved to the front in the order
    qubits[0], ..., qubits[k-1], so the array reshapes into a 2^k x 2^(n-k)
    matrix whose columns are exactly the 2^(n-k) sets of Section 3 and whose
    row index has qubits[0] as its most significant bit.  Each column is
    multiplied by m (one library matmul), and the axes are put back.
    """
    m = np.asarray(m, dtype=np.complex128)
    k = _check_gate(n, qubits, m)
    axes = [n - 1 - q for q in qubits]
    t = np.moveaxis(psi.reshape((2,) * n), axes, list(range(k)))
    shape = t.shape
    cols = t.reshape(1 << k, -1)
    out = (m @ cols).reshape(shape)
    return np.ascontiguousarray(np.moveaxis(out, list(range(k)), axes)).reshape(-1)


def simulate(n: int, gates: Iterable, psi0: np.ndarray | None = None) -> np.ndarray:
    """psi_out = U_L ... U_1 psi_0 (default psi_0 = |0...0>), gate by gate.

    `gates` yields objects with `.qubits` and `.matrix`, or (qubits, matrix)
    pairs."""
    psi = zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128)
    if psi.shape != (1 << n,):
        raise ValueError("initial state has the wrong size")
    for g in gates:
        qs, m = (g.qubits, g.matrix) if hasattr(g, "qubits") else g
        psi = apply_gate(psi, n, qs, m)
    return psi


def gate_unitary(n: int, qubits: Sequence[int], m) -> np.ndarray:
    """The 2^n x 2^n matrix of one gate, entry by entry (Section 3's padded
    operator): U[j_out, j_in] = m[l_out, l_in] when j_out and j_in agree on
    every bit outside `qubits`, where l is the 'qubits[0]-first' local index."""
    m = np.asarray(m, dtype=np.complex128)
    k = _check_gate(n, qubits, m)
    if n > 10:
        raise ValueError("full_unitary is only for n <= 10")
    dim = 1 << n
    mask = 0
    for q in qubits:
        mask |= 1 << q
    u = np.zeros((dim, dim), dtype=np.complex128)
    for j_in in range(dim):
        l_in = 0
        for i, q in enumerate(qubits):
            l_in |= ((j_in >> q) & 1) << (k - 1 - i)
        rest = j_in & ~mask
        for l_out in range(1 << k):
            j_out = rest
            for i, q in enumerate(qubits):
                j_out |= ((l_out >> (k - 1 - i)) & 1) << q
            u[j_out, j_in] = m[l_out, l_in]
    return u


def full_unitary(n: int, gates: Iterable) -> np.ndarray:
    """U_L ... U_1 as one 2^n x 2^n matrix (the method Section 3 calls
    infeasible at scale; used only as a brute-force check, n <= 10)."""
    u = np.eye(1 << n, dtype=np.complex128)
    for g in gates:
        qs, m = (g.qubits, g.matrix) if hasattr(g, "qubits") else g
        u = gate_unitary(n, qs, m) @ u
    return u


def norm_sq(psi: np.ndarray) -> float:
    """sum_j |alpha_j|^2, correctly rounded (Section 4.1's norm check)."""
    a = np.asarray(psi, dtype=np.complex128)
    return math.fsum((a.real * a.real + a.imag * a.imag).tolist())


def probabilities(psi: np.ndarray) -> np.ndarray:
    """|alpha_j|^2 (Section 2: outcome probabilities come from the amplitudes)."""
    return np.abs(psi) ** 2


def apply_pauli_string(psi: np.ndarray, n: int, ops: Sequence[Tuple[int, str]]) -> np.ndarray:
    for q, p in ops:
        psi = apply_gate(psi, n, (q,), _PAULI[p])
    return psi


def apply_pauli_sum(psi: np.ndarray, n: int, terms) -> np.ndarray:
    """H psi for H = sum_t c_t P_t."""
    out = np.zeros_like(psi)
    for t in terms:
        out += t.coeff * apply_pauli_string(psi, n, t.ops)
    return out


def expectation(psi: np.ndarray, n: int, terms) -> float:
    """<psi|H|psi> = sum_t c_t <psi|P_t|psi> (real for Hermitian H)."""
    total = 0.0
    for t in terms:
        total += t.coeff * np.vdot(psi, apply_pauli_string(psi, n, t.ops)).real
    return float(total)


def energy(n: int, build: Callable[[np.ndarray], Iterable], theta: np.ndarray, terms) -> float:
    """E(theta) = <0|U(theta)^dag H U(theta)|0>; `build(theta)` returns the gates."""
    return expectation(simulate(n, build(theta)), n, terms)


def parameter_shift_gradient(n: int, build, theta: np.ndarray, terms,
                             params: Sequence[int] | None = None) -> np.ndarray:
    """dE/dtheta_p = [E(theta_p + pi/2) - E(theta_p - pi/2)] / 2.

    Exact when theta_p enters through exactly one gate exp(-i theta_p P / 2)
    with P^2 = I: E(theta_p) = a + b cos(theta_p) + c sin(theta_p)."""
    theta = np.asarray(theta, dtype=np.float64)
    plist = list(range(theta.size)) if params is None else list(params)
    g = np.zeros(len(plist))
    for out_i, p in enumerate(plist):
        tp = theta.copy(); tp[p] += math.pi / 2
        tm = theta.copy(); tm[p] -= math.pi / 2
        g[out_i] = 0.5 * (energy(n, build, tp, terms) - energy(n, build, tm, terms))
    return g


def central_fd_gradient(n: int, build, theta: np.ndarray, terms, h: float = 1e-4,
                        params: Sequence[int] | None = None) -> np.ndarray:
    """[E(theta_p + h) - E(theta_p - h)] / (2h); truncation error O(h^2)."""
    theta = np.asarray(theta, dtype=np.float64)
    plist = list(range(theta.size)) if params is None else list(params)
    g = np.zeros(len(plist))
    for out_i, p in enumerate(plist):
        tp = theta.copy(); tp[p] += h
        tm = theta.copy(); tm[p] -= h
        g[out_i] = (energy(n, build, tp, terms) - energy(n, build, tm, terms)) / (2 * h)
    return g
