"""Gate matrices of the synthetic workloads (inputs, not simulation code).

Convention shared by every consumer of a gate: a k-qubit gate on
``qubits = (q0, q1, ..., q_{k-1})`` has a 2^k x 2^k matrix in Kronecker order
with ``q0`` the MOST significant local bit, exactly as the paper prints CNOT
and CZ with the control first (Section 2, Eq. 1).  So a gate on (a, b) with
matrix ``kron(A, B)`` equals A on a followed by B on b.

The single-qubit set is the Sycamore-style {sqrt(X), sqrt(Y), sqrt(W)}.
sqrt(X) is printed in Section 2.  The paper's printed sqrt(Y) squares to -Y,
so the principal square root (which squares to +Y) is used instead.  sqrt(W)
and fSim are not in the paper; their standard definitions are used:
for an involution P, sqrt(P) = ((1+i) I + (1-i) P) / 2, and
fSim(theta, phi) = [[1,0,0,0],[0,cos t,-i sin t,0],[0,-i sin t,cos t,0],
[0,0,0,exp(-i phi)]].
"""

from __future__ import annotations

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)          # the paper's P = Z^(1/2)
T = np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128)
W = (X + Y) / np.sqrt(2.0)

CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]],
                dtype=np.complex128)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]],
                dtype=np.complex128)


def sqrt_involution(p: np.ndarray) -> np.ndarray:
    """Principal square root of an involution P (P @ P = I)."""
    return ((1 + 1j) * np.eye(p.shape[0]) + (1 - 1j) * p) / 2.0


SQRT_X = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
SQRT_Y = 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128)
SQRT_W = 0.5 * np.array([[1 + 1j, -1j * np.sqrt(2.0)], [np.sqrt(2.0), 1 + 1j]],
                        dtype=np.complex128)

ONE_QUBIT_SET = {"sqrt_x": SQRT_X, "sqrt_y": SQRT_Y, "sqrt_w": SQRT_W}


def _snap(x: float) -> float:
    """cos/sin values within a few ulp of 0 or +-1 are those exact values
    (cos(pi/2) evaluates to 6e-17); exact zeros keep fSim(pi/2, phi) a
    permutation-with-phase matrix."""
    for v in (0.0, 1.0, -1.0):
        if abs(x - v) < 4e-16:
            return v
    return float(x)


def fsim(theta: float, phi: float) -> np.ndarray:
    c, s = _snap(np.cos(theta)), _snap(np.sin(theta))
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, complex(_snap(np.cos(phi)), -_snap(np.sin(phi)))]],
                    dtype=np.complex128)


def cphase(phi: float) -> np.ndarray:
    return np.diag([1, 1, 1, np.exp(1j * phi)]).astype(np.complex128)


PAULI = {"I": I2, "X": X, "Y": Y, "Z": Z}


def pauli_rotation(paulis: str, theta: float) -> np.ndarray:
    """exp(-i theta P / 2) = cos(theta/2) I - i sin(theta/2) P for a Pauli
    string P (first letter = most significant local qubit)."""
    p = np.array([[1.0 + 0j]])
    for c in paulis:
        p = np.kron(p, PAULI[c])
    return np.cos(theta / 2) * np.eye(p.shape[0]) - 1j * np.sin(theta / 2) * p


def ry(theta: float) -> np.ndarray:
    return pauli_rotation("Y", theta)


def rz(theta: float) -> np.ndarray:
    return pauli_rotation("Z", theta)
