"""Block adjoint sweep (complex64, 12 or more qubits): every gradient inside a
fused 6-qubit block comes from the block's 64 x 64 Gram matrix
M = sum_s psi_s lambda_s^dagger and a recursion over the block's gates.

The circuits are built from layers on chosen six-qubit sets, so that blocks
with every kind of target placement occur and each copy form of the Gram
kernel runs: qubit 0 a target but not qubits 1 and 2 (row pairs), qubits
0-2 targets (64-byte row groups), qubit 0 not a target (16-byte set pairs),
and only high qubits.  Each layer mixes one-qubit rotations with X, Y and Z
generators, a CZ chain, a ZZ and an XY rotation, and a fixed gate, so runs
of diagonal gates (merged in the recursion) and dense gates alternate.
Reference: exact parameter shift on the FP64 oracle."""

import numpy as np
import pytest

import oracle
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C
from workloads import gates as G
from workloads.rng import Xoshiro256ss

pytestmark = pytest.mark.gpu

SETS = [(0, 3, 5, 7, 9, 11), (0, 1, 2, 6, 8, 12), (1, 4, 6, 8, 10, 12), (7, 8, 9, 10, 11, 12)]


def block_circuit(n, reps, theta):
    circ = C.Circuit(n)
    p = 0

    def rot(qubits, gen):
        nonlocal p
        circ.append(qubits, G.pauli_rotation(gen, theta[p]), gen, p, gen)
        p += 1

    for r in range(reps):
        for k, S in enumerate(SETS):
            for i, q in enumerate(S):
                rot((q,), "XYZ"[(i + r + k) % 3])
                rot((q,), "Z")
            for a, b in zip(S, S[1:]):
                circ.append((a, b), G.CZ, "cz")
            rot((S[0], S[-1]), "ZZ")
            rot((S[1], S[2]), "XY")
            circ.append((S[3],), G.SQRT_X if (r + k) % 2 else G.H, "fixed")
    circ.num_params = p
    return circ


def test_block_sweep_target_placements(qs):
    n, reps = 13, 2
    P = block_circuit(n, reps, np.zeros(100000)).num_params
    rng = Xoshiro256ss(515)
    theta = np.array([rng.uniform_range(-np.pi, np.pi) for _ in range(P)])
    terms = C.ising_hamiltonian(n) + [C.PauliTerm(0.5, ((2, "Y"), (n - 1, "X"))),
                                      C.PauliTerm(0.3, ((0, "Z"), (7, "Y")))]
    build = lambda t: block_circuit(n, reps, t).gates
    ps = oracle.parameter_shift_gradient(n, build, theta, terms)
    e_ref = oracle.energy(n, build, theta, terms)
    c = B.circuit_from(block_circuit(n, reps, theta))
    h = B.PauliSum(n, terms)
    # two calls in a row: the second reuses the cached grouping and the library's memory pool
    for _ in range(2):
        e, g = B.adjoint_gradient(c, theta, h, B.State(n, "c64"), B.State(n, "c64", init=None))
        assert abs(e - e_ref) < 1e-4 * max(1.0, abs(e_ref))
        assert np.linalg.norm(g - ps) / np.linalg.norm(ps) < 1e-4, np.max(np.abs(g - ps))
