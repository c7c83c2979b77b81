"""Fused reverse-sweep passes of the adjoint gradient (stages whose
non-diagonal gates act on one qubit, done tile by tile in registers).

(1) Layered circuits that use every op of the fused pass: one-qubit gates
with X, Y and Z generators and fixed complex ones (sqrt X, sqrt Y, H) on
qubits held in each register layout, diagonal stages with chunk tables,
gates across 8-qubit chunks (CZ, RZZ, a three-qubit phase), multi-qubit Z
generators, and stages that mix diagonal and one-qubit members.  Reference:
exact parameter shift on the FP64 oracle.

(2) At 24 qubits, beyond the oracle's reach: the gradient against exact
parameter shift computed from GPU forward evaluations (a different path:
fused forward plans and the expectation kernel), on sampled parameters."""

import numpy as np
import pytest

import oracle
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C
from workloads import gates as G
from workloads.rng import Xoshiro256ss

pytestmark = pytest.mark.gpu


def layered_circuit(n, layers, theta, seed=11):
    rng = Xoshiro256ss(seed)
    circ = C.Circuit(n)
    p = 0

    def rot(qubits, gen):
        nonlocal p
        circ.append(qubits, G.pauli_rotation(gen, theta[p]), gen, p, gen)
        p += 1

    ccz = np.diag([1, 1, 1, 1, 1, 1, 1, np.exp(0.7j)]).astype(np.complex128)
    for layer in range(layers):
        for q in range(n):
            rot((q,), "XYZ"[(q + layer) % 3] if q % 4 else "Y")
        for q in range(n - 1):
            circ.append((q, q + 1), G.CZ, "cz")
        for q in range(0, n - 5, 5):
            rot((q, q + 5), "ZZ")
        circ.append((2, min(9, n - 2), n - 1), ccz, "ccz")
        circ.append((n - 2,), G.T, "t")
        for q in range(n):  # fixed one-qubit gates, some complex
            u = (G.SQRT_X, G.SQRT_Y, G.H)[rng.randint(3)]
            circ.append((q,), u, "fixed")
        for q in range(1, n, 2):  # a stage mixing RZ (diagonal) and RX (one qubit)
            rot((q,), "Z")
            rot((q - 1,), "X")
    circ.num_params = p
    return circ


def count_params(n, layers):
    return layered_circuit(n, layers, np.zeros(100000)).num_params


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,layers,nsample", [(12, 3, 40), (16, 2, 16)])
def test_fused_sweep_layered(qs, dtype, n, layers, nsample):
    P = count_params(n, layers)
    rng = Xoshiro256ss(200 + n)
    theta = np.array([rng.uniform_range(-np.pi, np.pi) for _ in range(P)])
    terms = C.ising_hamiltonian(n) + [C.PauliTerm(0.4, ((3, "Y"), (n - 1, "Z")))]
    build = lambda t: layered_circuit(n, layers, t).gates
    sample = sorted({rng.randint(P) for _ in range(2 * nsample)})[:nsample]
    ps = oracle.parameter_shift_gradient(n, build, theta, terms, params=sample)
    e_ref = oracle.energy(n, build, theta, terms)
    spec = layered_circuit(n, layers, theta)
    c = B.circuit_from(spec)
    h = B.PauliSum(n, terms)
    e, g = B.adjoint_gradient(c, theta, h, B.State(n, dtype), B.State(n, dtype, init=None))
    tol = 1e-4 if dtype == "c64" else 1e-10
    assert abs(e - e_ref) < tol * max(1.0, abs(e_ref))
    assert np.linalg.norm(g[sample] - ps) / np.linalg.norm(ps) < tol, np.max(np.abs(g[sample] - ps))


def _gpu_energy(n, layers, theta, h, dtype):
    c = B.circuit_from(C.ansatz_circuit(n, layers, theta))
    s = B.State(n, dtype)
    B.apply_circuit(s, c)
    e = B.expectation(s, h)
    s.close()
    c.close()
    return e


def test_fused_sweep_full_size_shift_rule(qs):
    """24 qubits, 4 ansatz layers: complex128 gradient against parameter
    shift on GPU energies; complex64 within its precision of complex128."""
    n, layers = 24, 4
    theta = C.ansatz_theta(n, layers, seed=9)
    h = B.PauliSum(n, C.ising_hamiltonian(n))
    grads = {}
    for dt in ("c128", "c64"):
        c = B.circuit_from(C.ansatz_circuit(n, layers, theta))
        e, grads[dt] = B.adjoint_gradient(c, theta, h, B.State(n, dt), B.State(n, dt, init=None))
        c.close()
    rng = Xoshiro256ss(77)
    sample = sorted({rng.randint(theta.size) for _ in range(8)})
    ps = []
    for p in sample:
        tp, tm = theta.copy(), theta.copy()
        tp[p] += np.pi / 2
        tm[p] -= np.pi / 2
        ps.append((_gpu_energy(n, layers, tp, h, "c128") - _gpu_energy(n, layers, tm, h, "c128")) / 2)
    ps = np.array(ps)
    assert np.max(np.abs(grads["c128"][sample] - ps)) < 1e-9 * max(1.0, np.max(np.abs(ps)))
    ref = grads["c128"]
    assert np.linalg.norm(grads["c64"] - ref) / np.linalg.norm(ref) < 1e-4


def test_gradient_reuses_grouping_across_angles(qs):
    """One circuit object, several angle sets: the block grouping found for
    the first call is reused while the gates' kinds stay the same; gradients
    equal those of freshly built circuits, also when angles of 0 turn RY
    gates into the identity (a different kind, so a new grouping)."""
    n, layers = 14, 3
    h = B.PauliSum(n, C.ising_hamiltonian(n))
    t1 = C.ansatz_theta(n, layers, seed=21)
    t2 = C.ansatz_theta(n, layers, seed=22)
    t3 = t2.copy()
    t3[::7] = 0.0
    c = B.circuit_from(C.ansatz_circuit(n, layers, t1))
    for theta in (t1, t2, t3, t1):
        e, g = B.adjoint_gradient(c, theta, h, B.State(n, "c64"), B.State(n, "c64", init=None))
        fresh = B.circuit_from(C.ansatz_circuit(n, layers, theta))
        e0, g0 = B.adjoint_gradient(fresh, theta, h, B.State(n, "c64"), B.State(n, "c64", init=None))
        fresh.close()
        assert e == e0 and np.array_equal(g, g0)
    c.close()


@pytest.mark.parametrize("dtype,n", [("c64", 11), ("c64", 12), ("c64", 13), ("c128", 10), ("c128", 11)])
def test_sweep_smallest_sizes(qs, dtype, n):
    """At and just below the fused pass's tile size (12 qubits for complex64,
    11 for complex128; smaller states take the per-gate paths): gradients
    against oracle parameter shift."""
    layers = 2
    P = count_params(n, layers)
    rng = Xoshiro256ss(500 + n)
    theta = np.array([rng.uniform_range(-np.pi, np.pi) for _ in range(P)])
    terms = C.ising_hamiltonian(n)
    build = lambda t: layered_circuit(n, layers, t).gates
    sample = sorted({rng.randint(P) for _ in range(40)})[:20]
    ps = oracle.parameter_shift_gradient(n, build, theta, terms, params=sample)
    c = B.circuit_from(layered_circuit(n, layers, theta))
    e, g = B.adjoint_gradient(c, theta, B.PauliSum(n, terms), B.State(n, dtype), B.State(n, dtype, init=None))
    tol = 1e-4 if dtype == "c64" else 1e-10
    assert np.linalg.norm(g[sample] - ps) / np.linalg.norm(ps) < tol
