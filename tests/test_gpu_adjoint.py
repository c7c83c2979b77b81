"""Adjoint gradient on circuits that exercise every path of the reverse
sweep: diagonal stages (phase tables, gates across 8-qubit chunks, ZZ
generators), general commuting stages (X, Y and two-qubit XY generators,
gradients from tile passes, inverse as fused passes) and short runs that
take the per-gate tile sweep (fixed H, sqrt(X), dense two-qubit gates).
Reference: exact parameter shift on the FP64 oracle."""

import numpy as np
import pytest

import oracle
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C
from workloads import gates as G
from workloads.rng import Xoshiro256ss, random_unitary

pytestmark = pytest.mark.gpu


def mixed_circuit(n, layers, theta, seed=3):
    """Per layer: RY, RZ per qubit; RX on even qubits; RZZ(q, q+3); XY(q, q+1)
    on every third q; CZ ladder; then a few fixed non-commuting gates."""
    rng = Xoshiro256ss(seed)
    circ = C.Circuit(n)
    p = 0

    def rot(qubits, gen):
        nonlocal p
        circ.append(qubits, G.pauli_rotation(gen, theta[p]), gen, p, gen)
        p += 1

    for layer in range(layers):
        for q in range(n):
            rot((q,), "Y")
            rot((q,), "Z")
        for q in range(0, n, 2):
            rot((q,), "X")
        for q in range(n - 3):
            rot((q, q + 3), "ZZ")
        for q in range(0, n - 1, 3):
            rot((q, q + 1), "XY")
        for q in range(n - 1):
            circ.append((q, q + 1), G.CZ, "cz")
        for _ in range(3):
            q = rng.randint(n)
            circ.append((q,), G.H if rng.randint(2) else G.SQRT_X, "fixed")
        a = rng.randint(n - 1)
        circ.append((a, a + 1), random_unitary(2, rng), "u2")
    circ.num_params = p
    return circ


def count_params(n, layers):
    return mixed_circuit(n, layers, np.zeros(100000)).num_params


_REF = {}


def _reference(n, layers, nsample):
    """theta, H terms, sampled parameters, their parameter-shift gradient and
    the energy (FP64 oracle), computed once for both dtypes."""
    key = (n, layers, nsample)
    if key not in _REF:
        P = count_params(n, layers)
        rng = Xoshiro256ss(100 + n)
        theta = np.array([rng.uniform_range(-np.pi, np.pi) for _ in range(P)])
        terms = C.ising_hamiltonian(n) + [C.PauliTerm(0.5, ((1, "Y"), (n - 2, "X"))),
                                          C.PauliTerm(0.3, ((0, "Z"), (9, "Y")))]
        build = lambda t: mixed_circuit(n, layers, t).gates
        sample = sorted({rng.randint(P) for _ in range(2 * nsample)})[:nsample]
        ps = oracle.parameter_shift_gradient(n, build, theta, terms, params=sample)
        _REF[key] = (theta, terms, sample, ps, oracle.energy(n, build, theta, terms))
    return _REF[key]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,layers,nsample", [(14, 3, 60), (17, 2, 24)])
def test_adjoint_mixed_circuit(qs, dtype, n, layers, nsample):
    theta, terms, sample, ps, e_ref = _reference(n, layers, nsample)
    spec = mixed_circuit(n, layers, theta)
    spec.theta = theta
    c = B.circuit_from(spec)
    h = B.PauliSum(n, terms)
    psi, lam = B.State(n, dtype), B.State(n, dtype)
    e, g = B.adjoint_gradient(c, theta, h, psi, lam)
    tol = 1e-4 if dtype == "c64" else 1e-10
    assert abs(e - e_ref) < tol * max(1.0, abs(e_ref))
    assert np.linalg.norm(g[sample] - ps) / np.linalg.norm(ps) < tol, np.max(np.abs(g[sample] - ps))


def test_adjoint_batch_matches_single_calls(qs):
    """qs_adjoint_gradient_batch: gradients of several circuits (different n,
    some sharing a stream) equal the single-call results; the small ones
    also match parameter shift."""
    import torch
    # several 12-14 qubit circuits at once: the same kernels launched from
    # concurrent host threads with different tile layouts and shared memory
    specs = [(8, 3), (10, 2), (12, 2), (13, 1), (14, 1), (9, 4)] + [(12 + i % 3, 6) for i in range(12)]
    streams = [torch.cuda.Stream() for _ in range(4)]
    circs, thetas, hams, psis, lams, refs = [], [], [], [], [], []
    for i, (n, layers) in enumerate(specs):
        theta = C.ansatz_theta(n, layers, seed=50 + i)
        circs.append(B.circuit_from(C.ansatz_circuit(n, layers, theta)))
        thetas.append(theta)
        hams.append(B.PauliSum(n, C.ising_hamiltonian(n)))
        st = streams[i % len(streams)]
        psis.append(B.State(n, "c64", stream=st))
        lams.append(B.State(n, "c64", stream=st, init=None))
    for c, t, h in zip(circs, thetas, hams):
        n = c.n
        refs.append(B.adjoint_gradient(c, t, h, B.State(n, "c64"), B.State(n, "c64", init=None)))
    energies, grads = B.adjoint_gradient_batch(circs, thetas, hams, psis, lams)
    for i, (e_ref, g_ref) in enumerate(refs):
        assert abs(energies[i] - e_ref) <= 1e-12 * max(1.0, abs(e_ref))
        assert np.array_equal(grads[i], g_ref), i
    for i in (0, 1):
        n, layers = specs[i]
        build = lambda t, n=n, layers=layers: C.ansatz_circuit(n, layers, t).gates
        ps = oracle.parameter_shift_gradient(n, build, thetas[i], C.ising_hamiltonian(n))
        assert np.linalg.norm(grads[i] - ps) / np.linalg.norm(ps) < 1e-4


def test_adjoint_batch_rejects_shared_objects(qs):
    n = 8
    theta = C.ansatz_theta(n, 2, seed=1)
    c = B.circuit_from(C.ansatz_circuit(n, 2, theta))
    h = B.PauliSum(n, C.ising_hamiltonian(n))
    s = [B.State(n, "c64") for _ in range(4)]
    with pytest.raises(B.QsError) as e:
        B.adjoint_gradient_batch([c, c], [theta, theta], [h, h], [s[0], s[1]], [s[2], s[3]])
    assert e.value.status == 1
    c2 = B.circuit_from(C.ansatz_circuit(n, 2, theta))
    with pytest.raises(B.QsError) as e:
        B.adjoint_gradient_batch([c, c2], [theta, theta], [h, h], [s[0], s[0]], [s[2], s[3]])
    assert e.value.status == 1
