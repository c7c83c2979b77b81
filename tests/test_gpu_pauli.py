"""Pauli sums on the GPU (tile passes that each read psi once) against the
FP64 oracle: H psi and <psi|H|psi> for Hamiltonians that need several
passes, flip masks wider than a tile (partners read from global memory),
a diagonal group larger than one pass holds, Z terms across 8-qubit chunks,
and Y / Z mixtures on flipped qubits."""

import numpy as np
import pytest

import oracle
from oracle.metrics import rel_l2
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C
from workloads.rng import Xoshiro256ss, random_state
from gpu_util import to_state

pytestmark = pytest.mark.gpu


def hamiltonian(n, seed):
    rng = Xoshiro256ss(seed)
    terms = C.ising_hamiltonian(n)
    for _ in range(100):  # diagonal terms: more than one pass holds
        a, b = rng.randint(n), rng.randint(n)
        ops = ((a, "Z"),) if a == b else ((a, "Z"), (b, "Z"))
        terms.append(C.PauliTerm(rng.uniform_range(-1, 1), ops))
    for _ in range(40):  # random strings on 1-4 qubits
        qs = sorted({rng.randint(n) for _ in range(1 + rng.randint(4))})
        terms.append(C.PauliTerm(rng.uniform_range(-1, 1), tuple((q, "XYZ"[rng.randint(3)]) for q in qs)))
    # a flip over many high qubits (wider than a tile)
    terms.append(C.PauliTerm(0.3, tuple((q, "X" if q % 2 else "Y") for q in range(5, n))))
    terms.append(C.PauliTerm(-0.2, ((0, "Z"), (n - 1, "Y"), (n - 2, "X"))))
    return terms


_REF = {}


def _reference(n):
    """(terms, psi, <psi|H|psi>, H psi) from the FP64 oracle, once per n."""
    if n not in _REF:
        terms = hamiltonian(n, 40 + n)
        psi0 = random_state(n, 9 + n)
        _REF[n] = (terms, psi0, oracle.expectation(psi0, n, terms), oracle.apply_pauli_sum(psi0, n, terms))
    return _REF[n]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [12, 17, 20])
def test_pauli_sum_tiled(qs, dtype, n):
    terms, psi0, ref, hp = _reference(n)
    h = B.PauliSum(n, terms)
    s = to_state(psi0, n, dtype)
    tol = 2e-5 if dtype == "c64" else 1e-12
    got = B.expectation(s, h)
    assert abs(got - ref) < tol * max(1.0, abs(ref)), (got, ref)
    out = to_state(np.zeros(1 << n), n, dtype)
    B.apply_pauli_sum(s, h, out)
    assert rel_l2(out.amplitudes(), hp) < (2e-6 if dtype == "c64" else 1e-13)


def test_pauli_sum_empty_and_identity(qs):
    n = 14
    psi0 = random_state(n, 2)
    s = to_state(psi0, n, "c128")
    out = to_state(np.ones(1 << n), n, "c128")
    B.apply_pauli_sum(s, B.PauliSum(n, []), out)
    assert np.all(out.amplitudes() == 0)
    assert B.expectation(s, B.PauliSum(n, [])) == 0.0
    h = B.PauliSum(n, [C.PauliTerm(1.5, ())])
    B.apply_pauli_sum(s, h, out)
    assert rel_l2(out.amplitudes(), 1.5 * psi0) < 1e-15
    assert abs(B.expectation(s, h) - 1.5 * np.vdot(psi0, psi0).real) < 1e-12


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9, 11])
def test_pauli_sum_small_states(qs, dtype, n):
    """Tiles smaller than a full pass tile (down to one qubit): every term
    kind, against the oracle."""
    rng = Xoshiro256ss(300 + n)
    terms = [C.PauliTerm(0.7, ())]
    for _ in range(12):
        qs_ = sorted({rng.randint(n) for _ in range(1 + rng.randint(3))})
        terms.append(C.PauliTerm(rng.uniform_range(-1, 1), tuple((q, "XYZ"[rng.randint(3)]) for q in qs_)))
    psi0 = random_state(n, 40 + n)
    h = B.PauliSum(n, terms)
    s = to_state(psi0, n, dtype)
    ref = oracle.expectation(psi0, n, terms)
    tol = 2e-5 if dtype == "c64" else 1e-12
    assert abs(B.expectation(s, h) - ref) < tol * max(1.0, abs(ref))
    out = to_state(np.zeros(1 << n), n, dtype)
    B.apply_pauli_sum(s, h, out)
    assert rel_l2(out.amplitudes(), oracle.apply_pauli_sum(psi0, n, terms)) < (2e-6 if dtype == "c64" else 1e-13)
