"""The C/OpenMP form of the oracle's Section 3 update (oracle/sv_omp.c).

It is pinned by the same facts as the numpy oracle: every check in pins.py
runs with the C update in place of ``apply_gate`` (brute force against the
full unitary, Eq. 1, Eq. 2, closed forms, invariants, gradients).  It also
agrees with the numpy oracle on random circuits with gates of up to 6
qubits and on the grid circuit, gives bit-identical results for any thread
count (the sets are disjoint), and rejects bad gates."""

import numpy as np
import pytest

import oracle
import oracle.statevector as sv
import pins
from oracle import omp
from workloads import circuits as C
from workloads.rng import random_state


@pytest.fixture(scope="module", autouse=True)
def _built():
    omp.build()


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pins_hold_for_the_c_update(monkeypatch, check):
    monkeypatch.setattr(sv, "apply_gate", omp.apply_gate)
    monkeypatch.setattr(oracle, "apply_gate", omp.apply_gate)
    check()


@pytest.mark.parametrize("n,gates,k,seed", [(6, 40, 3, 1), (10, 60, 4, 2), (12, 30, 6, 3), (13, 80, 2, 4)])
def test_matches_numpy_oracle(n, gates, k, seed):
    circ = C.random_circuit(n, gates, seed, max_k=k)
    psi0 = random_state(n, seed + 10)
    a = oracle.simulate(n, circ.gates, psi0)
    b = omp.simulate(n, circ.gates, psi0)
    assert np.max(np.abs(a - b)) < 1e-13


def test_grid_circuit_matches_numpy_oracle():
    circ = C.scale_grid_circuit(16, 6, seed=2)
    a = oracle.simulate(16, circ.gates)
    b = omp.simulate(16, circ.gates)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-14


def test_thread_count_does_not_change_results():
    circ = C.random_circuit(12, 40, 7, max_k=4)
    before = omp.threads()
    try:
        omp.set_threads(1)
        a = omp.simulate(12, circ.gates)
        omp.set_threads(max(2, before))
        b = omp.simulate(12, circ.gates)
    finally:
        omp.set_threads(before)
    assert np.array_equal(a, b)


def test_rejects_bad_gates():
    psi = np.zeros(8, dtype=np.complex128)
    for qs in ((0, 0), (3,), (-1,)):
        with pytest.raises(ValueError):
            omp.apply_gate_inplace(psi, 3, qs, np.eye(1 << len(qs)))
    with pytest.raises(ValueError):
        omp.apply_gate_inplace(psi.astype(np.complex64), 3, (0,), np.eye(2))
