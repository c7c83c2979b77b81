"""Plant plausible mistakes in the oracle (on the CPU, by monkeypatching)
and check that at least one pin catches each of them."""

import numpy as np
import pytest

import oracle
import oracle.statevector as sv
import pins

_orig_apply = sv.apply_gate


def _transposed(psi, n, qubits, m):
    return _orig_apply(psi, n, qubits, np.asarray(m).T)


def _reversed_qubits(psi, n, qubits, m):
    return _orig_apply(psi, n, tuple(qubits)[::-1], m)


def _conjugated(psi, n, qubits, m):
    return _orig_apply(psi, n, qubits, np.conj(m))


def _off_by_one_qubit(psi, n, qubits, m):
    return _orig_apply(psi, n, tuple((q + 1) % n for q in qubits), m)


def _norm_float32(psi):
    a = np.asarray(psi, dtype=np.complex64)
    return float(np.sum((a.real * a.real + a.imag * a.imag).astype(np.float32)))


_orig_expect = sv.expectation


def _expect_no_conj(psi, n, terms):
    total = 0.0
    for t in terms:
        total += t.coeff * np.dot(psi, sv.apply_pauli_string(psi, n, t.ops)).real
    return float(total)


_orig_ps = sv.parameter_shift_gradient


def _ps_wrong_sign(n, build, theta, terms, params=None):
    return -_orig_ps(n, build, theta, terms, params)


MUTATIONS = [
    ("apply_gate", _transposed),
    ("apply_gate", _reversed_qubits),
    ("apply_gate", _conjugated),
    ("apply_gate", _off_by_one_qubit),
    ("norm_sq", _norm_float32),
    ("expectation", _expect_no_conj),
    ("parameter_shift_gradient", _ps_wrong_sign),
]


@pytest.mark.parametrize("name,fn", MUTATIONS, ids=lambda x: getattr(x, "__name__", str(x)))
def test_mutation_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(sv, name, fn)
    monkeypatch.setattr(oracle, name, fn)
    failures = 0
    for check in pins.ALL_CHECKS:
        try:
            check()
        except AssertionError:
            failures += 1
    assert failures > 0, f"no pin caught the planted mistake in {name}"
