"""Plant plausible mistakes in the oracle (on the CPU, by monkeypatching)
and check that at least one pin catches each of them."""

import numpy as np
import pytest

import oracle
import oracle.metrics as metrics
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


def _pauli_sum_overwrite(psi, n, terms):
    """= in place of += over the terms: only the last term survives"""
    out = np.zeros_like(psi)
    for t in terms:
        out = t.coeff * sv.apply_pauli_string(psi, n, t.ops)
    return out


def _pauli_sum_conj_strings(psi, n, terms):
    """each Pauli string conjugated (Y -> -Y)"""
    out = np.zeros_like(psi)
    for t in terms:
        out += t.coeff * np.conj(sv.apply_pauli_string(np.conj(psi), n, t.ops))
    return out


def _pauli_sum_no_coeff(psi, n, terms):
    out = np.zeros_like(psi)
    for t in terms:
        out += sv.apply_pauli_string(psi, n, t.ops)
    return out


def _pauli_sum_reversed_qubits(psi, n, terms):
    out = np.zeros_like(psi)
    for t in terms:
        out += t.coeff * sv.apply_pauli_string(psi, n, tuple((n - 1 - q, p) for q, p in t.ops))
    return out


def _maxp_on_amplitudes(psi, ref):
    return float(np.max(np.abs(np.abs(psi) - np.abs(ref))))


def _maxp_no_abs(psi, ref):
    return float(np.max(np.abs(psi) ** 2 - np.abs(ref) ** 2))


def _tv_no_half(psi, ref):
    return float(np.sum(np.abs(np.abs(psi) ** 2 - np.abs(ref) ** 2)))


def _tv_signed(psi, ref):
    return float(0.5 * abs(np.sum(np.abs(psi) ** 2 - np.abs(ref) ** 2)))


def _rel_l2_phase_blind(psi, ref):
    return float(np.linalg.norm(np.abs(psi) - np.abs(ref)) / np.linalg.norm(ref))


MUTATIONS = [
    (sv, "apply_gate", _transposed),
    (sv, "apply_gate", _reversed_qubits),
    (sv, "apply_gate", _conjugated),
    (sv, "apply_gate", _off_by_one_qubit),
    (sv, "norm_sq", _norm_float32),
    (sv, "expectation", _expect_no_conj),
    (sv, "parameter_shift_gradient", _ps_wrong_sign),
    (sv, "apply_pauli_sum", _pauli_sum_overwrite),
    (sv, "apply_pauli_sum", _pauli_sum_conj_strings),
    (sv, "apply_pauli_sum", _pauli_sum_no_coeff),
    (sv, "apply_pauli_sum", _pauli_sum_reversed_qubits),
    (metrics, "max_prob_error", _maxp_on_amplitudes),
    (metrics, "max_prob_error", _maxp_no_abs),
    (metrics, "tv_distance", _tv_no_half),
    (metrics, "tv_distance", _tv_signed),
    (metrics, "rel_l2", _rel_l2_phase_blind),
]


@pytest.mark.parametrize("mod,name,fn", MUTATIONS, ids=lambda x: getattr(x, "__name__", str(x)))
def test_mutation_is_caught(monkeypatch, mod, name, fn):
    monkeypatch.setattr(mod, name, fn)
    if hasattr(oracle, name):
        monkeypatch.setattr(oracle, name, fn)
    failures = 0
    for check in pins.ALL_CHECKS:
        try:
            check()
        except AssertionError:
            failures += 1
    assert failures > 0, f"no pin caught the planted mistake in {name}"
