"""Checks that pin the FP64 oracle to facts outside itself.

Each ``check_*`` raises AssertionError on failure.  They are run as tests in
test_oracle_pins.py and, with a deliberately planted mistake in the oracle,
in test_oracle_mutations.py (which asserts that some check then fails).
None of them re-types the formula it checks: each compares against a
textbook routine (np.kron), an entry-by-entry construction, a closed form,
exact rational arithmetic or an invariant.
"""

from __future__ import annotations

import cmath
import math
from fractions import Fraction

import numpy as np

import oracle
from workloads import gates as G
from workloads.circuits import Circuit, PauliTerm, ising_hamiltonian, random_circuit
from workloads.rng import Xoshiro256ss, random_state, random_unitary


def _close(a, b, tol):
    a = np.asarray(a); b = np.asarray(b)
    err = np.max(np.abs(a - b)) if a.size else 0.0
    assert err <= tol, f"max deviation {err:.3e} > {tol:.1e}"


# ----------------------------------------------------------------- conventions
def check_basis_convention():
    """Qubit q <-> index bit q: X on qubit q maps |0..0> to index 2^q; CNOT
    with control = qubits[0] (Section 2's matrix, first qubit most
    significant) maps index 2^c to 2^c + 2^t."""
    n = 5
    for q in range(n):
        psi = oracle.simulate(n, [((q,), G.X)])
        assert abs(psi[1 << q] - 1) < 1e-15 and abs(oracle.norm_sq(psi) - 1) < 1e-15
    for c, t in [(0, 3), (4, 1), (2, 3)]:
        psi = oracle.simulate(n, [((c, t), G.CNOT)], oracle.basis_state(n, 1 << c))
        assert abs(psi[(1 << c) | (1 << t)] - 1) < 1e-15
        psi = oracle.simulate(n, [((c, t), G.CNOT)], oracle.basis_state(n, 1 << t))
        assert abs(psi[1 << t] - 1) < 1e-15


def check_eq1_cz():
    """Eq. 1: (I (x) H) CNOT (I (x) H) = CZ, as matrices and as circuits."""
    lhs = np.kron(G.I2, G.H) @ G.CNOT @ np.kron(G.I2, G.H)
    _close(lhs, G.CZ, 1e-15)
    n = 5
    psi0 = random_state(n, 7)
    for c, t in [(0, 1), (3, 1), (4, 0)]:
        a = oracle.simulate(n, [((t,), G.H), ((c, t), G.CNOT), ((t,), G.H)], psi0)
        b = oracle.simulate(n, [((c, t), G.CZ)], psi0)
        _close(a, b, 1e-14)


# ----------------------------------------------------------------- brute force
def check_unitary_builder_vs_kron():
    """The entry-by-entry padded operator equals np.kron padding for gates on
    adjacent qubits listed most-significant first."""
    rng = Xoshiro256ss(3)
    n = 6
    for q in range(n):
        m = random_unitary(1, rng)
        _close(oracle.gate_unitary(n, (q,), m),
               np.kron(np.kron(np.eye(1 << (n - q - 1)), m), np.eye(1 << q)), 1e-15)
    for q in range(n - 2):
        m = random_unitary(2, rng)
        _close(oracle.gate_unitary(n, (q + 1, q), m),
               np.kron(np.kron(np.eye(1 << (n - q - 2)), m), np.eye(1 << q)), 1e-15)
    m = random_unitary(3, rng)
    _close(oracle.gate_unitary(n, (4, 3, 2), m),
           np.kron(np.kron(np.eye(2), m), np.eye(4)), 1e-15)


def check_brute_force(n=7, num_gates=24, seed=11, max_k=3):
    """Gate-by-gate simulation equals the full 2^n x 2^n unitary applied to
    the initial state (Section 3's padded evaluation), on random circuits
    with dense, diagonal and monomial gates on arbitrary qubit subsets."""
    circ = random_circuit(n, num_gates, seed, max_k=max_k)
    psi0 = random_state(n, seed + 100)
    a = oracle.simulate(n, circ.gates, psi0)
    b = oracle.full_unitary(n, circ.gates) @ psi0
    _close(a, b, 1e-13)


def check_kron_coalescing():
    """Eq. 2 generalised: a gate kron(A, B) on (a, b) equals A on a then B
    on b; in particular (sqrtY (x) sqrtY)(H (x) H) = sqrtY H (x) sqrtY H."""
    rng = Xoshiro256ss(5)
    n = 6
    psi0 = random_state(n, 9)
    for a, b in [(0, 1), (5, 2), (3, 4)]:
        A = random_unitary(1, rng); B = random_unitary(1, rng)
        x = oracle.simulate(n, [((a, b), np.kron(A, B))], psi0)
        y = oracle.simulate(n, [((a,), A), ((b,), B)], psi0)
        _close(x, y, 1e-14)
    lhs = np.kron(G.SQRT_Y, G.SQRT_Y) @ np.kron(G.H, G.H)
    _close(lhs, np.kron(G.SQRT_Y @ G.H, G.SQRT_Y @ G.H), 1e-15)
    A = random_unitary(2, rng); B = random_unitary(1, rng)
    x = oracle.simulate(n, [((4, 0, 2), np.kron(A, B))], psi0)
    y = oracle.simulate(n, [((4, 0), A), ((2,), B)], psi0)
    _close(x, y, 1e-14)


# ----------------------------------------------------------------- closed forms
def check_h_layer_uniform():
    """H on every qubit of |0..0> gives 2^(-n/2) everywhere (the initial H
    layer that Section 4.5 replaces by uniform initialisation)."""
    for n in range(1, 13):
        psi = oracle.simulate(n, [((q,), G.H) for q in range(n)])
        _close(psi, np.full(1 << n, 2.0 ** (-n / 2)), 1e-14)


def check_ghz():
    for n in (2, 5, 9):
        gs = [((0,), G.H)] + [((q, q + 1), G.CNOT) for q in range(n - 1)]
        psi = oracle.simulate(n, gs)
        ref = np.zeros(1 << n, dtype=complex)
        ref[0] = ref[-1] = 1 / math.sqrt(2)
        _close(psi, ref, 1e-15)


def qft_gates(n):
    """Textbook QFT circuit (most significant qubit first, then reversal)."""
    gs = []
    for j in range(n - 1, -1, -1):
        gs.append(((j,), G.H))
        for m in range(j - 1, -1, -1):
            gs.append(((j, m), G.cphase(math.pi / (1 << (j - m)))))
    for i in range(n // 2):
        gs.append(((i, n - 1 - i), G.SWAP))
    return gs


def check_qft_basis():
    """QFT|x> = 2^(-n/2) sum_y exp(2 pi i x y / 2^n) |y> (QFT: Section 4.3)."""
    for n in (3, 6, 8):
        dim = 1 << n
        for x in (0, 1, 5 % dim, dim - 1, (dim // 3) | 1):
            psi = oracle.simulate(n, qft_gates(n), oracle.basis_state(n, x))
            ref = np.array([cmath.exp(2j * math.pi * x * y / dim) for y in range(dim)]) / math.sqrt(dim)
            _close(psi, ref, 1e-13)


# ----------------------------------------------------------------- invariants
def check_norm_preserved():
    for seed in range(3):
        circ = random_circuit(8, 40, seed + 20, max_k=4)
        psi = oracle.simulate(8, circ.gates, random_state(8, seed))
        assert abs(oracle.norm_sq(psi) - 1.0) < 1e-13


def check_norm_exact():
    """norm_sq against exact rational arithmetic on the same FP64 inputs."""
    cases = [random_state(10, 40 + seed) * (0.7317 + 0.123 * seed) for seed in range(3)]
    # one large amplitude and many tiny ones: a running FP64 sum drops the
    # tiny contributions (the failure mode Section 4.1 warns about)
    spread = np.full(1 << 10, 1e-9 + 3e-10j)
    spread[17] = 1.0
    cases.append(spread)
    for psi in cases:
        exact = sum(Fraction(float(v.real)) ** 2 + Fraction(float(v.imag)) ** 2 for v in psi)
        got = Fraction(oracle.norm_sq(psi))
        assert abs(got - exact) <= Fraction(2.0 ** -51) * exact, float(abs(got - exact) / exact)


def _is_diag(m):
    return np.count_nonzero(m - np.diag(np.diagonal(m))) == 0


def _commute(g1, g2):
    return not (set(g1.qubits) & set(g2.qubits)) or (_is_diag(g1.matrix) and _is_diag(g2.matrix))


def check_reorder_invariance():
    """Reordering commuting gates (disjoint support, or both diagonal:
    Sections 4.2 and 4.5) leaves the output unchanged."""
    for seed in range(3):
        n = 7
        circ = random_circuit(n, 60, seed + 30, max_k=3)
        gates = list(circ.gates)
        rng = Xoshiro256ss(seed + 99)
        for _ in range(400):
            i = rng.randint(len(gates) - 1)
            if _commute(gates[i], gates[i + 1]):
                gates[i], gates[i + 1] = gates[i + 1], gates[i]
        assert any(a is not b for a, b in zip(gates, circ.gates))
        psi0 = random_state(n, seed)
        _close(oracle.simulate(n, gates, psi0), oracle.simulate(n, circ.gates, psi0), 1e-13)


# ----------------------------------------------------------------- gate library
def check_gate_constants():
    for m in (G.H, G.SQRT_X, G.SQRT_Y, G.SQRT_W, G.T, G.S, G.fsim(0.3, 1.1), G.CNOT, G.CZ):
        _close(m.conj().T @ m, np.eye(m.shape[0]), 1e-15)
    T8 = np.linalg.matrix_power(G.T, 8)
    _close(T8, G.I2, 1e-15)                                   # T^8 = I (Section 4.3)
    _close(G.T @ G.T, G.S, 1e-15)                             # P = T^2
    _close(np.linalg.matrix_power(G.T, 4), G.Z, 1e-15)        # Z = T^4
    _close(G.H @ G.S @ G.H, G.SQRT_X, 1e-15)                  # X^(1/2) = H P H (Section 2)
    _close(G.SQRT_X @ G.SQRT_X, G.X, 1e-15)
    _close(G.SQRT_Y @ G.SQRT_Y, G.Y, 1e-15)
    _close(G.SQRT_W @ G.SQRT_W, G.W, 1e-15)
    _close(G.sqrt_involution(G.W), G.SQRT_W, 1e-15)
    # the sqrt(Y) printed in Section 2 squares to -Y: the reading used here
    # replaces it by the principal root, which squares to +Y
    printed = 0.5 * np.array([[1 + 1j, 1 + 1j], [-1 - 1j, 1 + 1j]])
    _close(printed @ printed, -G.Y, 1e-15)
    _close(G.fsim(0.0, math.pi), G.CZ, 1e-15)
    iswap_dag = np.array([[1, 0, 0, 0], [0, 0, -1j, 0], [0, -1j, 0, 0], [0, 0, 0, 1]])
    _close(G.fsim(math.pi / 2, 0.0), iswap_dag, 1e-15)


# ----------------------------------------------------------------- expectation & gradients
def _product_circuit(n, a, b):
    gs = []
    for q in range(n):
        gs.append(((q,), G.ry(a[q])))
        gs.append(((q,), G.rz(b[q])))
    return gs


def _ising_product_energy(a, b):
    """Closed form for the Ising H on the product state (x)_q RZ(b_q)RY(a_q)|0>:
    <Z_q> = cos a_q, <X_q> = sin a_q cos b_q, <Z_q Z_q+1> = cos a_q cos a_q+1."""
    n = len(a)
    return sum(math.cos(a[i]) * math.cos(a[i + 1]) for i in range(n - 1)) + \
        sum(math.sin(a[i]) * math.cos(b[i]) for i in range(n))


def check_expectation_closed_forms():
    for n in (1, 2, 6):
        H = ising_hamiltonian(n)
        assert abs(oracle.expectation(oracle.zero_state(n), n, H) - (n - 1)) < 1e-14
        plus = oracle.simulate(n, [((q,), G.H) for q in range(n)])
        assert abs(oracle.expectation(plus, n, H) - n) < 1e-13
        rng = Xoshiro256ss(n)
        a = [rng.uniform_range(-3, 3) for _ in range(n)]
        b = [rng.uniform_range(-3, 3) for _ in range(n)]
        psi = oracle.simulate(n, _product_circuit(n, a, b))
        assert abs(oracle.expectation(psi, n, H) - _ising_product_energy(a, b)) < 1e-13
    # a Y term: <Y> on RZ(b)RY(a)|0> is sin a sin b
    a, b = 0.7, -1.3
    psi = oracle.simulate(1, _product_circuit(1, [a], [b]))
    e = oracle.expectation(psi, 1, [PauliTerm(2.0, ((0, "Y"),))])
    assert abs(e - 2 * math.sin(a) * math.sin(b)) < 1e-14


def _product_build(n):
    def build(theta):
        return _product_circuit(n, theta[0::2], theta[1::2])
    return build


def _product_grad(a, b):
    n = len(a)
    g = np.zeros(2 * n)
    for i in range(n):
        nb = (math.cos(a[i - 1]) if i > 0 else 0.0) + (math.cos(a[i + 1]) if i < n - 1 else 0.0)
        g[2 * i] = -math.sin(a[i]) * nb + math.cos(a[i]) * math.cos(b[i])
        g[2 * i + 1] = -math.sin(a[i]) * math.sin(b[i])
    return g


def check_gradients_closed_form():
    """Parameter shift is exact and central differences are O(h^2) close,
    against the analytic derivative of the product-state energy."""
    for n in (1, 4):
        rng = Xoshiro256ss(50 + n)
        theta = np.array([rng.uniform_range(-math.pi, math.pi) for _ in range(2 * n)])
        ref = _product_grad(theta[0::2], theta[1::2])
        H = ising_hamiltonian(n)
        ps = oracle.parameter_shift_gradient(n, _product_build(n), theta, H)
        _close(ps, ref, 1e-13)
        fd = oracle.central_fd_gradient(n, _product_build(n), theta, H, h=1e-4)
        _close(fd, ref, 1e-7)



# ----------------------------------------------------------------- Pauli sums
def _pauli_sum_dense(n, terms):
    """sum_t c_t P_t as a 2^n x 2^n matrix built with np.kron from the
    textbook Pauli matrices of the gate library (qubit q is index bit q, so
    it is the (n-1-q)-th factor of the Kronecker product)."""
    mats = {"X": G.X, "Y": G.Y, "Z": G.Z}
    h = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for t in terms:
        ops = dict(t.ops)
        m = np.ones((1, 1), dtype=np.complex128)
        for q in range(n - 1, -1, -1):
            m = np.kron(m, mats[ops[q]] if q in ops else G.I2)
        h += t.coeff * m
    return h


def _random_terms(n, count, rng):
    terms = []
    for _ in range(count):
        length = 1 + rng.randint(min(n, 3))
        qs = []
        while len(qs) < length:
            q = rng.randint(n)
            if q not in qs:
                qs.append(q)
        ops = tuple((q, "XYZ"[rng.randint(3)]) for q in qs)
        terms.append(PauliTerm(rng.uniform_range(-2.0, 2.0), ops))
    return terms


def check_pauli_sum_dense():
    """H psi equals the np.kron-built matrix of the Pauli sum times psi, on
    basis states (each column of H) and random states; <psi|H psi> is the
    expectation."""
    rng = Xoshiro256ss(61)
    for n in (1, 3, 6, 8):
        terms = _random_terms(n, 2 + 2 * n, rng)
        terms.append(PauliTerm(0.75, ((n - 1, "Y"),)))    # a Y on the top qubit in every case
        h = _pauli_sum_dense(n, terms)
        for j in (0, 1, (1 << n) - 1, (5 * n) % (1 << n)):
            _close(oracle.apply_pauli_sum(oracle.basis_state(n, j), n, terms), h[:, j], 1e-14)
        psi = random_state(n, 70 + n)
        hpsi = oracle.apply_pauli_sum(psi, n, terms)
        _close(hpsi, h @ psi, 1e-13)
        assert abs(np.vdot(psi, hpsi).real - oracle.expectation(psi, n, terms)) < 1e-13
        assert abs(np.vdot(psi, h @ psi).imag) < 1e-13          # Hermitian: a real expectation


# ----------------------------------------------------------------- error measures
def check_error_metrics():
    """Relative L2, max |dp| and total variation on vectors worked by hand:
    psi = (1, 0) against ref = (0.6, 0.8): d = (0.4, -0.8), |d| = sqrt(0.8);
    p = (1, 0), p_ref = (0.36, 0.64): max |dp| = 0.64, TV = (0.64 + 0.64)/2.
    A relative phase changes the amplitudes (relative L2 = 1 below) but no
    probability (max |dp| = TV = 0)."""
    from oracle import metrics as M
    psi, ref = np.array([1.0, 0.0]), np.array([0.6, 0.8])
    assert abs(M.rel_l2(psi, ref) - math.sqrt(0.8)) < 1e-15
    assert abs(M.max_prob_error(psi, ref) - 0.64) < 1e-15
    assert abs(M.tv_distance(psi, ref) - 0.64) < 1e-15
    s = 1 / math.sqrt(2)
    psi, ref = np.array([1j * s, s]), np.array([s, s])
    assert abs(M.rel_l2(psi, ref) - 1.0) < 1e-15
    assert M.max_prob_error(psi, ref) < 1e-16 and M.tv_distance(psi, ref) < 1e-16
    # three outcomes, two of them moved: TV is half the summed moves, max the largest
    psi = np.array([math.sqrt(0.5), math.sqrt(0.3), math.sqrt(0.2)])
    ref = np.array([math.sqrt(0.4), math.sqrt(0.3), math.sqrt(0.3)])
    assert abs(M.max_prob_error(psi, ref) - 0.1) < 1e-15
    assert abs(M.tv_distance(psi, ref) - 0.1) < 1e-15
    psi = np.array([math.sqrt(0.7), math.sqrt(0.1), math.sqrt(0.2)])
    assert abs(M.max_prob_error(psi, ref) - 0.3) < 1e-15
    assert abs(M.tv_distance(psi, ref) - 0.3) < 1e-15         # (0.3 + 0.2 + 0.1) / 2
    # the same pair swapped: the largest move is now a decrease (-0.3)
    assert abs(M.max_prob_error(ref, psi) - 0.3) < 1e-15
    assert abs(M.tv_distance(ref, psi) - 0.3) < 1e-15
    assert abs(M.rel_l2_vec(np.array([3.0, 4.0]), np.array([0.0, 5.0])) - math.sqrt(10) / 5) < 1e-15

ALL_CHECKS = [
    check_basis_convention, check_eq1_cz, check_unitary_builder_vs_kron, check_brute_force,
    check_kron_coalescing, check_h_layer_uniform, check_ghz, check_qft_basis,
    check_norm_preserved, check_norm_exact, check_reorder_invariance, check_gate_constants,
    check_expectation_closed_forms, check_gradients_closed_form, check_pauli_sum_dense, check_error_metrics,
]
