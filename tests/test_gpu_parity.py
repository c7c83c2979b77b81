"""CUDA path against the FP64 oracle, element by element, on seeded inputs.

Sizes are ones the oracle finishes in seconds, spanning several shared-memory
tiles (2^12 / 2^11 amplitudes) and odd qubit counts (ragged tile grids).
Tolerances: relative L2 1e-12 for complex128, 2e-5 for complex64."""

import math

import numpy as np
import pytest

import oracle
from oracle.metrics import rel_l2
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C
from workloads import gates as G
from workloads.rng import Xoshiro256ss, random_state, random_unitary

from gpu_util import TOL, run_gates, run_plan, to_state

pytestmark = pytest.mark.gpu

DTYPES = ["c64", "c128"]


def _positions(n, k):
    """Qubit lists covering low, high, scattered and reversed placements."""
    low = list(range(k))
    high = list(range(n - k, n))
    scat = [((2 * i + 1) * n) // (2 * k) for i in range(k)]
    out = [low, high[::-1], scat]
    if k >= 2:
        out.append([0, n - 1] + list(range(2, k)))
    return [p for p in out if len(set(p)) == k]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_single_dense_gate(qs, dtype, k):
    n = 13
    rng = Xoshiro256ss(100 + k)
    psi0 = random_state(n, k)
    for qubits in _positions(n, k):
        m = random_unitary(k, rng)
        ref = oracle.apply_gate(psi0, n, qubits, m)
        got = run_gates(n, [(qubits, m)], dtype, psi0)
        assert rel_l2(got, ref) < (1e-6 if dtype == "c64" else 1e-14), (qubits, rel_l2(got, ref))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_single_diagonal_and_monomial_gate(qs, dtype, k):
    n = 12
    psi0 = random_state(n, 30 + k)
    circ = C.random_circuit(n, 12, seed=40 + k, max_k=k, kinds=("diag", "monomial"))
    for g in circ.gates:
        ref = oracle.apply_gate(psi0, n, g.qubits, g.matrix)
        got = run_gates(n, [g], dtype, psi0)
        assert rel_l2(got, ref) < (1e-6 if dtype == "c64" else 1e-14), g.qubits


@pytest.mark.parametrize("dtype", DTYPES)
def test_multiply_free_phases(qs, dtype):
    """+-1 / +-i phases (Z, S, CZ, iSWAP-like) take the multiply-free path."""
    n = 11
    psi0 = random_state(n, 5)
    iswap = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]])
    gates = [((3,), G.Z), ((0,), G.S), ((9, 2), G.CZ), ((1, 7), iswap), ((10,), G.X), ((0, 5), G.SWAP)]
    ref = oracle.simulate(n, gates, psi0)
    got = run_gates(n, gates, dtype, psi0)
    assert rel_l2(got, ref) < (1e-7 if dtype == "c64" else 1e-15)


def test_small_grid_circuit_unfused_c128(qs):
    """12 qubits, 3x4 grid, 8 cycles, fSim(pi/2, pi/6): unfused, complex128,
    the whole 4096-amplitude state against the oracle."""
    circ = C.small_grid_circuit(seed=1)
    ref = oracle.simulate(12, circ.gates)
    got, info = run_plan(circ, "c128", fuse=False, use_tile=False)
    assert info["passes"] == len(circ.gates)
    assert rel_l2(got, ref) < 1e-12
    got2 = run_gates(12, circ.gates, "c128")
    assert rel_l2(got2, ref) < 1e-12


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("k_max", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("use_tile", [False, True])
def test_grid_circuit_fused(qs, dtype, k_max, use_tile):
    """The scale-generator (patterns ABCDCDAB, random fSim) at 17 qubits."""
    n = 17
    circ = C.scale_grid_circuit(n, 10, seed=2)
    ref = oracle.simulate(n, circ.gates)
    got, info = run_plan(circ, dtype, k_max=k_max, use_tile=use_tile)
    assert rel_l2(got, ref) < TOL[dtype], info


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [6, 9, 12, 14])
def test_tile_pass_sizes(qs, dtype, n):
    """Tiles larger than, equal to and smaller than the state."""
    circ = C.random_circuit(n, 60, seed=n, max_k=3)
    psi0 = random_state(n, n + 1)
    ref = oracle.simulate(n, circ.gates, psi0)
    for L in (6, 8, 11):
        got, info = run_plan(circ, dtype, psi0=psi0, k_max=3, use_tile=True, tile_qubits=L)
        assert rel_l2(got, ref) < TOL[dtype], (L, info)


@pytest.mark.parametrize("dtype", DTYPES)
def test_random_circuits_all_kinds(qs, dtype):
    for seed in range(3):
        n = 15
        circ = C.random_circuit(n, 80, seed=200 + seed, max_k=4)
        psi0 = random_state(n, seed)
        ref = oracle.simulate(n, circ.gates, psi0)
        for k_max in (2, 4, 6):
            got, info = run_plan(circ, dtype, psi0=psi0, k_max=k_max)
            assert rel_l2(got, ref) < TOL[dtype], (seed, k_max, info)


@pytest.mark.parametrize("dtype", DTYPES)
def test_norm(qs, dtype):
    for n in (1, 2, 7, 16):
        psi0 = random_state(n, n) * 1.37
        s = to_state(psi0, n, dtype)
        ref = oracle.norm_sq(psi0.astype(np.complex64) if dtype == "c64" else psi0)
        assert abs(s.norm() - ref) <= 1e-13 * ref
        s.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_expectation_and_h_apply(qs, dtype):
    n = 12
    psi0 = random_state(n, 3)
    terms = C.ising_hamiltonian(n) + [C.PauliTerm(0.5, ((1, "Y"), (4, "X"))), C.PauliTerm(-0.25, ((2, "Y"),)),
                                      C.PauliTerm(0.75, ((0, "Z"), (3, "Y"), (11, "Y")))]
    h = B.PauliSum(n, terms)
    s = to_state(psi0, n, dtype)
    ref = oracle.expectation(psi0, n, terms)
    tol = 1e-5 if dtype == "c64" else 1e-12
    assert abs(B.expectation(s, h) - ref) < tol * max(1.0, abs(ref))
    out = to_state(np.zeros(1 << n), n, dtype)
    B.apply_pauli_sum(s, h, out)
    assert rel_l2(out.amplitudes(), oracle.apply_pauli_sum(psi0, n, terms)) < (1e-6 if dtype == "c64" else 1e-13)


@pytest.mark.parametrize("dtype", DTYPES)
def test_adjoint_gradient_vs_parameter_shift(qs, dtype):
    n, layers = 6, 3
    theta = C.ansatz_theta(n, layers, seed=5)
    spec = C.ansatz_circuit(n, layers, theta)
    terms = C.ising_hamiltonian(n)
    build = lambda t: C.ansatz_circuit(n, layers, t).gates
    ps = oracle.parameter_shift_gradient(n, build, theta, terms)
    e_ref = oracle.energy(n, build, theta, terms)
    c = B.circuit_from(spec)
    h = B.PauliSum(n, terms)
    psi, lam = B.State(n, dtype), B.State(n, dtype)
    e, g = B.adjoint_gradient(c, theta, h, psi, lam)
    tol = 1e-4 if dtype == "c64" else 1e-10
    assert abs(e - e_ref) < tol
    assert np.linalg.norm(g - ps) / np.linalg.norm(ps) < tol


def test_init_uniform_and_basis(qs):
    for n in (1, 5, 12):
        for dtype in DTYPES:
            s = B.State(n, dtype, init="uniform")
            assert np.max(np.abs(s.amplitudes() - 2.0 ** (-n / 2))) < (1e-7 if dtype == "c64" else 1e-16)
            s.init_basis((1 << n) - 1)
            a = s.amplitudes()
            assert a[-1] == 1 and np.count_nonzero(a) == 1
            s.close()


def test_bad_arguments_return_status(qs):
    s = B.State(5, "c64")
    with pytest.raises(B.QsError) as e:
        B.apply_gate(s, [5], np.eye(2))
    assert e.value.status == 1
    with pytest.raises(B.QsError):
        B.apply_gate(s, [1, 1], np.eye(4))
    with pytest.raises(B.QsError):
        s.amplitudes(30, 5)
    c = B.circuit_from(C.small_grid_circuit())
    p = B.Plan(c, "c64")
    with pytest.raises(B.QsError):
        p.execute(s)   # plan for 12 qubits on a 5-qubit state
    s.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_adjoint_gradient_12q_20_layers_sampled(qs, dtype):
    """The differentiation workload's check size: 12 qubits, 20 layers (480
    parameters).  The adjoint gradient against exact parameter shift on a
    seeded sample of 48 parameters, and against central differences (h=1e-4,
    FP64 oracle) on 6 of them; energy against the oracle."""
    n, layers = 12, 20
    theta = C.ansatz_theta(n, layers, seed=1)
    terms = C.ising_hamiltonian(n)
    build = lambda t: C.ansatz_circuit(n, layers, t).gates
    rng = Xoshiro256ss(12)
    sample = sorted({rng.randint(theta.size) for _ in range(60)})[:48]
    ps = oracle.parameter_shift_gradient(n, build, theta, terms, params=sample)
    fd = oracle.central_fd_gradient(n, build, theta, terms, h=1e-4, params=sample[:6])
    c = B.circuit_from(C.ansatz_circuit(n, layers, theta))
    h = B.PauliSum(n, terms)
    psi, lam = B.State(n, dtype), B.State(n, dtype)
    e, g = B.adjoint_gradient(c, theta, h, psi, lam)
    tol = 1e-4 if dtype == "c64" else 1e-10
    assert abs(e - oracle.energy(n, build, theta, terms)) < tol * max(1.0, abs(e))
    assert np.linalg.norm(g[sample] - ps) / np.linalg.norm(ps) < tol
    assert np.max(np.abs(g[sample[:6]] - fd)) < (1e-4 if dtype == "c64" else 1e-7)
