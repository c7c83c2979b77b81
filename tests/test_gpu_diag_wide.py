"""Clustering by kind (Sections 4.2, 4.5): diagonal gates of any width in one
wide pass (eighth-root exponent tables, or complex tables), the other gates
fused among themselves, against the FP64 oracle."""

import numpy as np
import pytest

import oracle
from oracle.metrics import rel_l2
from workloads import circuits as C
from workloads import gates as G
from workloads.rng import Xoshiro256ss, random_state, random_unitary

from gpu_util import TOL, run_plan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,depth", [(14, 10), (17, 12), (9, 8)])
@pytest.mark.parametrize("k_max", [1, 2, 4])
def test_paper_gate_set_clusters(qs, dtype, n, depth, k_max):
    circ = C.paper_circuit(n, depth, seed=3)
    ref = oracle.simulate(n, circ.gates)
    got, info = run_plan(circ, dtype, k_max=k_max, diag_clusters=True)
    assert rel_l2(got, ref) < TOL[dtype], info
    if n >= 14:
        assert info["per_kind"].get("diagonal_wide", 0) > 0, info


def _random_diag(k, rng):
    return np.diag(np.exp(1j * np.array([rng.uniform_range(-np.pi, np.pi) for _ in range(1 << k)])))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [9, 13, 19])
def test_general_phase_clusters(qs, dtype, n):
    """Arbitrary phases (complex tables): RZ, controlled phases and random
    3-qubit diagonals across chunk boundaries, between dense layers."""
    rng = Xoshiro256ss(70 + n)
    circ = C.Circuit(n)
    psi0 = random_state(n, n)
    for layer in range(3):
        for q in range(n):
            circ.append((q,), G.rz(rng.uniform_range(-3, 3)))
        for q in range(n - 1):
            circ.append((q, q + 1), G.cphase(rng.uniform_range(-3, 3)))
        for _ in range(4):
            qs_ = sorted({rng.randint(n) for _ in range(3)})
            if len(qs_) == 3:
                circ.append(tuple(qs_[::-1]), _random_diag(3, rng))
        for q in range(0, n, 3):
            circ.append((q,), random_unitary(1, rng))
    ref = oracle.simulate(n, circ.gates, psi0)
    got, info = run_plan(circ, dtype, psi0=psi0, k_max=2, diag_clusters=True)
    assert rel_l2(got, ref) < TOL[dtype], info
    assert info["per_kind"].get("diagonal_wide", 0) > 0, info


def test_clusters_with_tensor_passes(qs):
    """diag_clusters with 6-qubit tensor-core blocks for the dense part."""
    n = 16
    circ = C.paper_circuit(n, 14, seed=5)
    ref = oracle.simulate(n, circ.gates)
    got, info = run_plan(circ, "c64", k_max=6, precision="3xtf32", diag_clusters=True)
    assert rel_l2(got, ref) < TOL["c64"], info


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [11, 15])
def test_multiply_free_tile_gates(qs, dtype, n):
    """Section 4.1: one-qubit gates that are a scalar times a {0, +-1, +-i}
    matrix (H, sqrt X, sqrt Y, X, Y, and H times an arbitrary phase, whose
    scalar is not an eighth root) run without multiplies in tile passes;
    each pass multiplies the product of the scalars at write-back."""
    rng = Xoshiro256ss(300 + n)
    psi0 = random_state(n, 7 + n)
    circ = C.Circuit(n)
    odd_h = np.exp(0.3j) * G.H
    pool = [G.H, G.SQRT_X, G.SQRT_Y, G.X, G.Y, odd_h]
    for layer in range(6):
        for q in range(n):
            circ.append((q,), pool[rng.randint(len(pool))])
        for q in range(layer % 2, n - 1, 2):
            circ.append((q, q + 1), G.CZ)
    ref = oracle.simulate(n, circ.gates, psi0)
    for dc in (False, True):
        got, info = run_plan(circ, dtype, psi0=psi0, k_max=1, diag_clusters=dc)
        assert rel_l2(got, ref) < TOL[dtype], (dc, info)
