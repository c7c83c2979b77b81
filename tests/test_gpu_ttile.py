"""Tensor tile pass: up to two dense 6-qubit blocks applied to 12-qubit
tiles in shared memory per HBM round trip (3xFP16 tensor cores), against the
FP64 oracle.  Cases: 12 qubits (one tile) and 13/14 qubits (tile counts that
leave partial groups of three), blocks on qubits 0 and 1, three blocks
whose first two share a pass, blocks separated by one-qubit gates that do or do not commute with
them, and the grid circuit fused at k_max = 6."""

import numpy as np
import pytest

import oracle
from oracle.metrics import rel_l2
from workloads import circuits as C
from workloads.rng import Xoshiro256ss, random_state, random_unitary

from gpu_util import run_plan

pytestmark = pytest.mark.gpu

# 3xFP16 keeps ~22 bits per operand: ~2e-7 relative per block, a few blocks
TOL = 3e-6


def _blocks_circuit(n, groups, seed, between=()):
    """groups: list of qubit lists (each 6 qubits) -> one random dense
    unitary each; between: (index, qubit) one-qubit gates inserted before
    group `index`."""
    rng = Xoshiro256ss(seed)
    circ = C.Circuit(n)
    ins = {}
    for idx, q in between:
        ins.setdefault(idx, []).append(q)
    for i, qs in enumerate(groups):
        for q in ins.get(i, []):
            circ.append((q,), random_unitary(1, rng))
        circ.append(tuple(qs), random_unitary(6, rng))
    return circ


CASES = [
    # n, blocks, expected tensor-tile passes
    (12, [[11, 9, 7, 5, 3, 2], [10, 8, 6, 4, 3, 2]], 1),
    (12, [[0, 1, 2, 3, 4, 5], [6, 7, 8, 9, 10, 11], [0, 2, 4, 6, 8, 10]], 1),
    (13, [[12, 10, 7, 5, 4, 2], [12, 10, 8, 6, 3, 2]], 1),
    (14, [[13, 11, 9, 7, 5, 3], [13, 11, 9, 6, 4, 2]], 1),
    (14, [[0, 5, 9, 11, 12, 13], [1, 2, 3, 4, 6, 7]], 1),          # qubit 0 then qubit 1 targeted
    (16, [[2, 3, 4, 5, 6, 7], [0, 1, 2, 3, 8, 9], [4, 5, 6, 7, 8, 9]], 1),
    (17, [[16, 15, 14, 13, 12, 11], [16, 15, 14, 10, 9, 8], [13, 12, 11, 10, 9, 8]], 1),
    (20, [[19, 3, 7, 11, 15, 2], [19, 3, 7, 13, 17, 4]], 1),
]


@pytest.mark.parametrize("n,groups,ntt", CASES, ids=[f"{c[0]}q-{len(c[1])}b-{i}" for i, c in enumerate(CASES)])
def test_tensor_tile_pass_blocks(qs, n, groups, ntt):
    circ = _blocks_circuit(n, groups, seed=n * 31 + len(groups))
    psi0 = random_state(n, n + 5)
    ref = oracle.simulate(n, circ.gates, psi0)
    got, info = run_plan(circ, "c64", psi0=psi0, k_max=6, precision="3xfp16", fuse=False, use_tile=False,
                         tensor_tiles=True)
    assert info["per_kind"].get("tensor_tile", 0) == ntt, info
    assert rel_l2(got, ref) < TOL, rel_l2(got, ref)


def test_tensor_tile_pass_respects_order(qs):
    """A one-qubit gate on a qubit of the second block sits between the
    blocks: the second block may not move ahead of it, so no grouping; a
    one-qubit gate on another qubit commutes and the blocks still group."""
    n = 16
    groups = [[15, 13, 11, 9, 7, 5], [15, 13, 11, 8, 6, 4]]
    psi0 = random_state(n, 3)
    blocked = _blocks_circuit(n, groups, 5, between=[(1, 8)])
    ref = oracle.simulate(n, blocked.gates, psi0)
    got, info = run_plan(blocked, "c64", psi0=psi0, k_max=6, precision="3xfp16", fuse=False, use_tile=False,
                         tensor_tiles=True)
    assert info["per_kind"].get("tensor_tile", 0) == 0, info
    assert rel_l2(got, ref) < TOL
    # the gate on qubit 3 touches neither block: the blocks group around it
    free = _blocks_circuit(n, groups + [[15, 14, 13, 12, 11, 10]], 6, between=[(1, 3)])
    ref = oracle.simulate(n, free.gates, psi0)
    got, info = run_plan(free, "c64", psi0=psi0, k_max=6, precision="3xfp16", fuse=False, use_tile=False,
                         tensor_tiles=True)
    assert info["per_kind"].get("tensor_tile", 0) >= 1, info
    assert rel_l2(got, ref) < TOL


@pytest.mark.parametrize("n", [14, 20, 23])
def test_grid_circuit_tensor_tiles(qs, n):
    circ = C.scale_grid_circuit(n, 14, seed=2)
    ref = oracle.simulate(n, circ.gates)
    got, info = run_plan(circ, "c64", k_max=6, precision="3xfp16", tensor_tiles=True)
    assert info["per_kind"].get("tensor_tile", 0) > 0, info
    assert rel_l2(got, ref) < 2e-5, (rel_l2(got, ref), info)
