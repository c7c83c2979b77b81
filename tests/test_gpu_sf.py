"""Schroedinger-Feynman mode (qs_sf_amplitudes): amplitudes from two
half-size simulations per path, summed over the Feynman paths through the
gates across the cut, against the FP64 oracle's full state.  Circuits: the
paper's gate set (H, CZ, T, sqrt X, sqrt Y; CZ splits into 2 terms) and the
grid circuit with fSim gates (4 terms each) at small depth, with cuts
between grid columns and an uneven cut."""

import numpy as np
import pytest

import oracle
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C

pytestmark = pytest.mark.gpu

TOL = {"c64": 2e-5, "c128": 1e-12}


def _check(circ, part_a, dtype, max_paths):
    ref = oracle.simulate(circ.n, circ.gates)
    rng = np.random.default_rng(circ.n)
    idx = np.unique(np.concatenate([np.arange(64), rng.integers(0, 1 << circ.n, 512)])).astype(np.uint64)
    c = B.circuit_from(circ)
    got, paths = B.sf_amplitudes(c, part_a, idx, dtype)
    assert 1 < paths <= max_paths, paths
    want = ref[idx.astype(np.int64)]
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < TOL[dtype], (err, paths)
    c.close()
    return paths


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_sf_paper_gate_set(qs, dtype):
    n = 16                                   # 4 x 4 grid, cut between columns 1 and 2
    circ = C.paper_circuit(n, depth=6, seed=3)
    rows, cols = C.grid_shape(n)
    part_a = [r * cols + cc for r in range(rows) for cc in range(cols // 2)]
    _check(circ, part_a, dtype, 1 << 16)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_sf_grid_fsim(qs, dtype):
    n = 12                                   # 3 x 4 grid, 3 cycles: fSim gates across the cut
    circ = C.grid_circuit(n, 3, seed=5)
    rows, cols = C.grid_shape(n)
    part_a = [r * cols + cc for r in range(rows) for cc in range(cols // 2)]
    _check(circ, part_a, dtype, 1 << 16)


def test_sf_uneven_cut_and_path_count(qs):
    """A cut with 3 of 10 qubits on one side; count 0 only reports paths."""
    n = 10
    circ = C.paper_circuit(n, depth=4, seed=8)
    part_a = [0, 1, 5]
    c = B.circuit_from(circ)
    empty, p0 = B.sf_amplitudes(c, part_a, [], "c64")
    assert empty.size == 0 and p0 >= 1
    c.close()
    assert _check(circ, part_a, "c128", 1 << 16) == p0


def test_sf_rejects_bad_cuts(qs):
    circ = C.paper_circuit(8, depth=2, seed=1)
    c = B.circuit_from(circ)
    with pytest.raises(B.QsError):
        B.sf_amplitudes(c, [], [0], "c64")             # empty half
    with pytest.raises(B.QsError):
        B.sf_amplitudes(c, list(range(8)), [0], "c64")  # nothing in the other half
    with pytest.raises(B.QsError):
        B.sf_amplitudes(c, [0, 9], [0], "c64")          # a qubit outside the circuit
    c.close()
