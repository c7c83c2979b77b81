"""The seeded input generator: structure of the synthetic grid circuits,
the ansatz and the Hamiltonian (no simulation here)."""

import math

import numpy as np
import pytest

from workloads import circuits as C
from workloads import gates as G
from workloads.rng import SplitMix64, Xoshiro256ss


def test_splitmix64_reference_values():
    # first outputs of SplitMix64 seeded with 0 (the published sequence)
    sm = SplitMix64(0)
    assert [sm.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                             0x06C45D188009454F]


def test_xoshiro_deterministic_and_uniform():
    a = Xoshiro256ss(123); b = Xoshiro256ss(123)
    xs = [a.uniform() for _ in range(20000)]
    assert xs[:50] == [b.uniform() for _ in range(50)]
    assert 0.49 < np.mean(xs) < 0.51 and min(xs) >= 0 and max(xs) < 1
    counts = np.bincount([a.randint(3) for _ in range(30000)], minlength=3)
    assert np.all(np.abs(counts - 10000) < 400)


@pytest.mark.parametrize("n,shape", [(12, (3, 4)), (30, (5, 6)), (32, (4, 8)), (28, (4, 7)),
                                     (24, (4, 6)), (26, (5, 6)), (11, (3, 4)), (10, (3, 4))])
def test_grid_shape(n, shape):
    assert C.grid_shape(n) == shape


def test_pattern_counts_3x4():
    counts = {p: len(C.coupling_pattern(3, 4, 12, p)) for p in "ABCD"}
    assert counts == {"A": 6, "B": 3, "C": 4, "D": 4}


def test_patterns_are_nearest_neighbour_and_disjoint():
    for n in (12, 26, 30):
        r, c = C.grid_shape(n)
        for p in "ABCD":
            pairs = C.coupling_pattern(r, c, n, p)
            used = [q for pr in pairs for q in pr]
            assert len(used) == len(set(used))
            for a, b in pairs:
                ra, ca = divmod(a, c); rb, cb = divmod(b, c)
                assert abs(ra - rb) + abs(ca - cb) == 1 and b < n


def test_small_grid_circuit_structure():
    circ = C.small_grid_circuit(seed=1)
    assert circ.n == 12
    assert [g.name for g in circ.gates[:12]] == ["h"] * 12
    fs = [g for g in circ.gates if g.name.startswith("fsim")]
    assert len(fs) == 2 * (6 + 3 + 4 + 4)
    ref = G.fsim(math.pi / 2, math.pi / 6)
    assert all(np.array_equal(g.matrix, ref) for g in fs)
    assert len(circ.gates) == 12 + 8 * 12 + len(fs)


def test_one_qubit_draw_never_repeats():
    circ = C.scale_grid_circuit(20, 10, seed=4)
    last = {}
    for g in circ.gates:
        if g.name.startswith("sqrt"):
            q = g.qubits[0]
            assert last.get(q) != g.name
            last[q] = g.name


def test_scale_circuit_counts_and_determinism():
    a = C.scale_grid_circuit(30, 14, seed=1)
    b = C.scale_grid_circuit(30, 14, seed=1)
    assert len(a) == 30 + 14 * 30 + 3 * 15 + 3 * 10 + 4 * 12 + 4 * 12
    assert all(np.array_equal(x.matrix, y.matrix) and x.qubits == y.qubits for x, y in zip(a.gates, b.gates))
    c = C.scale_grid_circuit(30, 14, seed=2)
    assert any(not np.array_equal(x.matrix, y.matrix) for x, y in zip(a.gates, c.gates))


def test_ansatz_layout():
    n, layers = 5, 3
    theta = C.ansatz_theta(n, layers, seed=1)
    assert theta.shape == (30,) and np.all(np.abs(theta) <= math.pi)
    circ = C.ansatz_circuit(n, layers, theta)
    assert len(circ) == layers * (2 * n + n - 1)
    params = [g.param for g in circ.gates if g.param >= 0]
    assert sorted(params) == list(range(30))
    assert {g.generator for g in circ.gates if g.param >= 0} == {"Y", "Z"}


def test_ising_terms():
    H = C.ising_hamiltonian(4)
    assert len(H) == 3 + 4
    assert all(t.coeff == 1.0 for t in H)


def test_batched_workload_ranges():
    ws = C.batched_workload(24, seed0=0)
    assert all(10 <= c.n <= 22 for c in ws)
    assert len({c.n for c in ws}) > 4


def test_paper_circuit_rules():
    """The paper's gate set, H layers first and last, at most one CZ per
    qubit per cycle, T as a qubit's first gate after H, no repeated
    one-qubit gate, seeded and deterministic."""
    n, depth = 20, 16
    c1 = C.paper_circuit(n, depth, seed=4)
    c2 = C.paper_circuit(n, depth, seed=4)
    assert [(g.qubits, g.name) for g in c1.gates] == [(g.qubits, g.name) for g in c2.gates]
    assert {g.name for g in c1.gates} <= {"h", "cz", "t", "sqrt_x", "sqrt_y"}
    assert [g.name for g in c1.gates[:n]] == ["h"] * n and [g.name for g in c1.gates[-n:]] == ["h"] * n
    last = ["h"] * n
    for g in c1.gates[n:-n]:
        if g.name == "cz":
            continue
        q = g.qubits[0]
        if last[q] == "h":
            assert g.name == "t"
        assert g.name != last[q]
        last[q] = g.name
    rows, cols = C.grid_shape(n)
    for p in range(8):
        pairs = C.paper_cz_layer(rows, cols, n, p)
        qs = [q for pr in pairs for q in pr]
        assert len(qs) == len(set(qs)) and pairs
        for a, b in pairs:  # nearest neighbours on the grid
            assert b - a in (1, cols) and (b - a != 1 or a // cols == b // cols)
