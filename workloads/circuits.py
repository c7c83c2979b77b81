"""Seeded synthetic circuits shaped like the paper's random-circuit workloads.

The paper benchmarks Google's grid "supremacy" circuits (Section 6): an
initial Hadamard layer, then cycles of one-qubit gates on every qubit and
two-qubit gates on one nearest-neighbour coupling pattern per cycle.  Those
circuit files are not available, so this module generates circuits with that
structure from a seed:

* grid R x C, qubit id r*C + c;
* coupling patterns A: (r,c)-(r,c+1) for even c, B: the same for odd c,
  C: (r,c)-(r+1,c) for even r, D: the same for odd r (bonds only between
  qubits that exist, for a partial last row);
* cycle 1 draws each qubit's gate uniformly from {sqrt X, sqrt Y, sqrt W};
  later cycles draw uniformly from the two gates that differ from that
  qubit's previous one; draws go qubit by qubit in ascending order, then
  the fSim angles in pair order;
* fSim(theta, phi) on every pair of the cycle's pattern, with fixed angles
  or theta ~ U(0, pi/2), phi ~ U(0, pi).

It also builds the hardware-efficient variational ansatz (RY and RZ on every
qubit per layer, then a CZ ladder) and the transverse-field Ising
Hamiltonian used for gradients.  A gate is data: qubits plus an FP64 matrix;
parametrised gates also carry a parameter id and a Pauli generator.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import gates as G
from .rng import Xoshiro256ss, random_unitary


@dataclass
class Gate:
    qubits: Tuple[int, ...]
    matrix: np.ndarray                   # 2^k x 2^k complex128, Kronecker order
    name: str = ""
    param: int = -1                      # parameter index, -1 when fixed
    generator: str = ""                  # Pauli string P for exp(-i theta P / 2)

    @property
    def k(self) -> int:
        return len(self.qubits)


@dataclass
class Circuit:
    n: int
    gates: List[Gate] = field(default_factory=list)
    num_params: int = 0
    theta: Optional[np.ndarray] = None   # parameter values the matrices were built with

    def append(self, qubits, matrix, name="", param=-1, generator=""):
        self.gates.append(Gate(tuple(int(q) for q in qubits),
                               np.asarray(matrix, dtype=np.complex128),
                               name, param, generator))

    def __len__(self):
        return len(self.gates)


# --------------------------------------------------------------------------
# grid geometry
# --------------------------------------------------------------------------

def grid_shape(n: int) -> Tuple[int, int]:
    """Rows and columns for n qubits: the largest divisor r <= sqrt(n) when
    n/r <= 2r, else r = floor(sqrt n) rows of ceil(n/r) columns with a
    partial last row."""
    r = max(d for d in range(1, int(math.isqrt(n)) + 1) if n % d == 0)
    if n // r <= 2 * r:
        return r, n // r
    r = math.isqrt(n)
    return r, -(-n // r)


def coupling_pattern(rows: int, cols: int, n: int, pattern: str) -> List[Tuple[int, int]]:
    pairs = []
    for r in range(rows):
        for c in range(cols):
            a = r * cols + c
            if a >= n:
                continue
            if pattern in "AB":
                if c % 2 == (0 if pattern == "A" else 1) and c + 1 < cols:
                    b = a + 1
                    if b < n:
                        pairs.append((a, b))
            else:
                if r % 2 == (0 if pattern == "C" else 1) and r + 1 < rows:
                    b = a + cols
                    if b < n:
                        pairs.append((a, b))
    return pairs


PATTERN_ABCD = "ABCD"
PATTERN_ABCDCDAB = "ABCDCDAB"


def grid_circuit(n: int, cycles: int, seed: int, *, rows: Optional[int] = None,
                 cols: Optional[int] = None, patterns: str = PATTERN_ABCDCDAB,
                 fixed_fsim: Optional[Tuple[float, float]] = None,
                 initial_h: bool = True) -> Circuit:
    """Random grid circuit: H layer, then `cycles` x (1q layer, fSim layer)."""
    if rows is None or cols is None:
        rows, cols = grid_shape(n)
    if rows * cols < n:
        raise ValueError("grid too small for n qubits")
    rng = Xoshiro256ss(seed)
    circ = Circuit(n)
    if initial_h:
        for q in range(n):
            circ.append((q,), G.H, "h")
    names = ["sqrt_x", "sqrt_y", "sqrt_w"]
    prev = [-1] * n
    for cyc in range(cycles):
        for q in range(n):
            if prev[q] < 0:
                g = rng.randint(3)
            else:
                choices = [i for i in range(3) if i != prev[q]]
                g = choices[rng.randint(2)]
            prev[q] = g
            circ.append((q,), G.ONE_QUBIT_SET[names[g]], names[g])
        pat = patterns[cyc % len(patterns)]
        for (a, b) in coupling_pattern(rows, cols, n, pat):
            if fixed_fsim is not None:
                th, ph = fixed_fsim
            else:
                th = rng.uniform_range(0.0, math.pi / 2)
                ph = rng.uniform_range(0.0, math.pi)
            circ.append((a, b), G.fsim(th, ph), f"fsim_{pat}")
    return circ


def small_grid_circuit(seed: int = 1) -> Circuit:
    """12 qubits on a 3x4 grid, 8 cycles, fSim(pi/2, pi/6), patterns ABCD."""
    return grid_circuit(12, 8, seed, rows=3, cols=4, patterns=PATTERN_ABCD,
                        fixed_fsim=(math.pi / 2, math.pi / 6))


def scale_grid_circuit(n: int = 30, cycles: int = 14, seed: int = 1) -> Circuit:
    """n qubits (30 -> 5x6), `cycles` cycles of ABCDCDAB with random fSim."""
    return grid_circuit(n, cycles, seed)


# --------------------------------------------------------------------------
# circuits in the paper's benchmark gate set (H, CZ, T, sqrt(X), sqrt(Y))
# --------------------------------------------------------------------------

# CZ layer order: horizontal and vertical layers alternate
PAPER_CZ_ORDER = (0, 4, 1, 5, 2, 6, 3, 7)


def paper_cz_layer(rows: int, cols: int, n: int, p: int) -> List[Tuple[int, int]]:
    """CZ layer p in 0..7 on the grid: p < 4 horizontal bonds (r,c)-(r,c+1),
    p >= 4 vertical bonds (r,c)-(r+1,c); of those, the bonds with the moving
    coordinate = p & 1 and the other coordinate = (p >> 1) & 1 (mod 2).  No
    qubit is in two bonds of one layer."""
    a, b = p & 1, (p >> 1) & 1
    pairs = []
    for r in range(rows):
        for c in range(cols):
            q = r * cols + c
            if q >= n:
                continue
            if p < 4 and c % 2 == a and r % 2 == b and c + 1 < cols and q + 1 < n:
                pairs.append((q, q + 1))
            if p >= 4 and r % 2 == a and c % 2 == b and r + 1 < rows and q + cols < n:
                pairs.append((q, q + cols))
    return pairs


def paper_circuit(n: int, depth: int = 26, seed: int = 1) -> Circuit:
    """Depth 1 + depth + 1 in the paper's gate set: an H layer, `depth`
    cycles, a final H layer.  Cycle c applies CZ layer PAPER_CZ_ORDER[c % 8];
    a qubit that had a CZ in the previous cycle and has none in this one gets
    a one-qubit gate: T the first time, afterwards a random choice among
    {T, sqrt(X), sqrt(Y)} other than its previous one-qubit gate (seeded,
    qubits in ascending order)."""
    rows, cols = grid_shape(n)
    rng = Xoshiro256ss(seed)
    circ = Circuit(n)
    for q in range(n):
        circ.append((q,), G.H, "h")
    last = ["h"] * n
    prev_cz = set()
    mats = {"t": G.T, "sqrt_x": G.SQRT_X, "sqrt_y": G.SQRT_Y}
    for c in range(depth):
        pairs = paper_cz_layer(rows, cols, n, PAPER_CZ_ORDER[c % 8])
        now = {q for pr in pairs for q in pr}
        for q in range(n):
            if q in prev_cz and q not in now:
                if last[q] == "h":
                    g = "t"
                else:
                    choices = [x for x in ("t", "sqrt_x", "sqrt_y") if x != last[q]]
                    g = choices[rng.randint(len(choices))]
                circ.append((q,), mats[g], g)
                last[q] = g
        for a, b in pairs:
            circ.append((a, b), G.CZ, "cz")
        prev_cz = now
    for q in range(n):
        circ.append((q,), G.H, "h")
    return circ


# --------------------------------------------------------------------------
# variational ansatz and Ising Hamiltonian
# --------------------------------------------------------------------------

def ansatz_num_params(n: int, layers: int) -> int:
    return 2 * n * layers


def ansatz_param_index(n: int, layer: int, qubit: int, which: int) -> int:
    """which = 0 for RY, 1 for RZ."""
    return layer * 2 * n + 2 * qubit + which


def ansatz_circuit(n: int, layers: int, theta: Sequence[float]) -> Circuit:
    """Per layer: RY(theta) then RZ(theta) on each qubit (own parameters),
    then CZ(i, i+1) for i = 0..n-2 (open chain)."""
    theta = np.asarray(theta, dtype=np.float64)
    if theta.shape != (ansatz_num_params(n, layers),):
        raise ValueError("theta has the wrong length")
    circ = Circuit(n, num_params=theta.size, theta=theta.copy())
    for l in range(layers):
        for q in range(n):
            p = ansatz_param_index(n, l, q, 0)
            circ.append((q,), G.ry(theta[p]), "ry", p, "Y")
            p = ansatz_param_index(n, l, q, 1)
            circ.append((q,), G.rz(theta[p]), "rz", p, "Z")
        for q in range(n - 1):
            circ.append((q, q + 1), G.CZ, "cz")
    return circ


def ansatz_theta(n: int, layers: int, seed: int) -> np.ndarray:
    rng = Xoshiro256ss(seed)
    return np.array([rng.uniform_range(-math.pi, math.pi)
                     for _ in range(ansatz_num_params(n, layers))])


@dataclass
class PauliTerm:
    coeff: float
    ops: Tuple[Tuple[int, str], ...]     # ((qubit, 'X'|'Y'|'Z'), ...)


def ising_hamiltonian(n: int) -> List[PauliTerm]:
    """H = sum_{i=0}^{n-2} Z_i Z_{i+1} + sum_i X_i, unit coefficients."""
    terms = [PauliTerm(1.0, ((i, "Z"), (i + 1, "Z"))) for i in range(n - 1)]
    terms += [PauliTerm(1.0, ((i, "X"),)) for i in range(n)]
    return terms


# --------------------------------------------------------------------------
# random circuits for tests and the batched workload
# --------------------------------------------------------------------------

def random_circuit(n: int, num_gates: int, seed: int, max_k: int = 3,
                   qubit_pool: Optional[Sequence[int]] = None,
                   kinds: Sequence[str] = ("dense", "diag", "monomial")) -> Circuit:
    """Random gates on random qubit subsets of size 1..max_k, mixing dense
    unitaries, diagonal phases and permutation-with-phase matrices."""
    rng = Xoshiro256ss(seed)
    pool = list(range(n)) if qubit_pool is None else list(qubit_pool)
    circ = Circuit(n)
    for _ in range(num_gates):
        k = 1 + rng.randint(min(max_k, len(pool)))
        qs = []
        while len(qs) < k:
            q = pool[rng.randint(len(pool))]
            if q not in qs:
                qs.append(q)
        kind = kinds[rng.randint(len(kinds))]
        d = 1 << k
        if kind == "dense":
            m = random_unitary(k, rng)
        elif kind == "diag":
            m = np.diag([np.exp(1j * rng.uniform_range(0, 2 * math.pi)) for _ in range(d)])
        else:
            perm = list(range(d))
            for i in range(d - 1, 0, -1):
                j = rng.randint(i + 1)
                perm[i], perm[j] = perm[j], perm[i]
            m = np.zeros((d, d), dtype=np.complex128)
            for r in range(d):
                m[r, perm[r]] = np.exp(1j * rng.uniform_range(0, 2 * math.pi))
        circ.append(qs, m, kind)
    return circ


def batched_workload(num_circuits: int = 512, seed0: int = 0,
                     n_range=(10, 22), depth_range=(8, 24)) -> List[Circuit]:
    """Circuits with qubit counts uniform in n_range and depth uniform in
    depth_range (inclusive), each on its near-square grid."""
    out = []
    for i in range(num_circuits):
        rng = Xoshiro256ss(seed0 + i)
        n = n_range[0] + rng.randint(n_range[1] - n_range[0] + 1)
        depth = depth_range[0] + rng.randint(depth_range[1] - depth_range[0] + 1)
        out.append(grid_circuit(n, depth, seed=(1 << 32) + seed0 + i))
    return out
