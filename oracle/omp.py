"""The oracle's Section 3 update in C with OpenMP over set ids (sv_omp.c).

TEST INFRASTRUCTURE ONLY: the tests, the package entry's smoke check and the
benchmark's CPU-baseline / reference leg use it; the product never imports
anything under oracle/.  It computes what ``statevector.apply_gate``
computes (the same definition, written as the set-by-set loop) and is the
form that runs on every host core: the full-state checks at 26-28 qubits and
the timed CPU baseline use it.  It is pinned by the same checks as the numpy
oracle (tests/test_oracle_omp.py runs every pin with this update in place of
``apply_gate``) and checked against the numpy oracle on random circuits.

``build()`` compiles sv_omp.c with gcc (-O2 -fopenmp -ffp-contract=off) into
oracle/_build/; building the checker is not using it.
"""

from __future__ import annotations

import ctypes as ct
import os
import subprocess
from typing import Iterable, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sv_omp.c")
OUTDIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUTDIR, "libsv_omp.so")

_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUTDIR, exist_ok=True)
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC",
           SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("building the C oracle failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        lib = ct.CDLL(build())
        lib.or_apply_gate.restype = ct.c_int
        lib.or_apply_gate.argtypes = [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int), ct.c_int, ct.c_void_p]
        lib.or_max_threads.restype = ct.c_int
        lib.or_set_threads.argtypes = [ct.c_int]
        _lib = lib
    return _lib


def threads() -> int:
    """Threads the parallel loop uses (OMP_NUM_THREADS, else every core)."""
    return int(load().or_max_threads())


def set_threads(t: int) -> None:
    load().or_set_threads(int(t))


def apply_gate_inplace(psi: np.ndarray, n: int, qubits: Sequence[int], m) -> np.ndarray:
    """Apply m on `qubits` to the complex128 vector psi in place (Section 3)."""
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.shape != (1 << n,):
        raise ValueError("psi must be a contiguous complex128 vector of 2^n amplitudes")
    m = np.ascontiguousarray(m, dtype=np.complex128)
    k = len(qubits)
    if m.shape != (1 << k, 1 << k):
        raise ValueError("matrix shape does not match the qubit count")
    q = (ct.c_int * k)(*[int(x) for x in qubits])
    if load().or_apply_gate(psi.ctypes.data, int(n), q, k, m.ctypes.data) != 0:
        raise ValueError(f"bad gate {tuple(qubits)} for n={n}")
    return psi


def apply_gate(psi: np.ndarray, n: int, qubits: Sequence[int], m) -> np.ndarray:
    """Same signature and result as statevector.apply_gate (returns a new array)."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    return apply_gate_inplace(out, n, qubits, m)


def simulate(n: int, gates: Iterable, psi0: Optional[np.ndarray] = None) -> np.ndarray:
    """psi_out = U_L ... U_1 psi_0 (default |0...0>), gate by gate, in place."""
    if psi0 is None:
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1.0
    else:
        psi = np.array(psi0, dtype=np.complex128, copy=True)
    for g in gates:
        qs, m = (g.qubits, g.matrix) if hasattr(g, "qubits") else g
        apply_gate_inplace(psi, n, qs, m)
    return psi
