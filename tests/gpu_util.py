"""Helpers for the GPU parity tests: move seeded states between numpy and
library states, run circuits through the C ABI, read back amplitudes."""

from __future__ import annotations

import numpy as np
import torch

from paper_2008_00216_gb300 import binding as B

TOL = {"c64": 2e-5, "c128": 1e-12}   # relative L2 against the FP64 oracle


def to_state(psi0: np.ndarray, n: int, dtype: str) -> B.State:
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    t = torch.from_numpy(np.asarray(psi0, dtype=np.complex128)).to(tdt).cuda()
    return B.State(n, dtype, tensor=t, init=None)


def run_gates(n, gates, dtype, psi0=None) -> np.ndarray:
    """Apply gates one by one with qs_apply_gate."""
    s = B.State(n, dtype) if psi0 is None else to_state(psi0, n, dtype)
    for g in gates:
        qs_, m = (g.qubits, g.matrix) if hasattr(g, "qubits") else g
        B.apply_gate(s, qs_, m)
    out = s.amplitudes()
    s.close()
    return out


def run_plan(circ, dtype, psi0=None, **opts) -> tuple:
    c = B.circuit_from(circ)
    p = B.Plan(c, dtype, **opts)
    s = B.State(circ.n, dtype) if psi0 is None else to_state(psi0, circ.n, dtype)
    p.execute(s)
    out = s.amplitudes()
    info = p.info()
    s.close(); p.close(); c.close()
    return out, info
