"""Parity at the workload's sizes.

(1) Stored FP64 oracle amplitudes (tests/golden, written by make_golden.py,
which imports only the oracle) of the seeded grid circuits at 26 and 28
qubits against the CUDA path in the configuration the benchmark times
(k_max = 6, 3xTF32 tensor-core passes), the FP32 tile path and complex128:
512 sampled amplitudes, the first 64, sum |a|^2 and sum |a|^4.

(2) At 30 qubits (the timed size, where the oracle would take over an hour)
properties that hold at any size: the circuit followed by its inverse
returns |0...0>, the norm stays 1, and two independent kernel paths (tensor
cores, FP32 shared-memory tiles) agree on sampled amplitudes."""

import json
import os

import numpy as np
import pytest
import torch

from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = sorted(f for f in os.listdir(os.path.join(HERE, "golden")) if f.endswith(".json"))

# (dtype, plan options, relative L2 bound on the sampled amplitudes)
CONFIGS = [
    ("c64", dict(k_max=6, precision="3xtf32"), 2e-5),
    ("c64", dict(k_max=3, precision="fp32"), 2e-5),
    ("c128", dict(k_max=4), 1e-12),
]


def _run(circ, dtype, opts):
    c = B.circuit_from(circ)
    p = B.Plan(c, dtype, **opts)
    s = B.State(circ.n, dtype)
    p.execute(s)
    s.sync()
    info = p.info()
    p.close()
    c.close()
    return s, info


@pytest.mark.parametrize("fname", GOLDEN)
@pytest.mark.parametrize("dtype,opts,tol", CONFIGS, ids=["c64-tensor", "c64-tile", "c128"])
def test_golden_sampled_amplitudes(qs, fname, dtype, opts, tol):
    g = json.load(open(os.path.join(HERE, "golden", fname)))
    circ = C.scale_grid_circuit(g["n"], g["cycles"], seed=g["seed"])
    assert len(circ.gates) == g["num_gates"]  # the generator still draws the same circuit
    s, info = _run(circ, dtype, opts)
    if opts.get("precision") == "3xtf32":
        assert info["per_kind"].get("tensor", 0) > 0, info
    idx = torch.tensor(g["indices"], dtype=torch.long, device=s.tensor.device)
    got = s.tensor[idx].cpu().numpy().astype(np.complex128)
    ref = np.array([complex(a, b) for a, b in g["amplitudes"]])
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    first = s.tensor[:64].cpu().numpy().astype(np.complex128)
    ref64 = np.array([complex(a, b) for a, b in g["first64"]])
    assert np.linalg.norm(first - ref64) / np.linalg.norm(ref64) < tol
    # with relative L2 error e, |sum|a|^2 - sum|b|^2| <= (2 + e) e sum|b|^2 and
    # sum p^2 moves by at most ~4 e relative: bounds follow from tol
    assert abs(s.norm() - g["sum_p"]) < 2.1 * tol * g["sum_p"]
    p = (s.tensor.abs() ** 2).to(torch.float64)
    assert abs(float((p * p).sum()) / g["sum_p2"] - 1) < 4.2 * tol
    s.close()


def _inverse(circ):
    inv = C.Circuit(circ.n)
    for gt in reversed(circ.gates):
        inv.append(gt.qubits, gt.matrix.conj().T)
    return inv


def test_full_size_mirror_and_norm(qs):
    """30 qubits, the timed configuration: U then U^dagger gives back |0>."""
    n = 30
    circ = C.scale_grid_circuit(n, 14, seed=1)
    opts = dict(k_max=6, precision="3xtf32")
    s, info = _run(circ, "c64", opts)
    assert info["per_kind"].get("tensor", 0) > 0
    # complex64 bound of 2e-5 relative L2 per circuit: norm within 2.1 x that
    assert abs(s.norm() - 1.0) < 4.2e-5
    c = B.circuit_from(_inverse(circ))
    p = B.Plan(c, "c64", **opts)
    p.execute(s)
    a0 = complex(s.tensor[0].item())
    assert abs(a0 - 1.0) < 4e-5, a0   # two circuits' worth of error
    assert abs(s.norm() - 1.0) < 8.4e-5
    p.close()
    c.close()
    s.close()


def test_full_size_two_kernel_paths_agree(qs):
    """30 qubits: tensor-core 6-qubit passes and FP32 shared-memory tile
    passes, two independent kernels, agree on 4096 sampled amplitudes."""
    n = 30
    circ = C.scale_grid_circuit(n, 14, seed=1)
    rng = np.random.default_rng(5)
    idx = torch.tensor(np.sort(rng.choice(1 << n, 4096, replace=False)), dtype=torch.long, device="cuda")
    s1, _ = _run(circ, "c64", dict(k_max=6, precision="3xtf32"))
    a = s1.tensor[idx].cpu().numpy().astype(np.complex128)
    s1.close()
    s2, info = _run(circ, "c64", dict(k_max=3, precision="fp32"))
    assert info["per_kind"].get("tensor", 0) == 0
    b = s2.tensor[idx].cpu().numpy().astype(np.complex128)
    s2.close()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 4e-5
