"""Full-state parity at the workload's sizes: every amplitude of the seeded
30-qubit-style grid circuit (patterns ABCDCDAB, random fSim angles, 14
cycles) at 26 and 28 qubits, CUDA path against the FP64 oracle computed on
the host in the same process (the C form of the oracle, all host cores).

Per configuration: relative L2 over all 2^n amplitudes, the largest
amplitude error, max |dp| and the total-variation distance.  Bounds:
  complex64, 3xTF32 or 3xFP16 tensor passes (one or two blocks per round
      trip), or FP32 tiles: 2e-5
  complex128: 1e-12
  complex64, TF32 tensor passes: 4e-3 -- one TF32 rounding (2^-11 relative)
      per operand in each of the ~20-25 passes, growing like sqrt(passes)
  complex64, 3xBF16 tensor passes: 6e-5 -- the bf16 hi/lo split keeps ~16
      mantissa bits per operand (2^-17 relative per pass), over ~25 passes
Max |dp| and TV are reported and checked against what the amplitude
errors allow: |p - p_ref| <= (2|a_ref| + |d|)|d| per amplitude, and
TV <= ||d|| (2||a_ref|| + ||d||) / 2 (Cauchy-Schwarz, ||a_ref|| = 1)."""

import numpy as np
import pytest
import torch

from oracle import omp
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C

pytestmark = pytest.mark.gpu

CONFIGS = {
    "c64-3xtf32": ("c64", dict(k_max=6, precision="3xtf32"), 2e-5),
    "c64-fp32-tile": ("c64", dict(k_max=3, precision="fp32"), 2e-5),
    "c128": ("c128", dict(k_max=4), 1e-12),                # 4-qubit blocks: the FP64 shared-memory tile
    "c128-ff": ("c128", dict(k_max=3), 1e-12),             # the float-float register tile (the default)
    "c64-tf32": ("c64", dict(k_max=6, precision="tf32"), 4e-3),
    "c64-3xbf16": ("c64", dict(k_max=6, precision="3xbf16"), 6e-5),
    "c64-3xfp16": ("c64", dict(k_max=6, precision="3xfp16"), 2e-5),
    "c64-3xfp16-tiles": ("c64", dict(k_max=6, precision="3xfp16", tensor_tiles=True), 2e-5),
}
CASES = [(26, name) for name in CONFIGS] + [(28, name) for name in
                                            ("c64-3xtf32", "c64-tf32", "c64-3xbf16", "c64-3xfp16-tiles", "c128",
                                             "c128-ff")]

_ORACLE = {}


def _oracle_state(n):
    """The oracle's final state of the grid circuit, on the GPU as complex128
    (computed once per size on the host cores)."""
    if n not in _ORACLE:
        _ORACLE.clear()
        circ = C.scale_grid_circuit(n, 14, seed=1)
        psi = omp.simulate(n, circ.gates)
        _ORACLE[n] = (circ, torch.from_numpy(psi).cuda())
        del psi
    return _ORACLE[n]


def _errors(got, ref):
    """relative L2, max |a - a_ref|, max |dp|, TV and max |a_ref| over every
    amplitude, in chunks (complex128 on the GPU)"""
    d2 = r2 = amax = pmax = tv = rmax = 0.0
    step = 1 << 24
    for i in range(0, ref.numel(), step):
        r = ref[i:i + step]
        x = got[i:i + step].to(torch.complex128)
        d = x - r
        d2 += float((d.abs() ** 2).sum())
        r2 += float((r.abs() ** 2).sum())
        amax = max(amax, float(d.abs().max()))
        dp = (x.abs() ** 2 - r.abs() ** 2).abs()
        pmax = max(pmax, float(dp.max()))
        tv += 0.5 * float(dp.sum())
        rmax = max(rmax, float(r.abs().max()))
    return (d2 / r2) ** 0.5, amax, pmax, tv, rmax


@pytest.mark.parametrize("n,name", CASES, ids=[f"{n}q-{c}" for n, c in CASES])
def test_full_state_against_oracle(qs, n, name):
    dtype, opts, tol = CONFIGS[name]
    circ, ref = _oracle_state(n)
    c = B.circuit_from(circ)
    p = B.Plan(c, dtype, **opts)
    if opts.get("precision", "fp32") != "fp32":
        assert p.info()["per_kind"].get("tensor", 0) > 0
    s = B.State(n, dtype)
    p.execute(s)
    s.sync()
    rel, amax, pmax, tv, rmax = _errors(s.tensor, ref)
    assert rel < tol, (name, n, "relative L2", rel, "max |da|", amax, "max |dp|", pmax, "TV", tv)
    assert pmax <= 1.01 * (2 * rmax + amax) * amax, (pmax, amax, rmax)
    assert tv <= 1.01 * 0.5 * (2 + rel) * rel, (tv, rel)
    p.close()
    c.close()
    s.close()
