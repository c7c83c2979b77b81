"""Batched persistent execution: many circuits of uneven width in one
launch, each final state against the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle
from oracle import omp
from oracle.metrics import rel_l2
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C

pytestmark = pytest.mark.gpu

TOL = {"c64": 2e-5, "c128": 1e-12}


def _workload(count, seed0, n_range, depth_range):
    return C.batched_workload(count, seed0=seed0, n_range=n_range, depth_range=depth_range)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("tile", [8, 0])
def test_batch_matches_oracle(qs, dtype, tile):
    """tile=8 sends every circuit wider than 8 qubits through the multi-pass
    work queue; tile=0 (default width) keeps them inside one block each."""
    specs = _workload(20, 100, (5, 14), (3, 8))
    circs = [B.circuit_from(s) for s in specs]
    bt = B.Batch(circs, dtype, k_max=3, tile_qubits=tile)
    bt.run()
    bt.sync()
    for i, s in enumerate(specs):
        ref = oracle.simulate(s.n, s.gates)
        got = bt.state(i).to(torch.complex128).cpu().numpy()
        assert rel_l2(got, ref) < TOL[dtype], (i, s.n, rel_l2(got, ref))
    assert bt.info()["items"] >= len(specs)


def test_batch_replay_and_loop_equivalence(qs):
    specs = _workload(12, 7, (9, 15), (4, 10))
    circs = [B.circuit_from(s) for s in specs]
    bt = B.Batch(circs, "c64", k_max=2, tile_qubits=9)
    bt.run(); bt.sync()
    first = bt.states.clone()
    bt.run(); bt.sync()                       # graph replay, counters reset
    assert torch.equal(first, bt.states)
    for i, (s, c) in enumerate(zip(specs, circs)):
        p = B.Plan(c, "c64", k_max=2)
        st = B.State(s.n, "c64")
        p.execute(st)
        assert rel_l2(st.tensor.cpu().numpy(), bt.state(i).cpu().numpy()) < 2e-5


def test_batch_autotune(qs):
    specs = _workload(16, 3, (6, 13), (3, 6))
    circs = [B.circuit_from(s) for s in specs]
    best = B.batch_autotune(circs, "c64")
    assert 2 <= best.k_max <= 4 and best.tile_qubits in (12, 13)
    bt = B.Batch(circs, "c64", opts=best)
    bt.run(); bt.sync()
    s = specs[-1]
    assert rel_l2(bt.state(len(specs) - 1).cpu().numpy(), oracle.simulate(s.n, s.gates)) < 2e-5


def test_bounded_wait_timeout_is_reported(qs):
    """A work item whose dependency count is never reached (injected through
    the testing option) gives up after its bounded wait; the host reads
    QS_ERR_TIMEOUT and the context stays usable."""
    specs = _workload(6, 11, (10, 12), (3, 5))
    circs = [B.circuit_from(s) for s in specs]
    bad = B.Batch(circs, "c64", k_max=2, tile_qubits=8, inject_wait_timeout=True)
    bad.run()
    with pytest.raises(B.QsError) as e:
        bad.sync()
    assert e.value.status == 5
    bad.close()
    good = B.Batch(circs, "c64", k_max=2, tile_qubits=8)
    good.run()
    good.sync()
    s = specs[0]
    assert rel_l2(good.state(0).cpu().numpy(), oracle.simulate(s.n, s.gates)) < 2e-5


def test_batched_workload_sample_matches_oracle(qs):
    """The batched workload itself (512 grid circuits, n ~ U{10..22}, 8-24
    cycles, seeds 0..511) in one launch with autotuned options; 16 circuits
    drawn with a fixed seed (plus the widest) against the oracle."""
    specs = C.batched_workload(512, seed0=0)
    circs = [B.circuit_from(s) for s in specs]
    best = B.batch_autotune(circs, "c64")
    bt = B.Batch(circs, "c64", opts=best)
    bt.run()
    bt.sync()
    rng = np.random.default_rng(12)
    pick = sorted(set(rng.choice(len(specs), 16, replace=False).tolist()) |
                  {max(range(len(specs)), key=lambda i: (specs[i].n, len(specs[i].gates)))})
    for i in pick:
        s = specs[i]
        ref = omp.simulate(s.n, s.gates)
        got = bt.state(i).to(torch.complex128).cpu().numpy()
        assert rel_l2(got, ref) < 2e-5, (i, s.n, len(s.gates), rel_l2(got, ref))
