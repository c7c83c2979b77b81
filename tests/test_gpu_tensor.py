"""Dense 6-qubit (and padded 5-qubit) fused gates on the tcgen05 tensor
cores, in the three split-precision modes, against the FP64 oracle."""

import numpy as np
import pytest

import oracle
from oracle.metrics import rel_l2
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C
from workloads.rng import Xoshiro256ss, random_state, random_unitary

from gpu_util import run_plan, to_state

pytestmark = pytest.mark.gpu

# per-gate relative L2 bounds: TF32 keeps ~11 bits; the split modes ~FP32
GATE_TOL = {"tf32": 3e-3, "3xtf32": 2e-6, "3xbf16": 3e-5, "3xfp16": 2e-6}
PLACEMENTS = [[0, 1, 2, 3, 4, 5], [13, 12, 11, 10, 9, 8], [0, 13, 3, 7, 9, 11], [6, 2, 12, 1, 10, 5],
              [1, 2, 3, 4, 5, 6]]


def _one_gate_circuit(n, qubits, m):
    circ = C.Circuit(n)
    circ.append(qubits, m)
    return circ


@pytest.mark.parametrize("prec", ["tf32", "3xtf32", "3xbf16", "3xfp16"])
def test_single_6q_gate_all_placements(qs, prec):
    n = 14
    rng = Xoshiro256ss(77)
    psi0 = random_state(n, 3)
    for qubits in PLACEMENTS:
        m = random_unitary(6, rng)
        ref = oracle.apply_gate(psi0, n, qubits, m)
        got, info = run_plan(_one_gate_circuit(n, qubits, m), "c64", psi0=psi0, k_max=6, precision=prec,
                             use_tile=False)
        assert info["per_kind"] == {"tensor": 1}, info
        assert rel_l2(got, ref) < GATE_TOL[prec], (qubits, rel_l2(got, ref))


@pytest.mark.parametrize("prec", ["3xtf32", "3xbf16"])
@pytest.mark.parametrize("k", [4, 5])
def test_single_gate_padded_to_six(qs, prec, k):
    """4- and 5-qubit dense blocks are padded with the highest unused qubits
    (identity on them) and run on the 6-qubit tensor pass."""
    n = 13
    rng = Xoshiro256ss(78 + k)
    psi0 = random_state(n, 4)
    for qubits in ([0, 1, 2, 3, 4][:k], [12, 3, 7, 0, 9][:k], [11, 12, 5, 6, 1][:k]):
        m = random_unitary(k, rng)
        ref = oracle.apply_gate(psi0, n, qubits, m)
        got, info = run_plan(_one_gate_circuit(n, qubits, m), "c64", psi0=psi0, k_max=6, precision=prec,
                             use_tile=False)
        assert info["per_kind"] == {"tensor": 1}, info
        assert rel_l2(got, ref) < GATE_TOL[prec]


def test_tensor_matches_simt_fp32_path(qs):
    """Same fused k_max=6 plan: tensor-core 3xTF32 against the FP32 CUDA-core
    shared-memory GEMM, both against the oracle."""
    n = 18
    circ = C.scale_grid_circuit(n, 8, seed=5)
    ref = oracle.simulate(n, circ.gates)
    a, ia = run_plan(circ, "c64", k_max=6, precision="3xtf32")
    b, ib = run_plan(circ, "c64", k_max=6, precision="fp32")
    assert ia["per_kind"].get("tensor", 0) > 0 and ib["per_kind"].get("tensor", 0) == 0
    assert rel_l2(a, ref) < 2e-5 and rel_l2(b, ref) < 2e-5


@pytest.mark.parametrize("prec,tol", [("3xtf32", 2e-5), ("3xbf16", 2e-4), ("tf32", 2e-2)])
def test_grid_circuit_kmax6(qs, prec, tol):
    n = 20
    circ = C.scale_grid_circuit(n, 14, seed=1)
    ref = oracle.simulate(n, circ.gates)
    got, info = run_plan(circ, "c64", k_max=6, precision=prec)
    assert info["per_kind"].get("tensor", 0) > 10, info
    assert rel_l2(got, ref) < tol, rel_l2(got, ref)


def test_no_device_timeout_flag(qs):
    n = 16
    circ = C.random_circuit(n, 30, seed=9, max_k=3)
    c = B.circuit_from(circ)
    p = B.Plan(c, "c64", k_max=6, precision="3xtf32")
    s = B.State(n, "c64")
    p.execute(s)
    s.sync()   # raises QsError(status 5) if a bounded device wait had timed out


@pytest.mark.parametrize("n", [12, 13, 15, 21])
def test_tile_counts(qs, n):
    """One tile of 64 sets (n = 12), a grid smaller than the SM count, and
    several tiles per CTA (n = 21: 512 tiles on at most 152 CTAs)."""
    rng = Xoshiro256ss(90 + n)
    psi0 = random_state(n, n)
    for qubits in ([n - 1, n - 3, 6, 4, 2, 0], [n - 2, 9, 8, 5, 3, 1]):
        m = random_unitary(6, rng)
        ref = oracle.apply_gate(psi0, n, qubits, m)
        got, info = run_plan(_one_gate_circuit(n, qubits, m), "c64", psi0=psi0, k_max=6, precision="3xtf32",
                             use_tile=False)
        assert info["per_kind"] == {"tensor": 1}, info
        assert rel_l2(got, ref) < GATE_TOL["3xtf32"], (qubits, rel_l2(got, ref))


def test_below_one_tile_uses_cuda_cores(qs):
    """Fewer than 64 sets (n = 11): the planner keeps the 6-qubit block on
    the FP32 CUDA-core path."""
    n = 11
    rng = Xoshiro256ss(91)
    psi0 = random_state(n, 5)
    qubits = [10, 8, 6, 4, 2, 0]
    m = random_unitary(6, rng)
    got, info = run_plan(_one_gate_circuit(n, qubits, m), "c64", psi0=psi0, k_max=6, precision="3xtf32",
                         use_tile=False)
    assert "tensor" not in info["per_kind"], info
    assert rel_l2(got, oracle.apply_gate(psi0, n, qubits, m)) < 2e-6


@pytest.mark.parametrize("prec", ["3xtf32", "tf32", "3xbf16"])
def test_apply_circuit_streamed(qs, prec):
    """qs_apply_circuit on the tensor cores fuses and runs together (each block
    launched as the search finds it): the oracle's state, and the same state
    as a plan built from the same circuit; also on a repeat call (grouping
    cached on the circuit) and on a circuit with small remainder blocks."""
    tol = {"3xtf32": 2e-5, "tf32": 5e-3, "3xbf16": 2e-4}[prec]
    for n, cycles, seed in ((14, 6, 3), (17, 5, 4), (12, 3, 5)):
        circ = C.scale_grid_circuit(n, cycles, seed=seed)
        ref = oracle.simulate(n, circ.gates)
        c = B.circuit_from(circ)
        for _ in range(2):
            s = B.State(n, "c64")
            B.apply_circuit(s, c, prec)
            got = s.amplitudes()
            s.close()
            assert rel_l2(got, ref) < tol, (n, prec)
        p = B.Plan(c, "c64", k_max=6, precision=prec)
        s = B.State(n, "c64")
        p.execute(s)
        assert rel_l2(s.amplitudes(), ref) < tol
        s.close(); p.close(); c.close()


def test_tensor_pass_bounded_wait_timeout_is_reported(qs):
    """The tensor-core pass's bounded waits: with the testing option, one
    producer warp of the first thread block withholds its first "operand
    ready" arrival, so the MMA issuer's wait runs out (~2 s).  That block
    stops its other roles, frees its tensor memory and exits; the host reads
    QS_ERR_TIMEOUT from qs_state_sync, and a correct pass then runs on the
    same context."""
    n = 16
    rng = Xoshiro256ss(91)
    qubits = [13, 9, 7, 4, 2, 1]
    m = random_unitary(6, rng)
    psi0 = random_state(n, 5)
    c = B.circuit_from(_one_gate_circuit(n, qubits, m))
    bad = B.Plan(c, "c64", k_max=6, precision="3xtf32", use_tile=False, inject_mma_timeout=True)
    assert bad.info()["per_kind"] == {"tensor": 1}
    s = to_state(psi0, n, "c64")
    bad.execute(s)
    with pytest.raises(B.QsError) as e:
        s.sync()
    assert e.value.status == 5
    s.sync()                                  # the flag was cleared by the report
    bad.close()
    good = B.Plan(c, "c64", k_max=6, precision="3xtf32", use_tile=False)
    s2 = to_state(psi0, n, "c64")
    good.execute(s2)
    s2.sync()
    assert rel_l2(s2.amplitudes(), oracle.apply_gate(psi0, n, qubits, m)) < GATE_TOL["3xtf32"]
    good.close()
    c.close()


@pytest.mark.parametrize("scale", [1e-30, 3e-9, 1.0, 5e3, 1e25])
def test_3xfp16_scales_any_magnitude(qs, scale):
    """3xFP16 scales every set of amplitudes (and the gate) by a power of two
    into FP16's range, so states far outside it -- tiny, large, or with sets
    of very different magnitudes -- keep the split's ~22-bit accuracy."""
    n = 14
    rng = Xoshiro256ss(5)
    psi0 = random_state(n, 8) * scale
    psi0[: 1 << 7] *= 1e-6            # sets of very different magnitude within one state
    for qubits in ([13, 9, 7, 4, 2, 1], [0, 3, 5, 8, 10, 12]):
        m = random_unitary(6, rng)
        ref = oracle.apply_gate(psi0, n, qubits, m)
        got, info = run_plan(_one_gate_circuit(n, qubits, m), "c64", psi0=psi0, k_max=6, precision="3xfp16",
                             use_tile=False)
        assert info["per_kind"] == {"tensor": 1}, info
        assert rel_l2(got, ref) < GATE_TOL["3xfp16"], (scale, qubits, rel_l2(got, ref))


@pytest.mark.parametrize("prec", ["3xtf32", "3xfp16"])
def test_qubit0_kept_out_of_targets(qs, prec):
    """Runs of 6-qubit passes where several blocks touch qubit 0: the planner
    exchanges qubit 0's index bit with another qubit's inside earlier passes
    (and back), so the state between passes is stored permuted; the plan's
    result is in standard order and matches the oracle."""
    n = 16
    rng = Xoshiro256ss(17)
    circ = C.Circuit(n)
    for qs_ in ([15, 13, 9, 7, 5, 3], [0, 2, 4, 6, 8, 10], [1, 3, 11, 12, 14, 15], [0, 1, 5, 9, 13, 15],
                [2, 6, 7, 8, 12, 14], [0, 3, 4, 10, 11, 12]):
        circ.append(qs_, random_unitary(6, rng))
    psi0 = random_state(n, 23)
    ref = oracle.simulate(n, circ.gates, psi0)
    got, info = run_plan(circ, "c64", psi0=psi0, k_max=6, precision=prec, fuse=False, use_tile=False)
    assert info["per_kind"] == {"tensor": 6}, info
    assert rel_l2(got, ref) < 6 * GATE_TOL[prec], rel_l2(got, ref)


def test_low_qubit_store_forms_and_alignment(qs):
    """The pass's store forms for blocks on qubit 1 (lane pairs exchange
    values) and on qubits 0 and 1 (32-byte stores, used only when the state
    is 32-byte aligned): a torch state and a state wrapped 16 bytes into a
    larger buffer (16-byte aligned only), both against the oracle."""
    import torch
    n = 14
    rng = Xoshiro256ss(29)
    psi0 = random_state(n, 31)
    for qubits in ([1, 4, 6, 9, 11, 13], [0, 1, 5, 8, 10, 12], [1, 2, 3, 7, 8, 13], [0, 1, 2, 3, 12, 13]):
        m = random_unitary(6, rng)
        ref = oracle.apply_gate(psi0, n, qubits, m)
        circ = _one_gate_circuit(n, qubits, m)
        for offset in (0, 2):   # amplitudes (8 bytes each) into the buffer
            buf = torch.zeros((1 << n) + 4, dtype=torch.complex64, device="cuda")
            t = buf[offset:offset + (1 << n)]
            t.copy_(torch.from_numpy(psi0).to(torch.complex64))
            s = B.State(n, "c64", tensor=t, init=None)
            c = B.circuit_from(circ)
            p = B.Plan(c, "c64", k_max=6, precision="3xtf32", use_tile=False)
            p.execute(s)
            got = s.amplitudes()
            assert rel_l2(got, ref) < GATE_TOL["3xtf32"], (qubits, offset, rel_l2(got, ref))
            assert buf[:offset].abs().sum().item() == 0 and buf[offset + (1 << n):].abs().sum().item() == 0
            p.close(); c.close(); s.close()
