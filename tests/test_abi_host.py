"""The C ABI on the CPU: the library loads, exports every entry point the
header declares, rejects bad arguments with status codes, and its host-side
fusion (Sections 4.2 and 4.5) produces blocks whose product equals the
original circuit (checked with the FP64 oracle).  No device is needed."""

import os
import re

import numpy as np
import pytest

import oracle
import paper_2008_00216_gb300 as qs
from paper_2008_00216_gb300 import binding as B
from workloads import circuits as C
from workloads import gates as G
from workloads.rng import random_state

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qsgb.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\*?\s+\*?(qs_[a-z0-9_]+)\s*\(", text, re.M)))


def test_header_declares_what_the_binding_uses():
    decl = declared_symbols()
    assert len(decl) >= 30
    assert set(B.exported_symbols()) <= set(decl)


def test_library_exports_every_declared_symbol():
    lib = qs.load()
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_status_strings_and_version():
    lib = qs.load()
    assert b"sm_103a" in lib.qs_version()
    for s in range(7):
        assert lib.qs_status_string(s)


@pytest.mark.parametrize("qubits,k", [([0, 0], 2), ([12], 1), ([-1], 1), ([0, 1, 2, 3, 4, 5, 6], 7)])
def test_circuit_add_rejects_bad_gates(qubits, k):
    c = B.Circuit(12)
    m = np.eye(1 << min(k, 6), dtype=complex)
    with pytest.raises(B.QsError) as e:
        B._call("qs_circuit_add", c.handle, B._ints(qubits), k, B._mat(m))
    assert e.value.status == 1


def test_circuit_add_gates_matches_single_adds():
    """qs_circuit_add_gates appends the same gates (qubits, matrix, kind) as
    one qs_circuit_add per gate, rotations in between included."""
    circ = C.scale_grid_circuit(14, 4, seed=3)
    batched = B.circuit_from(circ)
    single = B.Circuit(14)
    for g in circ.gates:
        single.add(g)
    a, b = batched.gates(), single.gates()
    assert len(a) == len(b) == len(circ.gates)
    for x, y in zip(a, b):
        assert x[0] == y[0] and x[2] == y[2]
        assert np.array_equal(x[1], y[1])
    theta = C.ansatz_theta(6, 2, seed=1)
    spec = C.ansatz_circuit(6, 2, theta)
    spec.theta = theta
    mixed = B.circuit_from(spec)
    assert mixed.size() == (6, len(spec.gates), theta.size)


def test_circuit_add_gates_is_all_or_nothing():
    c = B.Circuit(12)
    ks = [1, 2, 1]
    qubits = [0, 3, 4, 12]            # the third gate's qubit is out of range
    mats = np.concatenate([np.eye(2).ravel(), np.eye(4).ravel(), np.eye(2).ravel()]).astype(complex)
    with pytest.raises(B.QsError) as e:
        B._call("qs_circuit_add_gates", c.handle, 3, B._ints(ks), B._ints(qubits),
                B._dbl(np.stack([mats.real, mats.imag], axis=-1)))
    assert e.value.status == 1
    assert c.size()[1] == 0
    with pytest.raises(B.QsError):
        B._call("qs_circuit_add_gates", c.handle, 1, B._ints([7]), B._ints([0]), B._dbl(np.zeros(2)))
    assert c.size()[1] == 0


def test_fuse_rejects_bad_kmax():
    c = B.circuit_from(C.small_grid_circuit())
    for k in (0, 7):
        with pytest.raises(B.QsError):
            B.fuse(c, k)


def test_rotation_matrix_roundtrip():
    circ = C.ansatz_circuit(3, 1, C.ansatz_theta(3, 1, seed=2))
    c = B.circuit_from(circ)
    for i, g in enumerate(circ.gates):
        qs_, m, kind = c.gate(i)
        assert qs_ == g.qubits
        assert np.max(np.abs(m - g.matrix)) < 1e-15


def test_gate_classification():
    c = B.Circuit(4, [((0, 1), G.CZ), ((2,), G.SQRT_X), ((1, 3), G.fsim(np.pi / 2, 0.3)), ((0,), G.T)])
    kinds = [c.gate(i)[2] for i in range(4)]
    assert kinds == ["diagonal", "dense", "monomial", "diagonal"]


def _oracle_of(circ_obj):
    return [(q, m) for q, m, _ in circ_obj.gates()]


@pytest.mark.parametrize("k_max", [1, 2, 3, 4, 5, 6])
def test_fusion_preserves_the_circuit(k_max):
    circ = C.grid_circuit(10, 6, seed=3)
    c = B.circuit_from(circ)
    f = B.fuse(c, k_max)
    blocks = f.gates()
    assert all(len(q) <= max(k_max, 2) for q, _, _ in blocks)  # wider gates pass through
    if k_max > 1:
        assert len(blocks) < len(circ.gates)
    psi0 = random_state(10, 1)
    ref = oracle.simulate(10, circ.gates, psi0)
    got = oracle.simulate(10, _oracle_of(f), psi0)
    assert oracle.metrics.rel_l2(got, ref) < 1e-13


def test_fusion_reorders_commuting_diagonals():
    # CZ(0,1), H(2), CZ(1,2) cannot merge directly, but CZ(0,1) and a later
    # CZ(0,3) commute with the skipped diagonal, so they join one block
    gates = [((0, 1), G.CZ), ((1, 2), G.CZ), ((2,), G.H), ((0, 3), G.CZ), ((3, 4), G.CZ)]
    c = B.Circuit(5, gates)
    f = B.fuse(c, 3)
    blocks = f.gates()
    psi0 = random_state(5, 2)
    assert oracle.metrics.rel_l2(oracle.simulate(5, _oracle_of(f), psi0), oracle.simulate(5, gates, psi0)) < 1e-14
    assert len(blocks) <= 3


def test_fusion_random_circuits_all_kinds():
    for seed in range(4):
        circ = C.random_circuit(8, 50, seed, max_k=3)
        c = B.circuit_from(circ)
        for k_max in (3, 4, 6):
            f = B.fuse(c, k_max)
            psi0 = random_state(8, seed)
            assert oracle.metrics.rel_l2(oracle.simulate(8, _oracle_of(f), psi0),
                                         oracle.simulate(8, circ.gates, psi0)) < 1e-13


def test_fused_block_kinds_are_exact():
    # a block of only diagonal gates must come out diagonal
    gates = [((0, 1), G.CZ), ((1,), G.T), ((0,), G.S), ((1, 2), G.cphase(0.3))]
    f = B.fuse(B.Circuit(3, gates), 3)
    assert [k for _, _, k in f.gates()] == ["diagonal"]


@pytest.mark.parametrize("k_max", [2, 4, 6])
def test_block_search_preserves_circuits_with_commuting_runs(k_max):
    """The block search moves gates past commuting ones (disjoint qubits, or
    diagonal past diagonal): circuits rich in such runs -- the paper's gate
    set (CZ and T layers), the ansatz (RZ and CZ layers), a diagonal-heavy
    random mix -- fuse to the same operator (FP64 oracle, 1e-13)."""
    n = 10
    circs = [C.paper_circuit(n, 8, seed=2), C.ansatz_circuit(n, 3, C.ansatz_theta(n, 3, seed=4)),
             C.grid_circuit(n, 8, seed=5)]
    rng = np.random.default_rng(7)
    gates = []
    for _ in range(120):
        a, b = rng.choice(n, 2, replace=False)
        r = rng.random()
        if r < 0.4:
            gates.append(((int(a), int(b)), G.CZ))
        elif r < 0.6:
            gates.append(((int(a),), G.T))
        elif r < 0.8:
            gates.append(((int(a), int(b)), G.cphase(float(rng.random()))))
        else:
            gates.append(((int(a),), G.SQRT_X if r < 0.9 else G.H))
    for circ in circs + [gates]:
        glist = circ if isinstance(circ, list) else circ.gates
        c = B.Circuit(n, glist) if isinstance(circ, list) else B.circuit_from(circ)
        f = B.fuse(c, k_max)
        assert all(len(q) <= max(k_max, 2) for q, _, _ in f.gates())
        psi0 = random_state(n, 11)
        ref = oracle.simulate(n, glist if isinstance(circ, list) else circ.gates, psi0)
        assert oracle.metrics.rel_l2(oracle.simulate(n, _oracle_of(f), psi0), ref) < 1e-13


def test_options_fusion_effort():
    """qs_options_default selects the block search with the lookahead step;
    an effort outside {0, 1} is rejected before any device work."""
    o = B.options()
    assert o.fusion_effort == 1 and o.k_max == 4 and o.fuse == 1
    assert B.options(fusion_effort=0).fusion_effort == 0
    c = B.circuit_from(C.small_grid_circuit())
    for bad in (-1, 2):
        with pytest.raises(B.QsError) as ei:
            B.Plan(c, "c64", opts=B.options(fusion_effort=bad))
        assert ei.value.status == 1  # QS_ERR_ARG


def test_norm_noalloc_binding_checks_the_tensor():
    """qs_norm_noalloc only receives a pointer, so the binding checks the
    tensor before the call: too few amplitudes for n, or a dtype other than
    the state's, raise before anything reaches the library."""
    import torch
    t = torch.zeros(8, dtype=torch.complex64)
    with pytest.raises(ValueError, match="amplitudes"):
        B.norm_noalloc(t, 4, "c64")                     # 8 amplitudes, n = 4 needs 16
    with pytest.raises(ValueError, match="dtype"):
        B.norm_noalloc(t, 3, "c128")                    # complex64 data read as complex128
    with pytest.raises(ValueError, match="contiguous"):
        B.norm_noalloc(torch.zeros(16, dtype=torch.complex64)[::2], 3, "c64")
    with pytest.raises(ValueError, match="CUDA"):
        B.norm_noalloc(t, 3, "c64")                     # right size and dtype, but host memory
