"""The complex64 block adjoint sweep's host logic, without a GPU.

The library's planner runs as it does before a GPU sweep (fusion groups,
block products, each block's Gram qubits and its gates as recursion records
in Gram coordinates, diagonal runs merged), and `tests/cpp/block_sweep_emulate.cpp`
redoes the device steps in FP64: per block, last first, the Gram matrix
M = sum_s psi_s lambda_s^dagger over its six qubits, the gradient kernel's
walk over the block's records, then B^dagger on both states.  Its inputs
psi = U|0> and lambda = H psi come from the FP64 oracle; its gradients must
equal exact parameter shift on the oracle (to the complex64 gate matrices'
rounding, which the records carry), with exactly one gradient record per
parameter.  Two circuits: blocks with every kind of target placement, and
the benchmark's layered ansatz."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import paper_2008_00216_gb300 as qs
from paper_2008_00216_gb300 import _build
from workloads import circuits as C
from workloads import gates as G
from workloads.rng import Xoshiro256ss

HERE = os.path.dirname(os.path.abspath(__file__))
SETS = [(0, 3, 5, 7, 9, 11), (0, 1, 2, 6, 8, 12), (1, 4, 6, 8, 10, 12), (7, 8, 9, 10, 11, 12)]


def block_circuit(n, reps, theta):
    circ = C.Circuit(n)
    p = 0

    def rot(qubits, gen):
        nonlocal p
        circ.append(qubits, G.pauli_rotation(gen, theta[p]), gen, p, gen)
        p += 1

    for r in range(reps):
        for k, S in enumerate(SETS):
            for i, q in enumerate(S):
                rot((q,), "XYZ"[(i + r + k) % 3])
                rot((q,), "Z")
            for a, b in zip(S, S[1:]):
                circ.append((a, b), G.CZ, "cz")
            rot((S[0], S[-1]), "ZZ")
            rot((S[1], S[2]), "XY")
            circ.append((S[3],), G.SQRT_X if (r + k) % 2 else G.H, "fixed")
    circ.num_params = p
    return circ


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    home = os.path.dirname(os.path.dirname(nvcc))
    return home if os.path.exists(os.path.join(home, "include", "cuda_runtime.h")) else None


def _compile(tmp):
    cuda = _cuda_home()
    if cuda is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    qs.load()  # builds the library if needed
    exe = os.path.join(tmp, "block_sweep_emulate")
    lib = os.path.dirname(_build.LIB)
    cmd = ["g++", "-O2", "-std=c++17", "-w", "-I", os.path.join(HERE, "..", "paper_2008_00216_gb300", "csrc"),
           "-I", _build.INCLUDE, "-I", os.path.join(cuda, "include"),
           os.path.join(HERE, "cpp", "block_sweep_emulate.cpp"), "-o", exe,
           "-L", lib, "-lqsgb", "-L", os.path.join(cuda, "lib64"), "-lcudart",
           f"-Wl,-rpath,{lib}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def _ansatz(n, layers, theta):
    circ = C.ansatz_circuit(n, layers, theta)
    circ.num_params = C.ansatz_num_params(n, layers)
    return circ


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    return _compile(str(tmp_path_factory.mktemp("emu")))


@pytest.mark.parametrize("case", ["placements", "ansatz", "ansatz-known-blocks"])
def test_block_sweep_host_logic_matches_parameter_shift(tmp_path, emulator, case):
    if case == "placements":
        n, make = 13, (lambda t: block_circuit(13, 2, t))
        P = make(np.zeros(100000)).num_params
    else:  # the benchmark's layered ansatz (RY, RZ, CZ chain); "known": blocks formed beforehand
        n, make = 12, (lambda t: _ansatz(12, 3, t))
        P = C.ansatz_num_params(12, 3)
    rng = Xoshiro256ss(727)
    theta = np.array([rng.uniform_range(-np.pi, np.pi) for _ in range(P)])
    terms = C.ising_hamiltonian(n) + [C.PauliTerm(0.5, ((2, "Y"), (n - 1, "X"))),
                                      C.PauliTerm(0.3, ((0, "Z"), (7, "Y")))]
    circ = make(theta)
    psi = oracle.simulate(n, circ.gates)
    lam = oracle.apply_pauli_sum(psi, n, terms)
    tmp = str(tmp_path)
    lines = [str(n)]
    for g in circ.gates:
        k = len(g.qubits)
        head = f"{k} " + " ".join(str(q) for q in g.qubits)
        if g.param >= 0:
            lines.append(f"R {head} {g.param} {g.generator} {float(theta[g.param])!r}")
        else:
            m = np.asarray(g.matrix, dtype=np.complex128).reshape(-1)
            lines.append(f"F {head} " + " ".join(repr(float(v)) for z in m for v in (z.real, z.imag)))
    with open(os.path.join(tmp, "circuit.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    psi.astype(np.complex128).tofile(os.path.join(tmp, "psi.bin"))
    lam.astype(np.complex128).tofile(os.path.join(tmp, "lam.bin"))
    args = [emulator, os.path.join(tmp, "circuit.txt"), os.path.join(tmp, "psi.bin"), os.path.join(tmp, "lam.bin")]
    if case.endswith("known-blocks"):
        args.append("known")
    r = subprocess.run(args, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    g = np.array([float(x) for x in r.stdout.split()])
    assert g.shape == (P,)
    ps = oracle.parameter_shift_gradient(n, lambda t: make(t).gates, theta, terms)
    # the records carry complex64 gate matrices: agreement to their rounding
    assert np.max(np.abs(g - ps)) < 1e-5 * max(1.0, np.max(np.abs(ps))), np.max(np.abs(g - ps))
