"""Thin Python binding of the C ABI in include/qsgb.h.

Argument marshalling only: every operation on amplitudes runs in the CUDA
library.  PyTorch provides device memory (states are torch complex tensors
wrapped with qs_state_wrap) and the current CUDA stream.  There is no CPU
fallback: if the shared library cannot be loaded, every call raises.
"""

from __future__ import annotations

import ctypes as ct
import os
from typing import Iterable, Optional, Sequence

import numpy as np

from . import _build

_lib = None

QS_C64, QS_C128 = 0, 1
QS_PREC_FP32, QS_PREC_TF32, QS_PREC_3XTF32, QS_PREC_3XBF16, QS_PREC_3XFP16 = 0, 1, 2, 3, 4
PRECISIONS = {"fp32": 0, "tf32": 1, "3xtf32": 2, "3xbf16": 3, "3xfp16": 4}
GATE_KINDS = {0: "dense", 1: "diagonal", 2: "monomial"}
PASS_KINDS = ["tile", "dense", "diagonal", "monomial", "tensor", "dense_smem", "diagonal_wide", "tensor_tile"]


class QsError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func} failed with status {status}: {msg}")
        self.status = status


class Options(ct.Structure):
    _fields_ = [("k_max", ct.c_int), ("tile_qubits", ct.c_int), ("use_tile", ct.c_int),
                ("precision", ct.c_int), ("fuse", ct.c_int), ("inject_wait_timeout", ct.c_int),
                ("diag_clusters", ct.c_int), ("fusion_effort", ct.c_int), ("inject_mma_timeout", ct.c_int),
                ("tensor_tiles", ct.c_int), ("reserved", ct.c_int * 3)]


_P = ct.c_void_p
_SIGS = {
    "qs_version": (ct.c_char_p, []),
    "qs_status_string": (ct.c_char_p, [ct.c_int]),
    "qs_last_error": (ct.c_char_p, []),
    "qs_options_default": (ct.c_int, [ct.POINTER(Options)]),
    "qs_state_create": (ct.c_int, [ct.c_int, ct.c_int, _P, ct.POINTER(_P)]),
    "qs_state_wrap": (ct.c_int, [_P, ct.c_int, ct.c_int, _P, ct.POINTER(_P)]),
    "qs_state_destroy": (ct.c_int, [_P]),
    "qs_state_set_stream": (ct.c_int, [_P, _P]),
    "qs_state_info": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(_P)]),
    "qs_state_init_basis": (ct.c_int, [_P, ct.c_uint64]),
    "qs_state_init_uniform": (ct.c_int, [_P]),
    "qs_state_copy": (ct.c_int, [_P, _P]),
    "qs_state_sync": (ct.c_int, [_P]),
    "qs_apply_gate": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.c_int, ct.POINTER(ct.c_double)]),
    "qs_circuit_create": (ct.c_int, [ct.c_int, ct.POINTER(_P)]),
    "qs_circuit_destroy": (ct.c_int, [_P]),
    "qs_circuit_add": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.c_int, ct.POINTER(ct.c_double)]),
    "qs_circuit_add_gates": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                        ct.POINTER(ct.c_double)]),
    "qs_circuit_add_rotation": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.c_int, ct.c_char_p, ct.c_int,
                                           ct.c_double]),
    "qs_circuit_set_params": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.c_int]),
    "qs_circuit_size": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "qs_circuit_gate": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                   ct.POINTER(ct.c_double), ct.POINTER(ct.c_int)]),
    "qs_fuse": (ct.c_int, [_P, ct.c_int, ct.POINTER(_P)]),
    "qs_plan_create": (ct.c_int, [_P, ct.c_int, ct.POINTER(Options), ct.POINTER(_P)]),
    "qs_plan_destroy": (ct.c_int, [_P]),
    "qs_plan_info": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "qs_plan_execute": (ct.c_int, [_P, _P]),
    "qs_plan_execute_range": (ct.c_int, [_P, _P, ct.c_int, ct.c_int]),
    "qs_plan_pass": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "qs_apply_circuit": (ct.c_int, [_P, _P, ct.c_int]),
    "qs_amplitudes": (ct.c_int, [_P, ct.c_uint64, ct.c_uint64, ct.POINTER(ct.c_double)]),
    "qs_norm": (ct.c_int, [_P, ct.POINTER(ct.c_double)]),
    "qs_norm_noalloc": (ct.c_int, [_P, ct.c_int, ct.c_int, _P, ct.POINTER(ct.c_double)]),
    "qs_pauli_sum_create": (ct.c_int, [ct.c_int, ct.POINTER(_P)]),
    "qs_pauli_sum_destroy": (ct.c_int, [_P]),
    "qs_pauli_sum_add": (ct.c_int, [_P, ct.c_double, ct.POINTER(ct.c_int), ct.c_char_p, ct.c_int]),
    "qs_expectation": (ct.c_int, [_P, _P, ct.POINTER(ct.c_double)]),
    "qs_apply_pauli_sum": (ct.c_int, [_P, _P, _P]),
    "qs_adjoint_gradient": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.c_int, _P, _P, _P,
                                       ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]),
    "qs_adjoint_gradient_batch": (ct.c_int, [ct.c_int, ct.POINTER(_P), ct.POINTER(ct.POINTER(ct.c_double)),
                                             ct.POINTER(ct.c_int), ct.POINTER(_P), ct.POINTER(_P), ct.POINTER(_P),
                                             ct.POINTER(ct.c_double), ct.POINTER(ct.POINTER(ct.c_double))]),
    "qs_batch_create": (ct.c_int, [ct.POINTER(_P), ct.c_int, ct.c_int, ct.POINTER(Options), ct.POINTER(_P)]),
    "qs_batch_layout": (ct.c_int, [_P, ct.POINTER(ct.c_uint64)]),
    "qs_batch_info": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                 ct.POINTER(ct.c_int)]),
    "qs_batch_run": (ct.c_int, [_P, _P, _P]),
    "qs_batch_sync": (ct.c_int, [_P]),
    "qs_batch_destroy": (ct.c_int, [_P]),
    "qs_batch_autotune": (ct.c_int, [ct.POINTER(_P), ct.c_int, ct.c_int, _P, _P, ct.POINTER(Options)]),
    "qs_sf_amplitudes": (ct.c_int, [_P, ct.c_uint64, ct.c_int, ct.POINTER(ct.c_uint64), ct.c_uint64, _P,
                                    ct.POINTER(ct.c_double), ct.POINTER(ct.c_uint64)]),
}


def exported_symbols() -> list:
    """Every entry point this binding expects the library to export."""
    return sorted(_SIGS)


def load(path: Optional[str] = None):
    """Load the shared library (building it first if the sources are newer).
    Raises if it cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.LIB if _build.up_to_date() else _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    lib = ct.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _call(name: str, *args):
    lib = load()
    st = getattr(lib, name)(*args)
    if st != 0:
        raise QsError(st, name, lib.qs_last_error().decode())
    return st


def _dbl(a) -> ct.Array:
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    return (ct.c_double * a.size).from_buffer_copy(a.tobytes()) if a.size else (ct.c_double * 1)()


def _mat(m) -> ct.Array:
    m = np.asarray(m, dtype=np.complex128)
    return _dbl(np.stack([m.real, m.imag], axis=-1))


def _ints(q) -> ct.Array:
    q = [int(x) for x in q]
    return (ct.c_int * max(1, len(q)))(*q)


def _stream_ptr(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def options(k_max: int = 4, tile_qubits: int = 0, use_tile: bool = True, precision="fp32",
            fuse: bool = True, inject_wait_timeout: bool = False, diag_clusters: bool = False,
            fusion_effort: int = 1, inject_mma_timeout: bool = False, tensor_tiles: bool = False) -> Options:
    o = Options()
    _call("qs_options_default", ct.byref(o))
    o.inject_wait_timeout = 1 if inject_wait_timeout else 0
    o.inject_mma_timeout = 1 if inject_mma_timeout else 0
    o.tensor_tiles = 1 if tensor_tiles else 0
    o.diag_clusters = 1 if diag_clusters else 0
    o.fusion_effort = int(fusion_effort)
    o.k_max = int(k_max)
    o.tile_qubits = int(tile_qubits)
    o.use_tile = 1 if use_tile else 0
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.fuse = 1 if fuse else 0
    return o


# ---------------------------------------------------------------------- state

class State:
    """A state of 2^n amplitudes in a torch complex64/complex128 CUDA tensor,
    wrapped by the library (qs_state_wrap).  `tensor` is the storage."""

    def __init__(self, n: int, dtype="c64", tensor=None, stream=None, init: str = "zero"):
        import torch
        self.n = int(n)
        self.dtype = dtype
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        if tensor is None:
            tensor = torch.empty(1 << self.n, dtype=tdt, device="cuda")
        if tensor.dtype != tdt or tensor.numel() != (1 << self.n) or not tensor.is_cuda:
            raise ValueError("tensor must be a CUDA tensor of 2^n amplitudes of the state dtype")
        if not tensor.is_contiguous():
            raise ValueError("tensor must be contiguous")
        self.tensor = tensor
        self._stream = stream
        h = ct.c_void_p()
        _call("qs_state_wrap", ct.c_void_p(tensor.data_ptr()), self.n, QS_C64 if dtype == "c64" else QS_C128,
              ct.c_void_p(_stream_ptr(stream)), ct.byref(h))
        self.handle = h
        if init == "zero":
            self.init_basis(0)
        elif init == "uniform":
            self.init_uniform()

    def sync_stream(self):
        _call("qs_state_set_stream", self.handle, ct.c_void_p(_stream_ptr(self._stream)))

    def init_basis(self, index: int = 0):
        self.sync_stream()
        _call("qs_state_init_basis", self.handle, ct.c_uint64(index))

    def init_uniform(self):
        self.sync_stream()
        _call("qs_state_init_uniform", self.handle)

    def sync(self):
        """Wait for the stream; raises QsError (status 5) if a device wait timed out."""
        self.sync_stream()
        _call("qs_state_sync", self.handle)

    def copy_from(self, other: "State"):
        self.sync_stream()
        _call("qs_state_copy", self.handle, other.handle)

    def amplitudes(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        count = (1 << self.n) - first if count is None else count
        out = np.empty(2 * count, dtype=np.float64)
        self.sync_stream()
        _call("qs_amplitudes", self.handle, ct.c_uint64(first), ct.c_uint64(count),
              out.ctypes.data_as(ct.POINTER(ct.c_double)))
        return out.view(np.complex128)

    def norm(self) -> float:
        v = ct.c_double()
        self.sync_stream()
        _call("qs_norm", self.handle, ct.byref(v))
        return v.value

    def close(self):
        if getattr(self, "handle", None):
            load().qs_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def norm_noalloc(tensor, n: int, dtype="c64", stream=None) -> float:
    """sum |alpha|^2 of a raw CUDA tensor through qs_norm_noalloc, which
    allocates no device memory (for callers that cannot allocate).  The C
    entry point only sees a pointer, so the tensor is checked here: the
    state dtype, exactly 2^n contiguous amplitudes, on a CUDA device (the
    call runs with that device current)."""
    import torch
    if dtype not in ("c64", "c128"):
        raise ValueError("dtype must be 'c64' or 'c128'")
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    if tensor.dtype != tdt:
        raise ValueError(f"tensor dtype {tensor.dtype} does not match the state dtype {dtype}")
    if not 1 <= int(n) <= 40 or tensor.numel() != (1 << int(n)):
        raise ValueError(f"tensor holds {tensor.numel()} amplitudes, not 2^{n}")
    if not tensor.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if not tensor.is_cuda:
        raise ValueError("tensor must be a CUDA tensor")
    v = ct.c_double()
    with torch.cuda.device(tensor.device):
        _call("qs_norm_noalloc", ct.c_void_p(tensor.data_ptr()), int(n), QS_C64 if dtype == "c64" else QS_C128,
              ct.c_void_p(_stream_ptr(stream)), ct.byref(v))
    return v.value


def apply_gate(state: State, qubits: Sequence[int], matrix):
    k = len(qubits)
    state.sync_stream()
    _call("qs_apply_gate", state.handle, _ints(qubits), k, _mat(matrix))


# ---------------------------------------------------------------------- circuits

class Circuit:
    """Host gate list (qs_circuit).  Build from gates with .qubits/.matrix
    (and optional .param/.generator for rotations exp(-i theta P / 2))."""

    def __init__(self, n: int, gates: Iterable = (), handle=None):
        self.n = int(n)
        if handle is None:
            h = ct.c_void_p()
            _call("qs_circuit_create", self.n, ct.byref(h))
            handle = h
        self.handle = handle
        fixed = []  # runs of fixed gates go to the library in one call
        for g in gates:
            param = getattr(g, "param", -1)
            if param is not None and param >= 0:
                self.add_many(fixed)
                fixed = []
                self.add(g)
            else:
                fixed.append(g)
        self.add_many(fixed)

    def add_many(self, gates):
        """Append fixed gates with one library call (qs_circuit_add_gates)."""
        if not gates:
            return
        ks, qubits, mats = [], [], []
        for g in gates:
            qs = g.qubits if hasattr(g, "qubits") else g[0]
            m = np.asarray(g.matrix if hasattr(g, "matrix") else g[1], dtype=np.complex128)
            ks.append(len(qs))
            qubits.extend(int(x) for x in qs)
            mats.append(m.ravel())
        flat = np.concatenate(mats)
        _call("qs_circuit_add_gates", self.handle, len(ks), _ints(ks), _ints(qubits),
              _dbl(np.stack([flat.real, flat.imag], axis=-1)))

    def add(self, g):
        qs = g.qubits if hasattr(g, "qubits") else g[0]
        param = getattr(g, "param", -1)
        if param is not None and param >= 0:
            theta = 0.0
            _call("qs_circuit_add_rotation", self.handle, _ints(qs), len(qs), g.generator.encode(), int(param),
                  ct.c_double(theta))
        else:
            m = g.matrix if hasattr(g, "matrix") else g[1]
            _call("qs_circuit_add", self.handle, _ints(qs), len(qs), _mat(m))

    def set_params(self, theta):
        theta = np.asarray(theta, dtype=np.float64)
        _call("qs_circuit_set_params", self.handle, _dbl(theta), int(theta.size))

    def size(self):
        n, g, p = ct.c_int(), ct.c_int(), ct.c_int()
        _call("qs_circuit_size", self.handle, ct.byref(n), ct.byref(g), ct.byref(p))
        return n.value, g.value, p.value

    def gate(self, i: int):
        k = ct.c_int()
        qs = (ct.c_int * 6)()
        m = (ct.c_double * (2 * 64 * 64))()
        kind = ct.c_int()
        _call("qs_circuit_gate", self.handle, int(i), ct.byref(k), qs, m, ct.byref(kind))
        d = 1 << k.value
        mat = np.frombuffer(m, dtype=np.float64, count=2 * d * d).copy().view(np.complex128).reshape(d, d)
        return tuple(qs[:k.value]), mat, GATE_KINDS[kind.value]

    def gates(self):
        return [self.gate(i) for i in range(self.size()[1])]

    def close(self):
        if getattr(self, "handle", None):
            load().qs_circuit_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def circuit_from(circ) -> Circuit:
    """Circuit from any object with .n and .gates; parametrised gates get the
    parameter values in circ.theta when present."""
    c = Circuit(circ.n, circ.gates)
    theta = getattr(circ, "theta", None)
    if theta is not None and c.size()[2] > 0:
        c.set_params(theta)
    return c


def fuse(circ: Circuit, k_max: int) -> Circuit:
    h = ct.c_void_p()
    _call("qs_fuse", circ.handle, int(k_max), ct.byref(h))
    return Circuit(circ.n, handle=h)


class Plan:
    def __init__(self, circ: Circuit, dtype="c64", opts: Optional[Options] = None, **kw):
        self.n = circ.n
        self.dtype = dtype
        opts = opts if opts is not None else options(**kw)
        h = ct.c_void_p()
        _call("qs_plan_create", circ.handle, QS_C64 if dtype == "c64" else QS_C128, ct.byref(opts), ct.byref(h))
        self.handle = h

    def info(self):
        npass, nl = ct.c_int(), ct.c_int()
        kinds = (ct.c_int * 8)()
        _call("qs_plan_info", self.handle, ct.byref(npass), ct.byref(nl), kinds)
        return {"passes": npass.value, "launches": nl.value,
                "per_kind": {PASS_KINDS[i]: kinds[i] for i in range(8) if kinds[i]}}

    def execute(self, state: State):
        state.sync_stream()
        _call("qs_plan_execute", state.handle, self.handle)

    def execute_range(self, state: State, first: int, count: int = 1):
        state.sync_stream()
        _call("qs_plan_execute_range", state.handle, self.handle, int(first), int(count))

    def passes(self):
        out = []
        for i in range(self.info()["passes"]):
            kind, width, ng = ct.c_int(), ct.c_int(), ct.c_int()
            _call("qs_plan_pass", self.handle, i, ct.byref(kind), ct.byref(width), ct.byref(ng))
            out.append((PASS_KINDS[kind.value], width.value, ng.value))
        return out

    def close(self):
        if getattr(self, "handle", None):
            load().qs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apply_circuit(state: State, circ: Circuit, precision="fp32"):
    state.sync_stream()
    _call("qs_apply_circuit", state.handle, circ.handle, PRECISIONS[precision])


# ---------------------------------------------------------------------- observables

class PauliSum:
    """sum_t c_t P_t; terms as (coeff, ((qubit, 'X'|'Y'|'Z'), ...)) or objects
    with .coeff and .ops."""

    def __init__(self, n: int, terms: Iterable = ()):
        self.n = int(n)
        h = ct.c_void_p()
        _call("qs_pauli_sum_create", self.n, ct.byref(h))
        self.handle = h
        for t in terms:
            coeff, ops = (t.coeff, t.ops) if hasattr(t, "ops") else t
            qs = [q for q, _ in ops]
            ps = "".join(p for _, p in ops)
            _call("qs_pauli_sum_add", self.handle, ct.c_double(coeff), _ints(qs), ps.encode(), len(qs))

    def close(self):
        if getattr(self, "handle", None):
            load().qs_pauli_sum_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def expectation(state: State, h: PauliSum) -> float:
    v = ct.c_double()
    state.sync_stream()
    _call("qs_expectation", state.handle, h.handle, ct.byref(v))
    return v.value


def apply_pauli_sum(state: State, h: PauliSum, out: State):
    out.sync_stream()
    _call("qs_apply_pauli_sum", state.handle, h.handle, out.handle)


def adjoint_gradient(circ: Circuit, theta, h: PauliSum, psi: State, lam: State):
    theta = np.asarray(theta, dtype=np.float64)
    e = ct.c_double()
    g = np.zeros(theta.size, dtype=np.float64)
    psi.sync_stream()
    lam.sync_stream()
    _call("qs_adjoint_gradient", circ.handle, _dbl(theta), int(theta.size), h.handle, psi.handle, lam.handle,
          ct.byref(e), g.ctypes.data_as(ct.POINTER(ct.c_double)))
    return e.value, g


def adjoint_gradient_batch(circs: Sequence[Circuit], thetas, hams: Sequence[PauliSum], psis: Sequence[State],
                           lams: Sequence[State]):
    """Gradients of many circuits at once (qs_adjoint_gradient_batch).  Give
    each (psi, lam) pair its own stream (State(..., stream=...)) so their work
    overlaps.  Returns (energies, list of gradient arrays)."""
    k = len(circs)
    if not (len(thetas) == len(hams) == len(psis) == len(lams) == k):
        raise ValueError("all sequences need one entry per gradient")
    th = [np.ascontiguousarray(t, dtype=np.float64) for t in thetas]
    grads = [np.zeros(t.size, dtype=np.float64) for t in th]
    DP = ct.POINTER(ct.c_double)
    for s in list(psis) + list(lams):
        s.sync_stream()
    energies = np.zeros(k, dtype=np.float64)
    _call("qs_adjoint_gradient_batch", k, (_P * k)(*[c.handle for c in circs]),
          (DP * k)(*[t.ctypes.data_as(DP) for t in th]), (ct.c_int * k)(*[t.size for t in th]),
          (_P * k)(*[h.handle for h in hams]), (_P * k)(*[s.handle for s in psis]),
          (_P * k)(*[s.handle for s in lams]), energies.ctypes.data_as(DP),
          (DP * k)(*[g.ctypes.data_as(DP) for g in grads]))
    return energies, grads


# ---------------------------------------------------------------------- batches

class Batch:
    """Many circuits in one persistent launch (qs_batch_*).  `states` is one
    torch tensor holding every circuit's final state at `offsets[i]`."""

    def __init__(self, circuits: Sequence[Circuit], dtype="c64", opts: Optional[Options] = None, **kw):
        import torch
        self.circuits = list(circuits)
        self.dtype = dtype
        arr = (ct.c_void_p * len(self.circuits))(*[c.handle.value for c in self.circuits])
        opts = opts if opts is not None else options(**({"k_max": 3} | kw))
        h = ct.c_void_p()
        _call("qs_batch_create", arr, len(self.circuits), QS_C64 if dtype == "c64" else QS_C128, ct.byref(opts),
              ct.byref(h))
        self.handle = h
        offs = (ct.c_uint64 * (len(self.circuits) + 1))()
        _call("qs_batch_layout", self.handle, offs)
        self.offsets = [int(x) for x in offs]
        tdt = torch.complex64 if dtype == "c64" else torch.complex128
        self.states = torch.empty(self.offsets[-1], dtype=tdt, device="cuda")

    def info(self):
        v = [ct.c_int() for _ in range(4)]
        _call("qs_batch_info", self.handle, *[ct.byref(x) for x in v])
        return dict(zip(("items", "passes", "gates", "grid"), (x.value for x in v)))

    def run(self, stream=None):
        _call("qs_batch_run", self.handle, ct.c_void_p(self.states.data_ptr()), ct.c_void_p(_stream_ptr(stream)))

    def sync(self):
        _call("qs_batch_sync", self.handle)

    def state(self, i: int):
        return self.states[self.offsets[i]:self.offsets[i + 1]]

    def close(self):
        if getattr(self, "handle", None):
            load().qs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_autotune(circuits: Sequence[Circuit], dtype="c64", stream=None) -> Options:
    """Fastest (k_max, tile width) for this batch, by timing each candidate."""
    import torch
    probe = Batch(circuits, dtype)
    arr = (ct.c_void_p * len(probe.circuits))(*[c.handle.value for c in probe.circuits])
    best = Options()
    _call("qs_batch_autotune", arr, len(probe.circuits), QS_C64 if dtype == "c64" else QS_C128,
          ct.c_void_p(probe.states.data_ptr()), ct.c_void_p(_stream_ptr(stream)), ct.byref(best))
    probe.close()
    return best


def sf_amplitudes(circ: Circuit, part_a: Sequence[int], indices, dtype="c64", stream=None):
    """Amplitudes at `indices` by the Schroedinger-Feynman mode
    (qs_sf_amplitudes): qubits `part_a` form one half, the rest the other.
    Returns (complex128 array, number of paths)."""
    mask = 0
    for q in part_a:
        mask |= 1 << int(q)
    idx = np.ascontiguousarray(np.asarray(indices, dtype=np.uint64).ravel())
    out = np.zeros(2 * max(1, idx.size), dtype=np.float64)
    paths = ct.c_uint64()
    _call("qs_sf_amplitudes", circ.handle, ct.c_uint64(mask), QS_C64 if dtype == "c64" else QS_C128,
          idx.ctypes.data_as(ct.POINTER(ct.c_uint64)), ct.c_uint64(idx.size), ct.c_void_p(_stream_ptr(stream)),
          out.ctypes.data_as(ct.POINTER(ct.c_double)), ct.byref(paths))
    return out[:2 * idx.size].view(np.complex128), int(paths.value)


def version() -> str:
    return load().qs_version().decode()
