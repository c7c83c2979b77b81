#!/usr/bin/env python
"""Benchmark: simulate the 30-qubit 5x6 grid circuit (14 cycles, patterns
ABCDCDAB, random fSim angles; the scale workload of the paper's random-circuit
benchmarks) on one GB300 per rank, and print one JSON line.

A step = initialise |0...0>, run the fused/tiled plan (every pass of the hot
path), and reduce the norm (Section 4.1's accuracy check).  The state (8 GB
complex64) is far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]

For N > 1 (torchrun) every rank simulates its own replica of the circuit
(the path has no exchange step at one state per GPU): weak scaling.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "circuit wall time & HBM GB/s at 30–32q; adjoint-gradient time vs forward"
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes (read + write) per amplitude of one launch, from the ncu
# captures summarised in profiles/ (26-qubit complex64 cases; traffic grows
# in proportion to the amplitudes, so a launch at n qubits moves
# bytes_per_amp * 2^n).  Must be cleared when the kernel changes.
NCU_TRAFFIC_PER_AMP_C64 = {
    "tensor": (536.983296e6 + 474.812160e6) / (1 << 26),   # k_gemm6, profiles/k_gemm6_grid26_3xtf32.md
    "tile": (536.981504e6 + 475.719936e6) / (1 << 26),     # k_rtile, profiles/k_rtile_grid26_k3_fp32.md
    "dense": None,
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--cycles", type=int, default=14)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64")
    ap.add_argument("--k-max", type=int, default=0, help="0 = pick by a short timing sweep")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--precision", default="auto",
                    help="fp32 | 3xtf32 | 3xfp16 | 3xbf16 | tf32 for dense k>=5 blocks; auto = fastest of the "
                         "FP32-accurate modes (fp32, 3xtf32, 3xfp16)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the adjoint, 32-qubit and batched measurements of the default line")
    ap.add_argument("--unfused", action="store_true", help="one pass per gate (no fusion, no tiles)")
    ap.add_argument("--circuit", choices=["grid", "grid_fixed", "ansatz", "paper"], default="grid",
                    help="grid: random fSim angles; grid_fixed: fSim(pi/2, pi/6) everywhere (permutation-with-"
                         "phase gates); ansatz: RY/RZ layers with CZ ladders (diagonal gates); paper: the paper's "
                         "gate set (H, CZ, T, sqrt X, sqrt Y), depth 1 + --depth + 1")
    ap.add_argument("--depth", type=int, default=26, help="cycles of the paper-gate-set circuit")
    ap.add_argument("--diag-clusters", choices=["auto", "on", "off"], default="auto",
                    help="cluster diagonal gates of any width into one pass (Sections 4.2, 4.5); auto: timed choice")
    ap.add_argument("--workload", choices=["grid", "adjoint", "batch", "batch_adjoint", "precision", "sf"],
                    default="grid",
                    help="grid: the headline circuit; adjoint: gradient vs forward on the ansatz; "
                         "batch: 512 uneven circuits in one launch; precision: tensor-core modes at 32q; "
                         "sf: Schroedinger-Feynman amplitudes of the paper's gate set across a grid cut")
    ap.add_argument("--layers", type=int, default=20)
    ap.add_argument("--count", type=int, default=None, help="circuits (batch: 512) or gradients (batch_adjoint: 256)")
    return ap.parse_args(argv)


def l2_note(n, dtype):
    """How the timed steps avoid a warm L2: the state is far larger than the
    129 MB L2 at the bench sizes; smaller states say so."""
    gb = (1 << n) * (8 if dtype == "c64" else 16) / 2**30
    if gb * 2**30 > 4 * 129e6:
        return f"inputs larger than L2 (state {gb:g} GiB)"
    return f"state {gb * 1024:g} MiB: within a few times L2, no flush between steps"


def workload_name(a):
    if a.circuit == "ansatz":
        return f"ansatz{a.n}_L{a.layers}_seed{a.seed}_{a.dtype}"
    if a.circuit == "grid_fixed":
        return f"grid{a.n}_c{a.cycles}_ABCDCDAB_fsim_pi2_pi6_seed{a.seed}_{a.dtype}"
    if a.circuit == "paper":
        return f"paper_gateset{a.n}_depth1+{a.depth}+1_seed{a.seed}_{a.dtype}"
    return f"grid{a.n}_5x6_c{a.cycles}_ABCDCDAB_fsim_random_seed{a.seed}_{a.dtype}" if a.n == 30 else \
        f"grid{a.n}_c{a.cycles}_ABCDCDAB_fsim_random_seed{a.seed}_{a.dtype}"


def max_over_ranks(values, device):
    """Element-wise maximum over ranks of per-rank values (the slowest
    rank's times); the identity without an initialised process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def replica_throughput(world, units_per_rank, seconds):
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- CPU (oracle) sample

def _circuit_spec(a):
    from workloads import circuits as C
    if a.circuit == "ansatz":
        return C.ansatz_circuit(a.n, a.layers, C.ansatz_theta(a.n, a.layers, a.seed))
    if a.circuit == "grid_fixed":
        return C.grid_circuit(a.n, a.cycles, a.seed, fixed_fsim=(math.pi / 2, math.pi / 6))
    if a.circuit == "paper":
        return C.paper_circuit(a.n, a.depth, a.seed)
    return C.scale_grid_circuit(a.n, a.cycles, a.seed)


def _host_memory_bytes():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    except (ValueError, OSError):
        return 0


def cpu_sample_cycle(n: int, cycles: int, seed: int) -> dict:
    """One whole cycle of the grid circuit (its one-qubit layer and its fSim
    layer) on the C form of the FP64 oracle, all host cores (OpenMP over set
    ids).  Returns the seconds per one-qubit and per two-qubit gate and the
    circuit's gate counts, so that circuit time = n1 t1 + n2 t2."""
    from oracle import omp
    from workloads import circuits as C
    circ = C.scale_grid_circuit(n, cycles, seed)
    gates = circ.gates
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    omp.apply_gate_inplace(psi, n, gates[0].qubits, gates[0].matrix)   # untimed: touches every page
    # the first cycle after the H layer: n one-qubit gates, then its fSim layer
    i = n
    sample = []
    while i < len(gates) and gates[i].k == 1:
        sample.append(gates[i]); i += 1
    while i < len(gates) and gates[i].k == 2:
        sample.append(gates[i]); i += 1
    t = {1: 0.0, 2: 0.0}
    cnt = {1: 0, 2: 0}
    for g in sample:
        t0 = time.perf_counter()
        omp.apply_gate_inplace(psi, n, g.qubits, g.matrix)
        t[g.k] += time.perf_counter() - t0
        cnt[g.k] += 1
    total = {1: sum(1 for g in gates if g.k == 1), 2: sum(1 for g in gates if g.k == 2)}
    return {"n": n, "threads": omp.threads(), "sec_per_1q": t[1] / max(1, cnt[1]), "sec_per_2q": t[2] / max(1, cnt[2]),
            "sample_1q": cnt[1], "sample_2q": cnt[2], "seconds": t[1] + t[2], "circuit_1q": total[1],
            "circuit_2q": total[2]}


def cpu_baseline(a) -> dict:
    """The oracle as it stands, in its C form on every host core (a fresh
    spawned process, away from the GPU process's threads): one whole cycle of
    the circuit timed per gate kind, scaled to the circuit's gate counts.
    At 30 qubits the oracle holds the state in complex128 (16 GB of host
    memory); with less memory the sample runs at 28 qubits and the time is
    scaled by the amplitude ratio."""
    need = 16 << a.n
    n_used = a.n if _host_memory_bytes() > 1.5 * need else min(a.n, 28)
    code = ("import json,bench;print(json.dumps(bench.cpu_sample_cycle(%d,%d,%d)))" % (n_used, a.cycles, a.seed))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("cpu baseline failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    scale = float(1 << (a.n - n_used))
    sec_circuit = scale * (d["sec_per_1q"] * d["circuit_1q"] + d["sec_per_2q"] * d["circuit_2q"])
    return {"value": 1.0 / sec_circuit, "unit": "circuits/s", "cores": d["threads"], "kind": "oracle",
            "sample": (f"C FP64 oracle (OpenMP over set ids, {d['threads']} threads): one whole cycle of the "
                       f"{d['n']}-qubit circuit ({d['sample_1q']} one-qubit + {d['sample_2q']} fSim gates, "
                       f"{d['seconds']:.1f} s), per-kind gate time x the circuit's {d['circuit_1q']} one-qubit "
                       f"+ {d['circuit_2q']} fSim gates"
                       + (f", x {int(scale)} (amplitude ratio {a.n} vs {n_used} qubits)" if scale > 1 else ""))}


# ----------------------------------------------------------------- own implementation

def time_passes(plan, state, steps, warmup):
    """Run |0> + every pass of the plan `steps` times after `warmup` untimed
    runs, with a CUDA event after each pass on the state's (current) stream.
    Returns (ms per step, {pass kind: (total ms, launches)}); the first pass
    of each step is left out of the per-kind sums (it includes the |0>
    initialisation)."""
    import torch
    stream = torch.cuda.current_stream()
    passes = plan.passes()
    npass = len(passes)
    for _ in range(warmup):
        state.init_basis(0)
        plan.execute(state)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(npass + 1)] for _ in range(steps)]
    for s in range(steps):
        ev[s][0].record(stream)
        state.init_basis(0)
        for i in range(npass):
            plan.execute_range(state, i, 1)
            ev[s][i + 1].record(stream)
    torch.cuda.synchronize()
    total = 0.0
    by_kind = {}
    for s in range(steps):
        total += ev[s][0].elapsed_time(ev[s][npass])
        for i in range(1, npass):
            dur = ev[s][i].elapsed_time(ev[s][i + 1])
            t, c = by_kind.get(passes[i][0], (0.0, 0))
            by_kind[passes[i][0]] = (t + dur, c + 1)
    return total / steps, by_kind


def run_own(a):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2008_00216_gb300 as pkg
    from paper_2008_00216_gb300 import binding as B

    pkg.load()
    esz = 8 if a.dtype == "c64" else 16
    state_bytes = (1 << a.n) * esz
    circ = _circuit_spec(a)
    c = B.circuit_from(circ)
    state = B.State(a.n, a.dtype)
    stream = torch.cuda.current_stream()

    def plan_for(circuit, k, prec, dc=False):
        if a.unfused:
            return B.Plan(circuit, a.dtype, k_max=1, fuse=False, use_tile=False, precision=prec)
        return B.Plan(circuit, a.dtype, k_max=k, tile_qubits=a.tile, use_tile=True, precision=prec,
                      diag_clusters=dc)

    def make_plan(k, prec, dc=False):
        return plan_for(c, k, prec, dc)

    # pick (k_max, precision) by timing one execution of each candidate
    # (excluded from the timed region); only modes at FP32-level accuracy
    cands = []
    precs = ["fp32", "3xtf32", "3xfp16"] if a.precision == "auto" else [a.precision]
    if a.dtype == "c128":
        precs = ["fp32"]
    dcs = {"auto": [False, True], "on": [True], "off": [False]}[a.diag_clusters]
    for k in ([a.k_max] if a.k_max else [1, 2, 3, 4, 6]):
        for pr in precs:
            if pr != "fp32" and k < 5:
                continue
            for dc in dcs:
                cands.append((k, pr, dc))
    if len(cands) == 1 or a.unfused:
        k_best, prec_best, dc_best = cands[0]
    else:
        best = None
        for k, pr, dc in cands:
            p = make_plan(k, pr, dc)
            p.execute(state)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p.execute(state)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if best is None or dt < best[0]:
                best = (dt, k, pr, dc)
            p.close()
        _, k_best, prec_best, dc_best = best
    plan = make_plan(k_best, prec_best, dc_best)
    passes = plan.passes()
    npass = len(passes)

    def step(events=None):
        state.init_basis(0)
        for i in range(npass):
            plan.execute_range(state, i, 1)
            if events is not None:
                events[i].record(stream)
        return state.norm()

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    pass_events = [[torch.cuda.Event(enable_timing=True) for _ in range(npass)] for _ in range(a.steps)]
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    norms = []
    for s in range(a.steps):
        starts[s].record(stream)
        norms.append(step(pass_events[s]))
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = max_over_ranks([ev0.elapsed_time(ev1)], "cuda")[0]

    # per-pass durations from the events recorded inside the timed region
    by_kind = {}
    for s in range(a.steps):
        prev = starts[s]
        for i in range(npass):
            dur = prev.elapsed_time(pass_events[s][i])
            prev = pass_events[s][i]
            if i == 0:
                continue  # includes the |0> initialisation
            kind = passes[i][0]
            tot, cnt = by_kind.get(kind, (0.0, 0))
            by_kind[kind] = (tot + dur, cnt + 1)
    state.sync()   # raises if a bounded device-side wait timed out during the run
    dom = max(by_kind, key=lambda k: by_kind[k][0])
    avg_ms = by_kind[dom][0] / by_kind[dom][1]
    peak, peak_src = measured_peaks()
    achieved = 2 * state_bytes / (avg_ms * 1e-3) / 1e9
    ms_step = elapsed_ms / a.steps
    value = replica_throughput(world, a.steps, elapsed_ms * 1e-3)
    step_bytes = (npass * 2 + 2) * state_bytes   # passes r+w, init write, norm read

    # end to end through the public API with host buffers
    e2e = None
    if rank == 0 or world > 1:
        e2e_steps = max(1, min(3, a.steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        # qs_apply_circuit when the chosen form is what it does on its own
        # (6-qubit blocks on the tensor cores: fused and run together), else a plan
        api = k_best == 6 and prec_best != "fp32" and a.dtype == "c64"
        for _ in range(e2e_steps):
            cc = B.circuit_from(circ)                    # host gate list -> library
            state.init_basis(0)
            if api:
                B.apply_circuit(state, cc, prec_best)    # fuse + upload + run
            else:
                pp = plan_for(cc, k_best, prec_best, dc_best)    # fuse + upload
                pp.execute(state)
                pp.close()
            nrm = state.norm()                           # D2H 8 bytes
            amps = state.amplitudes(0, 4096)             # D2H 4096 amplitudes
            h2d = sum(g.matrix.size * esz for g in circ.gates)
            d2h = 8 + 4096 * esz
            cc.close()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks([(time.perf_counter() - t0) / e2e_steps], "cuda")[0]
        e2e = {"value": replica_throughput(world, 1, e2e_s), "unit": "circuits/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
               "call": "qs_apply_circuit" if api else "qs_plan_create + qs_plan_execute"}

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value,
            "unit": "circuits/s",
            "n_gpus": world,
            "steps": a.steps,
            "warmup": a.warmup,
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": a.dtype,
            "data": "synthetic (seeded grid circuit generator)",
            "config": {"workload": workload_name(a), "n": a.n, "cycles": a.cycles, "gates": len(circ.gates),
                       "k_max": k_best, "precision": prec_best, "diag_clusters": dc_best,
                       "tile_qubits": a.tile or "auto", "passes": npass,
                       "pass_kinds": plan.info()["per_kind"], "l2": l2_note(a.n, a.dtype),
                       "parallelism": f"replicas{world}"},
            "circuit_wall_ms": ms_step,
            "hbm_gbs_effective": step_bytes / (ms_step * 1e-3) / 1e9,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (NCU_TRAFFIC_PER_AMP_C64[dom] * (1 << a.n)
                                     if a.dtype == "c64" and NCU_TRAFFIC_PER_AMP_C64.get(dom) else None),
                         "avg_launch_ms": avg_ms,
                         "algorithmic_bytes_per_launch": 2 * state_bytes},
            "pass_time_ms": {k: {"launches_per_step": v[1] / a.steps, "total_ms_per_step": v[0] / a.steps,
                                 "avg_launch_ms": v[0] / v[1],
                                 "hbm_frac": 2 * state_bytes / (v[0] / v[1] * 1e-3) / 1e9 / peak}
                             for k, v in by_kind.items()},
            "norm_last": norms[-1],
            "gpu_launches": a.steps * (1 + npass + 2),
            "e2e": e2e,
            "clocks": clk,
        }
        if not a.no_extras and a.workload == "grid" and a.circuit == "grid" and a.n == 30 and a.dtype == "c64":
            # the rest of the metric, measured in the same run: adjoint
            # gradient vs forward (24 qubits, both dtypes), the 32-qubit
            # circuit, and the batched form (each timed with CUDA events)
            del plan, c
            state.close()
            torch.cuda.empty_cache()
            extras = (("adjoint_c64", lambda: measure_adjoint(24, 20, 1, "c64", 5, 2)),
                      ("adjoint_c128", lambda: measure_adjoint(24, 20, 1, "c128", 3, 1)),
                      ("n32", lambda: measure_grid_tensor(32, 20, 1, 3, 1,
                                                          prec_best if prec_best != "fp32" else "3xtf32")),
                      ("batch", lambda: measure_batch(512, "c64", 5, 2)))
            for key, fn in extras:
                try:
                    out[key] = fn()
                except Exception as ex:  # reported, never silently dropped
                    out[key] = {"error": str(ex)[:300]}
            out["adjoint"] = {"n": 24, "layers": 20,
                              "c64": {k: out["adjoint_c64"].get(k) for k in ("forward_ms", "gradient_ms", "ratio")},
                              "c128": {k: out["adjoint_c128"].get(k) for k in ("forward_ms", "gradient_ms", "ratio")}}
        if not a.no_cpu_baseline:
            try:
                out["cpu_baseline"] = cpu_baseline(a)
            except Exception as ex:  # reported, never silently dropped
                out["cpu_baseline"] = {"error": str(ex)[:300]}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------- reference arm (the oracle)

def run_reference(a, step_target_s: float = 6.0):
    """The oracle (the C form, every host core) on the same circuit.  Each
    step runs the next chunk of the circuit's gates in order (wrapping
    around), sized from one untimed gate to take about `step_target_s`; the
    value is the circuits' worth of gates the timed steps ran over their
    time.  Rank 0 only; other ranks return without work."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import omp
    need = 16 << a.n
    n = a.n if _host_memory_bytes() > 1.5 * need else min(a.n, 28)
    circ = _circuit_spec(argparse.Namespace(**{**vars(a), "n": n}))
    gates = circ.gates
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    omp.apply_gate_inplace(psi, n, gates[0].qubits, gates[0].matrix)   # untimed: touches every page
    t0 = time.perf_counter()
    omp.apply_gate_inplace(psi, n, gates[1].qubits, gates[1].matrix)   # untimed: calibration
    per_gate = time.perf_counter() - t0
    chunk = max(1, min(len(gates), int(round(step_target_s / per_gate))))
    pos = 2
    times, done, kinds = [], 0, {1: 0, 2: 0}
    for i in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        ran = []
        for _ in range(chunk):
            g = gates[pos % len(gates)]
            omp.apply_gate_inplace(psi, n, g.qubits, g.matrix)
            ran.append(g.k)
            pos += 1
        dt = time.perf_counter() - t0
        if i >= a.warmup:
            times.append(dt)
            done += len(ran)
            for k in ran:
                kinds[k] = kinds.get(k, 0) + 1
    scale = float(1 << (a.n - n))
    sec = sum(times) * scale
    value = (done / len(gates)) / sec
    sample = (f"C FP64 oracle (OpenMP over set ids, {omp.threads()} threads) on the {n}-qubit circuit: "
              f"{a.steps} timed steps of {chunk} consecutive gates each ({kinds.get(1, 0)} one-qubit + "
              f"{kinds.get(2, 0)} two-qubit gates in all, {sum(times):.1f} s) = {done / len(gates):.3f} circuits"
              + (f", x {int(scale)} (amplitude ratio {a.n} vs {n} qubits)" if scale > 1 else ""))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "circuits/s", "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic (seeded grid circuit generator)",
           "config": {"workload": workload_name(a), "n": a.n, "cycles": a.cycles},
           "cpu_baseline": {"value": value, "unit": "circuits/s", "kind": "oracle", "cores": omp.threads(),
                            "sample": sample},
           "e2e": {"value": value, "unit": "circuits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- secondary workloads

def _events_ms(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def measure_adjoint(n, layers, seed, dtype, steps, warmup) -> dict:
    """Hardware-efficient ansatz (RY, RZ per qubit per layer + CZ ladder),
    transverse-field Ising H: adjoint gradient time against one forward
    evaluation of E(theta) (circuit + expectation), both with CUDA events."""
    import paper_2008_00216_gb300 as pkg
    from paper_2008_00216_gb300 import binding as B
    from workloads import circuits as C
    pkg.load()
    theta = C.ansatz_theta(n, layers, seed=seed)
    spec = C.ansatz_circuit(n, layers, theta)
    c = B.circuit_from(spec)
    h = B.PauliSum(n, C.ising_hamiltonian(n))
    psi, lam = B.State(n, dtype), B.State(n, dtype, init=None)
    best = None
    # the fastest forward evaluation the library offers (tensor-core
    # 6-qubit blocks included for complex64)
    cands = [(k, "fp32") for k in (1, 2, 3, 4)] + ([(6, "3xtf32"), (6, "3xfp16")] if dtype == "c64" else [])
    for k, prec in cands:
        p = B.Plan(c, dtype, k_max=k, precision=prec)
        ms = _events_ms(lambda: (psi.init_basis(0), p.execute(psi), B.expectation(psi, h)), 2, 1)
        if best is None or ms < best[0]:
            best = (ms, k, prec)
        p.close()
    plan = B.Plan(c, dtype, k_max=best[1], precision=best[2])
    fwd_ms = _events_ms(lambda: (psi.init_basis(0), plan.execute(psi), B.expectation(psi, h)), steps, warmup)
    adj_ms = _events_ms(lambda: B.adjoint_gradient(c, theta, h, psi, lam), steps, warmup)
    psi.sync()
    for o in (plan, c, h, psi, lam):
        o.close()
    return {"n": n, "layers": layers, "params": int(theta.size), "dtype": dtype, "forward_ms": fwd_ms,
            "forward_k_max": best[1], "forward_precision": best[2], "gradient_ms": adj_ms, "ratio": adj_ms / fwd_ms,
            "gradients_per_s": 1e3 / adj_ms, "steps": steps, "warmup": warmup}


def run_adjoint(a):
    d = measure_adjoint(a.n, a.layers, a.seed, a.dtype, a.steps, a.warmup)
    out = {"metric": "adjoint-gradient time vs forward", "workload": "adjoint", "value": d["ratio"],
           "unit": "adjoint/forward time ratio", "higher_is_better": False, **d, "adjoint_ms": d["gradient_ms"]}
    print(json.dumps(out), flush=True)


def run_batch_adjoint(a):
    """256 adjoint gradients of 20-layer ansatz circuits, n ~ U{12..20}
    (seeded), Ising H, complex64: one qs_adjoint_gradient_batch call (host
    threads plan concurrently, each gradient on one of 16 streams) against a
    loop of single qs_adjoint_gradient calls.  Wall-clock time of the calls,
    which include all host planning and synchronise."""
    import torch
    import paper_2008_00216_gb300 as pkg
    from paper_2008_00216_gb300 import binding as B
    from workloads import circuits as C
    from workloads.rng import Xoshiro256ss
    pkg.load()
    count = a.count or 256
    rng = Xoshiro256ss(a.seed)
    ns = [12 + rng.randint(9) for _ in range(count)]
    streams = [torch.cuda.Stream() for _ in range(16)]
    circs, thetas, hams, psis, lams = [], [], [], [], []
    for i, n in enumerate(ns):
        theta = C.ansatz_theta(n, 20, seed=a.seed + i)
        circs.append(B.circuit_from(C.ansatz_circuit(n, 20, theta)))
        thetas.append(theta)
        hams.append(B.PauliSum(n, C.ising_hamiltonian(n)))
        st = streams[i % len(streams)]
        psis.append(B.State(n, a.dtype, stream=st))
        lams.append(B.State(n, a.dtype, stream=st, init=None))
    torch.cuda.synchronize()
    for _ in range(max(1, a.warmup)):
        B.adjoint_gradient_batch(circs, thetas, hams, psis, lams)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        B.adjoint_gradient_batch(circs, thetas, hams, psis, lams)
        times.append(time.perf_counter() - t0)
    batch_s = sorted(times)[len(times) // 2]
    t0 = time.perf_counter()
    for i in range(count):
        B.adjoint_gradient(circs[i], thetas[i], hams[i], psis[i], lams[i])
    loop_s = time.perf_counter() - t0
    params = sum(t.size for t in thetas)
    out = {"metric": "batched adjoint gradients/s vs looped single gradients", "workload": "batch_adjoint",
           "value": count / batch_s, "unit": "gradients/s", "higher_is_better": True, "dtype": a.dtype,
           "gradients": count, "params_total": int(params), "n_range": [min(ns), max(ns)], "layers": 20,
           "batch_s": batch_s, "loop_s": loop_s, "loop_gradients_per_s": count / loop_s,
           "speedup_vs_loop": loop_s / batch_s, "streams": len(streams), "steps": a.steps, "warmup": a.warmup,
           "timing": "wall clock of the synchronous calls (host planning included)"}
    print(json.dumps(out), flush=True)


def measure_batch(count, dtype, steps, warmup) -> dict:
    """Seeded grid circuits, n ~ U{10..22}, depth ~ U{8..24}: one batched
    graph launch (autotuned) against looping the single-circuit plans."""
    import paper_2008_00216_gb300 as pkg
    from paper_2008_00216_gb300 import binding as B
    from workloads import circuits as C
    pkg.load()
    specs = C.batched_workload(count, seed0=0)
    circs = [B.circuit_from(s) for s in specs]
    t0 = time.perf_counter()
    best = B.batch_autotune(circs, dtype)
    tune_s = time.perf_counter() - t0
    bt = B.Batch(circs, dtype, opts=best)
    ms = _events_ms(lambda: bt.run(), steps, warmup)
    bt.sync()
    # loop of the single-circuit path: one plan and state per circuit, built beforehand
    plans = [B.Plan(c, dtype, k_max=best.k_max) for c in circs]
    states = [B.State(s.n, dtype) for s in specs]

    def loop():
        for p, st in zip(plans, states):
            st.init_basis(0)
            p.execute(st)
    loop_ms = _events_ms(loop, max(1, steps // 2), 1)
    amps_gates = sum((1 << s.n) * len(s.gates) for s in specs)
    info = bt.info()
    for o in plans + states + circs + [bt]:
        o.close()
    return {"circuits": count, "dtype": dtype, "circuits_per_s": count / (ms * 1e-3), "batch_ms": ms,
            "loop_ms": loop_ms, "loop_circuits_per_s": count / (loop_ms * 1e-3), "speedup_vs_loop": loop_ms / ms,
            "autotune": {"k_max": best.k_max, "tile_qubits": best.tile_qubits, "seconds": tune_s},
            "batch_info": info, "amplitude_gate_updates_per_s": amps_gates / (ms * 1e-3), "steps": steps,
            "warmup": warmup}


def run_batch(a):
    d = measure_batch(a.count or 512, a.dtype, a.steps, a.warmup)
    out = {"metric": "batched circuits/s vs looped single-circuit path", "workload": "batch",
           "value": d["circuits_per_s"], "unit": "circuits/s", "higher_is_better": True, **d}
    print(json.dumps(out), flush=True)


def measure_grid_tensor(n, cycles, seed, steps, warmup, precision="3xtf32") -> dict:
    """The grid circuit at n qubits (complex64, 6-qubit tensor-core blocks in
    a split precision): time per circuit with CUDA events around every pass,
    passes, and the tensor pass's fraction of the HBM roofline."""
    import torch
    import paper_2008_00216_gb300 as pkg
    from paper_2008_00216_gb300 import binding as B
    from workloads import circuits as C
    pkg.load()
    spec = C.scale_grid_circuit(n, cycles, seed)
    c = B.circuit_from(spec)
    plan = B.Plan(c, "c64", k_max=6, precision=precision)
    state = B.State(n, "c64")
    ms, by_kind = time_passes(plan, state, steps, warmup)
    state.sync()
    peak, src = measured_peaks()
    nbytes = 2 * (1 << n) * 8
    kinds = {k: {"launches_per_circuit": v[1] / steps, "avg_launch_ms": v[0] / v[1],
                 "hbm_frac": nbytes / (v[0] / v[1] * 1e-3) / 1e9 / peak} for k, v in by_kind.items()}
    out = {"n": n, "cycles": cycles, "gates": len(spec.gates), "precision": precision, "ms_per_circuit": ms,
           "passes": plan.info()["passes"],
           "pass_kinds": plan.info()["per_kind"], "per_kind": kinds,
           "hbm_frac": kinds.get("tensor", {}).get("hbm_frac"), "peak_gbs": peak, "peak_source": src,
           "steps": steps, "warmup": warmup}
    for o in (plan, c, state):
        o.close()
    torch.cuda.empty_cache()
    return out


def run_precision(a):
    """32-qubit 4x8 grid, 20 cycles, fused k_max 5 and 6 on a complex64
    state: time and error of the tensor-core modes and the FP32 CUDA-core
    path against the complex128 GPU path of the same circuit."""
    import torch
    import paper_2008_00216_gb300 as pkg
    from paper_2008_00216_gb300 import binding as B
    from workloads import circuits as C
    pkg.load()
    n = a.n
    spec = C.scale_grid_circuit(n, a.cycles, seed=a.seed)
    c = B.circuit_from(spec)
    ref = B.State(n, "c128")
    pref = B.Plan(c, "c128", k_max=2)
    pref.execute(ref)
    ref.sync()
    ref_ms = _events_ms(lambda: (ref.init_basis(0), pref.execute(ref)), 1, 0)
    rt = ref.tensor

    def errors(xt):
        """relative L2, max |dp| and TV distance against the complex128 state,
        in chunks of 2^26 amplitudes (bounded temporaries)"""
        d2 = r2 = mx = tv = 0.0
        step = 1 << 26
        for i in range(0, rt.numel(), step):
            r = rt[i:i + step]
            x = xt[i:i + step].to(torch.complex128)
            d2 += (torch.linalg.vector_norm(x - r) ** 2).item()
            r2 += (torch.linalg.vector_norm(r) ** 2).item()
            dp = (x.abs() ** 2 - r.abs() ** 2).abs()
            mx = max(mx, dp.max().item())
            tv += 0.5 * dp.sum().item()
        return math.sqrt(d2 / r2), mx, tv

    rows = []
    st = B.State(n, "c64")
    for k in (5, 6):
        for prec in ("fp32", "tf32", "3xtf32", "3xfp16", "3xbf16"):
            p = B.Plan(c, "c64", k_max=k, precision=prec)
            ms = _events_ms(lambda: (st.init_basis(0), p.execute(st)), a.steps, 1)
            st.sync()
            err, mx, tv = errors(st.tensor)
            rows.append({"k_max": k, "precision": prec, "ms": ms, "rel_l2_vs_c128": err,
                         "max_prob_err": mx, "tv": tv, "passes": p.info()["passes"]})
            p.close()
    out = {"metric": "split-precision tensor-core form vs FP32 (time and error vs complex128)", "workload": "precision",
           "n": n, "cycles": a.cycles, "c128_ms": ref_ms, "rows": rows}
    print(json.dumps(out), flush=True)


def run_sf(a):
    """Schroedinger-Feynman amplitudes (the paper's hybrid mode): the paper's
    gate-set circuit on the near-square grid, cut between the middle grid
    columns; `--count` amplitudes (default 4096: the first ones) from all
    paths.  Wall-clock time of the call (host path set-up included)."""
    import torch
    import paper_2008_00216_gb300 as pkg
    from paper_2008_00216_gb300 import binding as B
    from workloads import circuits as C
    pkg.load()
    n = a.n
    circ = C.paper_circuit(n, a.depth, a.seed)
    rows, cols = C.grid_shape(n)
    part_a = [r * cols + cc for r in range(rows) for cc in range(cols // 2) if r * cols + cc < n]
    c = B.circuit_from(circ)
    count = a.count or 4096
    idx = np.arange(count, dtype=np.uint64)
    _, paths = B.sf_amplitudes(c, part_a, [], a.dtype)
    for _ in range(max(1, a.warmup)):
        B.sf_amplitudes(c, part_a, idx, a.dtype)
    times = []
    for _ in range(a.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.sf_amplitudes(c, part_a, idx, a.dtype)
        times.append(time.perf_counter() - t0)
    sec = sorted(times)[len(times) // 2]
    out = {"metric": "Schroedinger-Feynman amplitudes", "workload": "sf", "value": sec, "unit": "s per call",
           "higher_is_better": False, "n": n, "depth": f"1+{a.depth}+1", "dtype": a.dtype, "paths": paths,
           "half_qubits": [len(part_a), n - len(part_a)], "amplitudes": count, "steps": a.steps,
           "timing": "wall clock of the synchronous call (path circuits built on the host included)"}
    print(json.dumps(out), flush=True)


def main():
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "adjoint":
        run_adjoint(a)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "precision":
        run_precision(a)
    elif a.workload == "batch_adjoint":
        run_batch_adjoint(a)
    elif a.workload == "sf":
        run_sf(a)
    else:
        run_own(a)


if __name__ == "__main__":
    main()
