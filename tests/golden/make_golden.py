"""Write sampled-amplitude fixtures of the scale grid circuits with the FP64
oracle only (no CUDA code is imported).

Circuit: the seeded grid generator with patterns ABCDCDAB and random fSim
angles (theta ~ U(0, pi/2), phi ~ U(0, pi)), 14 (or the given number of)
cycles, seed 1, at n qubits on the near-square grid.  Stored per file: n, seed, cycles, the number of
gates, 512 seeded sample indices with their amplitudes, the first 64
amplitudes, and two whole-state sums (sum |a|^2 and sum |a|^4) that depend
on every amplitude.

Usage:  python tests/golden/make_golden.py 26 [28 28:20 ...]   (n[:cycles], default 14 cycles)
"""

import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from workloads import circuits as C  # noqa: E402
from workloads.rng import Xoshiro256ss  # noqa: E402


def sample_indices(n, count=512, seed=7):
    rng = Xoshiro256ss(seed)
    return sorted({rng.next_u64() % (1 << n) for _ in range(count)})


def main(specs):
    for spec in specs:
        n, cycles = (int(x) for x in (spec.split(":") + ["14"])[:2])
        t0 = time.time()
        circ = C.scale_grid_circuit(n, cycles, seed=1)
        psi = oracle.simulate(n, circ.gates)
        idx = sample_indices(n)
        p = np.abs(psi) ** 2
        out = {
            "what": "FP64 oracle amplitudes of the scale grid circuit (ABCDCDAB, random fSim)",
            "n": n, "cycles": cycles, "seed": 1, "num_gates": len(circ.gates),
            "indices": idx,
            "amplitudes": [[float(psi[i].real), float(psi[i].imag)] for i in idx],
            "first64": [[float(a.real), float(a.imag)] for a in psi[:64]],
            "sum_p": math.fsum(p.tolist()),
            "sum_p2": math.fsum((p * p).tolist()),
            "oracle_seconds": time.time() - t0,
        }
        path = os.path.join(HERE, f"grid{n}_c{cycles}_seed1.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=0)
        print(path, f"{time.time() - t0:.0f}s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["26"])
