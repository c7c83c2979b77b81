"""Error measures between a computed state and the oracle's (test
infrastructure only, like the rest of this package).

* relative L2 error ||psi - psi_ref|| / ||psi_ref|| (no global-phase
  alignment: a unitary circuit fixes the phase);
* output-probability errors max_j |p_j - p_ref_j| and the total-variation
  distance (1/2) sum_j |p_j - p_ref_j| (Section 2: outcome probabilities
  are |alpha_j|^2).
"""

from __future__ import annotations

import numpy as np


def rel_l2(psi: np.ndarray, ref: np.ndarray) -> float:
    ref = np.asarray(ref, dtype=np.complex128)
    d = np.asarray(psi, dtype=np.complex128) - ref
    return float(np.sqrt(np.vdot(d, d).real) / np.sqrt(np.vdot(ref, ref).real))


def max_prob_error(psi: np.ndarray, ref: np.ndarray) -> float:
    return float(np.max(np.abs(np.abs(psi) ** 2 - np.abs(ref) ** 2)))


def tv_distance(psi: np.ndarray, ref: np.ndarray) -> float:
    return float(0.5 * np.sum(np.abs(np.abs(psi) ** 2 - np.abs(ref) ** 2)))


def rel_l2_vec(g: np.ndarray, ref: np.ndarray) -> float:
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(g, dtype=np.float64) - ref) / np.linalg.norm(ref))
