"""Seeded pseudo-random numbers for the synthetic workloads.

Every circuit, angle and test state in this repository is drawn from this
generator so that the same seed yields the same input on any machine and any
numpy version.  Two published generators are restated here:

* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014) expands a 64-bit seed into the 256-bit state.
* xoshiro256** (Blackman and Vigna, "Scrambled linear pseudorandom number
  generators", ACM TOMS 2021) produces the stream.

Nothing here touches a quantum state; this module holds no simulation
arithmetic.
"""

from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & _M64


class SplitMix64:
    """SplitMix64: a Weyl sequence with golden-ratio increment, then a
    two-round xor-shift-multiply finaliser."""

    def __init__(self, seed: int):
        self.x = seed & _M64

    def next(self) -> int:
        self.x = (self.x + 0x9E3779B97F4A7C15) & _M64
        z = self.x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)


class Xoshiro256ss:
    """xoshiro256**: 256-bit linear engine with the '**' scrambler
    (rotate-left of s1*5 by 7, times 9)."""

    def __init__(self, seed: int):
        sm = SplitMix64(seed)
        self.s = [sm.next() for _ in range(4)]

    def next_u64(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & _M64, 7) * 9) & _M64
        t = (s[1] << 17) & _M64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def randint(self, m: int) -> int:
        """Uniform integer in [0, m) by rejection (no modulo bias)."""
        if m <= 0:
            raise ValueError("randint needs m > 0")
        limit = ((1 << 64) // m) * m
        while True:
            x = self.next_u64()
            if x < limit:
                return x % m

    def normal(self) -> float:
        """Standard normal by the Box-Muller transform."""
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        return float(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2))


def random_unitary(k: int, rng: Xoshiro256ss) -> np.ndarray:
    """Haar-like random 2^k x 2^k unitary: QR of a complex Gaussian matrix
    with the phases of R's diagonal divided out (Mezzadri 2007)."""
    d = 1 << k
    z = np.array([[complex(rng.normal(), rng.normal()) for _ in range(d)]
                  for _ in range(d)]) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diagonal(r) / np.abs(np.diagonal(r))
    return q * ph[None, :]


def random_state(n: int, seed: int) -> np.ndarray:
    """Normalised complex Gaussian state of 2^n amplitudes (complex128).

    Uses numpy's PCG64 seeded from SplitMix64 for speed at large n; PCG64's
    raw stream is stable across numpy releases and standard_normal of a
    fixed BitGenerator has been stable since numpy 1.17."""
    sm = SplitMix64(seed)
    g = np.random.Generator(np.random.PCG64(sm.next()))
    psi = g.standard_normal(1 << n) + 1j * g.standard_normal(1 << n)
    psi /= np.sqrt(np.vdot(psi, psi).real)
    return psi
