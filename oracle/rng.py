"""Oracle: the SplitMix64 counter-based generator used for Hutchinson probes.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; reference C by S. Vigna): the k-th output (k = 0, 1,
...) of a generator started from state ``seed`` is

    z = seed + (k + 1) * 0x9E3779B97F4A7C15            (mod 2^64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)

so any output is a pure function of (seed, k): a counter-based generator.

Probe convention of this engine (the paper only says "Hutchinson-style",
Sec. 5): for point p of a call, probe s of q, the ambient Rademacher vector
w in {+1, -1}^n has coordinate i equal to +1 if bit (i mod 64) of output
k = (p*q + s) * ceil(n/64) + i // 64 is 0, and -1 otherwise.
"""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, k: int) -> int:
    z = (seed + (k + 1) * GAMMA) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def rademacher(seed: int, p: int, s: int, q: int, n: int) -> np.ndarray:
    words = (n + 63) // 64
    base = (p * q + s) * words
    w = np.empty(n)
    for i in range(n):
        bit = (splitmix64(seed, base + i // 64) >> (i % 64)) & 1
        w[i] = -1.0 if bit else 1.0
    return w
