"""Measurement sampling (the backend's "sample" operation, Section 4.1) -- oracle side.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper names sampling as the third backend operation next to initialisation and gate
application but prints no procedure.  The reading both sides implement draws from an
exact integer cumulative distribution, so that the sampled indices are reproducible bit
for bit and the prefix sums may be formed in any order:

1. p_k = |alpha_k|^2 in the state's precision (complex64: float32 products and sum).
2. P_k = floor(p_k 2^58), an integer: p_k 2^58 is exact in FP64 (a power-of-two scale),
   so the floor is exact too.  States of norm below 64 keep every sum below 2^64.
3. C_k = P_0 + ... + P_k (exact integers), T = C_{N-1}; T = 0 (a zero state, or one
   whose probabilities are all below 2^-58) has no distribution to sample: an error.
4. Shot i: z = SplitMix64 output for the counter x_i = seed + (i + 1) * 0x9E3779B97F4A7C15
   (mod 2^64) -- Steele, Lea and Flood's generator: z = x_i; z = (z ^ (z >> 30)) *
   0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB; z ^= z >> 31 (mod 2^64);
   u = z >> 11 (53 bits); target = floor(u T / 2^53), an integer in [0, T).
5. The outcome is the k with C_{k-1} <= target < C_k (C_{-1} = 0).

Outcome k is drawn with probability P_k / T (up to the 2^-53 grid of u): outcomes with
P_k = 0 are never drawn, and for a normalised state the frequencies converge to p_k
(pinned by chi-square tests in tests/test_oracle_sampling.py).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1
SCALE_BITS = 58


def splitmix64(x: int) -> int:
    """The SplitMix64 output function applied to the 64-bit counter value x."""
    z = x & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def u53(seed: int, nshots: int) -> list:
    """The 53-bit integers z_i >> 11 of shots i = 0..nshots-1."""
    return [splitmix64((seed + (i + 1) * GAMMA) & M64) >> 11 for i in range(nshots)]


def uniforms(seed: int, nshots: int) -> np.ndarray:
    """u_i 2^-53 in [0, 1) (exact in FP64)."""
    return np.array([float(v) * 2.0 ** -53 for v in u53(seed, nshots)], dtype=np.float64)


def fixed(p_state: np.ndarray) -> np.ndarray:
    """Step 2: P_k = floor(p_k 2^58) as uint64."""
    p = np.asarray(p_state)
    return np.floor(p.astype(np.float64) * 2.0 ** SCALE_BITS).astype(np.uint64)


def sample(p_state: np.ndarray, seed: int, nshots: int) -> np.ndarray:
    """nshots outcome indices by steps 1-5; p_state: |alpha_k|^2 in the state's precision."""
    P = fixed(p_state)
    C = np.cumsum(P, dtype=np.uint64)
    T = int(C[-1]) if C.size else 0
    if T == 0:
        raise ValueError("sampling needs a state with nonzero probabilities")
    targets = np.array([(u * T) >> 53 for u in u53(seed, nshots)], dtype=np.uint64)
    return np.searchsorted(C, targets, side="right").astype(np.uint64)
