"""Measurement sampling (the backend's "sample" operation, Section 4.1) -- oracle side.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper names sampling as the third backend operation next to initialisation and gate
application but prints no procedure; this is the reading both sides implement, every
floating-point step in a fixed order so that the sampled indices are reproducible bit
for bit:

1. p_k = |alpha_k|^2 in the state's precision (complex64: float32 products and sum),
   widened to FP64.
2. Blocks of B = min(64, 2^n) outcomes: S_b = p_{Bb} + p_{Bb+1} + ... summed in index
   order in FP64, starting from 0.
3. Chunks of C = min(4096, #blocks) blocks: within a chunk the exclusive prefix L_b of
   the S_b in index order; the chunk totals (the inclusive prefix at its last block); the
   exclusive prefix O_c of the totals in index order and their sum T (the total mass).
   The block prefix is P_b = O_{chunk(b)} + L_b.
4. Shot i: z = SplitMix64 output for the counter x_i = seed + (i + 1) * 0x9E3779B97F4A7C15
   (mod 2^64) -- Steele, Lea and Flood's generator: z = x_i; z = (z ^ (z >> 30)) *
   0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB; z ^= z >> 31 (mod 2^64);
   u = (z >> 11) * 2^-53 in [0, 1); target = u * T (FP64).
5. b = the largest block with P_b <= target and S_b > 0 (the largest with P_b <= target,
   moved down past blocks with S_b = 0; the first block with S_b > 0 has P_b = 0, so one
   exists when T > 0); r = target - P_b; the outcome is the first k of the block whose
   running sum (index order, from 0) exceeds r, else the block's last outcome with p_k > 0.
   A state with T = 0 has no distribution to sample (an error).

Outcomes with p_k = 0 are never drawn; for a normalised state the frequencies converge
to p_k (pinned by chi-square tests in tests/test_oracle_sampling.py).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1
BLOCK = 64
CHUNK = 4096


def splitmix64(x: int) -> int:
    """The SplitMix64 output function applied to the 64-bit counter value x."""
    z = x & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def uniforms(seed: int, nshots: int) -> np.ndarray:
    """u_i = (SplitMix64(seed + (i + 1) gamma) >> 11) 2^-53, i = 0..nshots-1 (exact)."""
    out = np.empty(nshots, dtype=np.float64)
    for i in range(nshots):
        z = splitmix64((seed + (i + 1) * GAMMA) & M64)
        out[i] = float(z >> 11) * 2.0 ** -53
    return out


def block_prefix(p: np.ndarray):
    """Steps 2-3: block sums S, block prefixes P and the total T (all FP64, index order)."""
    n_out = p.size
    B = min(BLOCK, n_out)
    nb = n_out // B
    S = np.cumsum(p.reshape(nb, B), axis=1)[:, -1]          # sequential within a block
    C = min(CHUNK, nb)
    nc = nb // C
    inc = np.cumsum(S.reshape(nc, C), axis=1)               # sequential within a chunk
    L = np.zeros_like(inc)
    L[:, 1:] = inc[:, :-1]                                   # exclusive prefix
    tot = inc[:, -1]
    Oinc = np.cumsum(tot)
    O = np.zeros_like(Oinc)
    O[1:] = Oinc[:-1]
    T = float(Oinc[-1])
    P = (O[:, None] + L).reshape(nb)
    return B, S, P, T


def sample(p_state: np.ndarray, seed: int, nshots: int) -> np.ndarray:
    """nshots outcome indices by steps 1-5; p_state: |alpha_k|^2 in the state's precision."""
    p = np.asarray(p_state, dtype=np.float64)
    B, S, P, T = block_prefix(p)
    if not T > 0.0:
        raise ValueError("sampling needs a state with nonzero norm")
    u = uniforms(seed, nshots)
    out = np.empty(nshots, dtype=np.uint64)
    for i in range(nshots):
        target = np.float64(u[i]) * np.float64(T)
        b = int(np.searchsorted(P, target, side="right")) - 1
        b = max(b, 0)
        while S[b] == 0.0:
            b -= 1
        r = np.float64(target) - np.float64(P[b])
        blk = p[b * B:(b + 1) * B]
        c = np.float64(0.0)
        k = -1
        for j in range(B):
            c = c + np.float64(blk[j])
            if c > r:
                k = j
                break
        if k < 0:
            nz = np.flatnonzero(blk > 0)
            k = int(nz[-1]) if nz.size else B - 1
        out[i] = b * B + k
    return out
