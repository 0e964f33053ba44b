"""Pins of the oracle's measurement sampling (oracle/sampling.py): the generator's published
outputs, the counter structure, uniformity, chi-square agreement with the probabilities,
a direct sequential definition on single-block states, and the block/chunk prefix against
a flat prefix on a multi-chunk state."""
import numpy as np
import pytest

from oracle import sampling as S

scipy_stats = pytest.importorskip("scipy.stats")


def test_splitmix64_reference_outputs():
    # SplitMix64 seeded with 0: the first three outputs of the published generator
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [S.splitmix64((k * S.GAMMA) & S.M64) for k in (1, 2, 3)]
    assert got == want


def test_uniforms_counter_structure_and_range():
    u = S.uniforms(12345, 2000)
    assert np.all(u >= 0.0) and np.all(u < 1.0)
    # shot i of seed s is shot i - 1 of seed s + gamma
    assert np.array_equal(S.uniforms((12345 + S.GAMMA) & S.M64, 1999), u[1:])
    # 53-bit grid
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))


def test_uniforms_are_uniform():
    u = S.uniforms(2026, 100000)
    assert abs(u.mean() - 0.5) < 0.004
    assert scipy_stats.kstest(u, "uniform").pvalue > 1e-3


def _direct(p, u):
    """Sequential definition for a single block: first k with running sum > u T."""
    T = np.float64(0.0)
    for v in p:
        T = T + np.float64(v)
    out = []
    for ui in u:
        target = np.float64(ui) * T
        c = np.float64(0.0)
        k = -1
        for j, v in enumerate(p):
            c = c + np.float64(v)
            if c > target:
                k = j
                break
        if k < 0:
            k = int(np.flatnonzero(p > 0)[-1])
        out.append(k)
    return np.array(out, dtype=np.uint64)


def test_single_block_matches_sequential_definition():
    rng = np.random.default_rng(3)
    for n in (1, 3, 6):
        p = rng.random(1 << n)
        p[rng.integers(0, 1 << n, 1 + (1 << n) // 4)] = 0.0
        if not p.any():
            p[0] = 1.0
        p /= p.sum()
        got = S.sample(p, 99 + n, 500)
        assert np.array_equal(got, _direct(p, S.uniforms(99 + n, 500)))


def test_chi_square_against_probabilities():
    rng = np.random.default_rng(4)
    p = rng.random(16) ** 3
    p[[2, 9]] = 0.0
    p /= p.sum()
    shots = S.sample(p, 7, 60000)
    counts = np.bincount(shots.astype(np.int64), minlength=16)
    assert counts[2] == 0 and counts[9] == 0
    nz = p > 0
    chi2, pval = scipy_stats.chisquare(counts[nz], 60000 * p[nz])
    assert pval > 1e-4


def test_multi_chunk_prefix_agrees_with_a_flat_prefix():
    """2^20 outcomes = 4 chunks of 4096 blocks: the chunked prefix differs from a flat
    sequential prefix only by rounding; every sample lies in its outcome's interval of
    the exact (flat) cumulative distribution up to that rounding."""
    rng = np.random.default_rng(5)
    n = 20
    p = rng.exponential(size=1 << n)
    p[rng.integers(0, 1 << n, 1 << 16)] = 0.0
    p /= p.sum()
    B, Sb, P, T = S.block_prefix(p)
    assert B == 64 and P.size == (1 << n) // 64
    flat = np.concatenate([[0.0], np.cumsum(Sb)[:-1]])
    assert np.max(np.abs(P - flat)) < 1e-12
    shots = S.sample(p, 31, 3000)
    assert np.all(p[shots.astype(np.int64)] > 0)
    cdf = np.concatenate([[0.0], np.cumsum(p)])
    u = S.uniforms(31, 3000)
    k = shots.astype(np.int64)
    assert np.all(cdf[k] - 1e-11 <= u * T) and np.all(u * T <= cdf[k + 1] + 1e-11)


def test_deterministic_and_seed_dependent():
    p = np.full(256, 1.0 / 256)
    a = S.sample(p, 1, 300)
    assert np.array_equal(a, S.sample(p, 1, 300))
    assert not np.array_equal(a, S.sample(p, 2, 300))
    with pytest.raises(ValueError):
        S.sample(np.zeros(8), 1, 3)
