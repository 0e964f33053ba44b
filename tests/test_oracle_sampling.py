"""Pins of the oracle's measurement sampling (oracle/sampling.py): the generator's
published outputs and counter structure, uniformity, the fixed-point step against exact
rationals, a brute-force definition of the drawn outcome (the interval of the exact integer
cumulative distribution that holds the target), chi-square agreement with the
probabilities, zero-probability outcomes never drawn, and a planted off-by-one."""
from fractions import Fraction

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


def test_fixed_point_is_exact_floor():
    rng = np.random.default_rng(8)
    for dt in (np.float32, np.float64):
        p = (rng.random(500) * np.exp2(rng.integers(-70, 1, 500))).astype(dt)
        P = S.fixed(p)
        for pk, Pk in zip(p, P):
            q = Fraction(float(pk)) * 2 ** S.SCALE_BITS
            assert int(Pk) == q.numerator // q.denominator


def _brute(p, seed, nshots):
    """Outcome i = the k with C_{k-1} <= floor(u T / 2^53) < C_k, by a linear scan with
    Python integers."""
    P = [int(v) for v in S.fixed(p)]
    T = sum(P)
    out = []
    for u in S.u53(seed, nshots):
        target = (u * T) >> 53
        c = 0
        for k, v in enumerate(P):
            if c <= target < c + v:
                out.append(k)
                break
            c += v
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_matches_brute_force_definition(dt):
    rng = np.random.default_rng(3)
    for n in (0, 1, 3, 6, 9):
        p = rng.random(1 << n)
        p[rng.integers(0, 1 << n, 1 + (1 << n) // 4)] = 0.0
        if not p.any():
            p[0] = 1.0
        p = (p / p.sum()).astype(dt)
        assert np.array_equal(S.sample(p, 99 + n, 400), _brute(p, 99 + n, 400))


def test_target_interval_at_a_million_outcomes():
    """2^20 outcomes: every drawn k satisfies C_{k-1} <= target < C_k with the exact
    integer prefix (Python integers, independent of numpy's cumsum), and p_k > 0."""
    rng = np.random.default_rng(5)
    n = 20
    p = rng.exponential(size=1 << n)
    p[rng.integers(0, 1 << n, 1 << 16)] = 0.0
    p = (p / p.sum()).astype(np.float32)
    shots = S.sample(p, 31, 2000).astype(np.int64)
    assert np.all(p[shots] > 0)
    P = [int(v) for v in S.fixed(p)]
    pre = [0] * (len(P) + 1)
    for k, v in enumerate(P):
        pre[k + 1] = pre[k] + v
    T = pre[-1]
    for k, u in zip(shots, S.u53(31, 2000)):
        target = (u * T) >> 53
        assert pre[k] <= target < pre[k + 1]


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


def test_deterministic_and_seed_dependent():
    p = np.full(256, 1.0 / 256)
    a = S.sample(p, 1, 300)
    assert np.array_equal(a, S.sample(p, 1, 300))
    assert not np.array_equal(a, S.sample(p, 2, 300))
    with pytest.raises(ValueError):
        S.sample(np.zeros(8), 1, 3)


def test_an_off_by_one_search_is_caught(monkeypatch):
    # Planted mistake in the oracle: side="left" picks k with C_{k-1} < target <= C_k,
    # a neighbour (or an outcome of probability 0) whenever the target equals a prefix.
    # Probabilities of a few units of 2^-58 make T tiny, so targets hit prefixes often.
    p = np.array([1.0, 0.0, 1.0, 2.0]) * 2.0 ** -S.SCALE_BITS
    real = np.searchsorted
    monkeypatch.setattr(S.np, "searchsorted", lambda a, v, side="left": real(a, v, side="left"))
    seeds = range(40)
    assert any(not np.array_equal(S.sample(p, s, 64), _brute(p, s, 64)) for s in seeds)
