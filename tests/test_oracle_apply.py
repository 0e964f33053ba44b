"""Pins for the oracle's amplitude loops: brute-force Kronecker products (Eq. 3), closed
forms (Bell, GHZ-n, QFT of a basis state, uniform superposition), norm preservation,
mirror circuits, and the reductions against explicit operators."""
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle import gates as G
import workloads as W


def _rand_state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex128)


@pytest.mark.parametrize("seed", range(6))
def test_apply_matches_kronecker(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 9))
    specs = W.random_unitary_gates(n, 12, 5, rng)
    psi0 = _rand_state(n, rng)
    psi = oracle.run(psi0.copy(), G.gate_list(specs))
    want = brute.circuit_operator(n, G.gate_list(specs)) @ psi0
    assert np.max(np.abs(psi - want)) < 1e-13


def test_a_transposed_matrix_is_caught():
    # Planted mistake: applying U^T instead of U must fail the Kronecker pin.
    rng = np.random.default_rng(11)
    n = 4
    (spec,) = W.random_unitary_gates(n, 1, 2, rng)
    tg, u = G.gate_list([spec])[0]
    psi0 = _rand_state(n, rng)
    wrong = oracle.apply_gate(psi0.copy(), tg, u.T.copy())
    want = brute.full_operator(n, tg, u) @ psi0
    assert np.max(np.abs(wrong - want)) > 1e-3


def test_reversed_targets_are_caught():
    rng = np.random.default_rng(12)
    n = 5
    (spec,) = W.random_unitary_gates(n, 1, 2, rng)
    tg, u = G.gate_list([spec])[0]
    if len(tg) == 1:
        tg = (tg[0], (tg[0] + 1) % n)
        u = np.kron(G.matrix("h"), u)
    psi0 = _rand_state(n, rng)
    wrong = oracle.apply_gate(psi0.copy(), tuple(reversed(tg)), u)
    want = brute.full_operator(n, tg, u) @ psi0
    assert np.max(np.abs(wrong - want)) > 1e-3


def test_bell():
    psi = oracle.simulate(2, W.bell())
    want = np.zeros(4, complex)
    want[0] = want[3] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - want)) < 1e-15


@pytest.mark.parametrize("n", [2, 3, 5, 8, 10, 14])
def test_ghz(n):
    psi = oracle.simulate(n, W.ghz(n))
    want = np.zeros(1 << n, complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - want)) < 1e-15


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9, 12])
def test_qft_of_basis_state(n):
    rng = np.random.default_rng(n)
    for x in {0, (1 << n) - 1, int(rng.integers(0, 1 << n))}:
        psi = oracle.simulate(n, W.qft(n), x=x)
        y = np.arange(1 << n)
        want = np.exp(2j * np.pi * x * y / (1 << n)) / math.sqrt(1 << n)
        assert np.max(np.abs(psi - want)) < 1e-13


def test_qft_operator_is_dft_matrix():
    n = 6
    op = brute.circuit_operator(n, G.gate_list(W.qft(n)))
    N = 1 << n
    xy = np.outer(np.arange(N), np.arange(N))
    assert np.max(np.abs(op - np.exp(2j * np.pi * xy / N) / math.sqrt(N))) < 1e-13


def test_uniform_superposition():
    n = 11
    psi = oracle.simulate(n, [W.GateSpec("h", (q,)) for q in range(n)])
    assert np.max(np.abs(psi - 2 ** (-n / 2))) < 1e-15


def test_norm_preserved_and_mirror_returns_input():
    n = 12
    specs = W.brickwork(n, 20)
    psi = oracle.simulate(n, specs)
    assert abs(oracle.norm(psi) - 1) < 1e-13
    x = 1234
    back = oracle.simulate(n, W.mirror(specs), x=x)
    assert abs(abs(back[x]) - 1) < 1e-12
    assert abs(oracle.norm(back) - 1) < 1e-12


def test_probs_norm_inner():
    rng = np.random.default_rng(3)
    a, b = _rand_state(9, rng), _rand_state(9, rng)
    assert np.allclose(oracle.probs(a), np.abs(a) ** 2, atol=1e-16)
    assert abs(oracle.norm(a) - np.vdot(a, a).real) < 1e-14
    assert abs(oracle.inner(a, b) - np.vdot(a, b)) < 1e-14
    assert abs(oracle.fidelity(a, a) - 1) < 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_pauli_expectation_matches_operator(seed):
    rng = np.random.default_rng(100 + seed)
    n = 7
    psi = _rand_state(n, rng)
    for _ in range(10):
        x, z = int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n))
        want = np.vdot(psi, brute.pauli_operator(n, x, z) @ psi)
        got = oracle.expect_pauli(psi, x, z)
        assert abs(got - want) < 1e-13
        assert abs(got.imag) < 1e-13


def test_pauli_closed_forms():
    bell = oracle.simulate(2, W.bell())
    assert abs(oracle.expect_pauli(bell, 0, 0b11) - 1) < 1e-15       # <Z0 Z1> = 1
    assert abs(oracle.expect_pauli(bell, 0b11, 0) - 1) < 1e-15       # <X0 X1> = 1
    assert abs(oracle.expect_pauli(bell, 0b11, 0b11) + 1) < 1e-15    # <Y0 Y1> = -1
    assert abs(oracle.expect_pauli(bell, 0, 0b01)) < 1e-15           # <Z0> = 0
    n = 10
    g = oracle.simulate(n, W.ghz(n))
    for i in range(n - 1):
        assert abs(oracle.expect_pauli(g, 0, 3 << i) - 1) < 1e-14
    assert abs(oracle.expect_pauli(g, (1 << n) - 1, 0) - 1) < 1e-14  # <X^n> = 1
    xs, zs, cs = W.zz_chain(n)
    assert abs(oracle.expect(g, xs, zs, cs) - (n - 1)) < 1e-13


def test_zz_chain_weight_closed_form():
    n = 9
    k = np.arange(1 << n)
    direct = np.zeros(1 << n, dtype=np.int64)
    for i in range(n - 1):
        direct += 1 - 2 * (((k >> i) & 1) ^ ((k >> (i + 1)) & 1))
    assert np.array_equal(oracle.zz_chain_weight(n, k), direct)


def test_topk_order_and_ties():
    rng = np.random.default_rng(9)
    p = rng.integers(0, 5, size=300).astype(float)           # many exact ties
    idx, val = oracle.topk(p, 64)
    want = sorted(range(300), key=lambda i: (-p[i], i))[:64]
    assert list(idx) == want and np.array_equal(val, p[want])
    n = 7
    u = oracle.probs(oracle.simulate(n, [W.GateSpec("h", (q,)) for q in range(n)]))
    idx, _ = oracle.topk(u, 64)
    assert list(idx) == list(range(64))
    small, _ = oracle.topk(np.array([0.1, 0.9, 0.0]), 64)    # fewer than 64 outcomes
    assert list(small) == [1, 0, 2]


def test_probs_in_precision_and_topk_valid():
    rng = np.random.default_rng(21)
    psi = _rand_state(8, rng)
    assert np.array_equal(oracle.probs_in_precision(psi), oracle.probs(psi))
    p32 = oracle.probs_in_precision(psi.astype(np.complex64))
    assert p32.dtype == np.float32
    assert np.max(np.abs(p32 - oracle.probs(psi))) < 1e-6
    p = oracle.probs(psi)
    idx, _ = oracle.topk(p, 10)
    assert oracle.topk_valid(idx, p, 10, 0.0)
    bad = idx.copy()
    bad[3] = np.argmin(p)
    assert not oracle.topk_valid(bad, p, 10, 1e-9)
    assert not oracle.topk_valid(np.array([idx[0], idx[0]]), p, 2, 1.0)
