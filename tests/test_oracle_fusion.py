"""Pins for the oracle's DAG fusion (Algorithm 2) and precision rule (Eqs. 11-12)."""
import math

import numpy as np
import pytest

import oracle
from oracle import brute, fusion, precision
from oracle import gates as G
import workloads as W


def _op(n, gl):
    return brute.circuit_operator(n, gl)


@pytest.mark.parametrize("qmax", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("seed", range(3))
def test_fused_equals_unfused_random(qmax, seed):
    # Eq. 10: fusing adjacent gates leaves U_m ... U_1 unchanged.
    rng = np.random.default_rng(1000 * qmax + seed)
    n = 7
    gl = G.gate_list(W.random_unitary_gates(n, 25, 3, rng))
    fused = oracle.fuse(gl, n, qmax)
    assert all(len(t) <= max(qmax, 3) for t, _ in fused)
    assert all(list(t) == sorted(t) for t, _ in fused)
    assert np.max(np.abs(_op(n, fused) - _op(n, gl))) < 1e-12


@pytest.mark.parametrize("qmax", [2, 3, 4, 5])
def test_fused_equals_unfused_structured(qmax):
    n = 8
    x, specs = W.qft_brickwork(n, 3, seed=7)
    for circ in (specs, W.grid_random(n, 6, seed=3), W.hea(n, 2, seed=4), W.brickwork(n, 5)):
        gl = G.gate_list(circ)
        fused = oracle.fuse(gl, n, qmax)
        assert len(fused) < len(gl)
        assert all(len(t) <= qmax for t, _ in fused)
        psi_f = oracle.run(oracle.basis(n, x), fused)
        psi_u = oracle.run(oracle.basis(n, x), gl)
        assert np.max(np.abs(psi_f - psi_u)) < 1e-12


def test_fusion_order_is_v_times_u():
    # Eq. 9: U_fused = U_v . U_u, u applied first.
    f = oracle.fuse([((0,), G.H), ((0,), G.S)], 1, 1)
    assert len(f) == 1 and np.allclose(f[0][1], G.S @ G.H)
    assert not np.allclose(G.S @ G.H, G.H @ G.S)


def test_bell_fuses_to_one_gate():
    gl = G.gate_list(W.bell())
    f = oracle.fuse(gl, 2, 2)
    assert len(f) == 1 and f[0][0] == (0, 1)
    assert np.allclose(f[0][1], G.matrix("cnot") @ np.kron(np.eye(2), G.H))


def test_no_fusion_when_qmax_zero():
    gl = [((3, 1), G.matrix("cnot")), ((2,), G.H)]
    f = oracle.fuse(gl, 4, 0)
    assert [t for t, _ in f] == [(1, 3), (2,)]
    # sorting targets relabels the matrix: CNOT with control 3, target 1
    assert np.allclose(brute.full_operator(4, (1, 3), f[0][1]),
                       brute.full_operator(4, (3, 1), G.matrix("cnot")))


def test_detour_blocks_fusion():
    # u=(0,1) -> x=(1,4,5) -> v=(0,4) and u -> v directly.  |q(u)|q(v)| = 3 <= 3, but
    # contracting (u, v) would put x both before and after the fused gate: no fusion.
    rng = np.random.default_rng(2)
    specs = W.random_unitary_gates(6, 3, 1, rng)
    u2 = G.gate_list(W.random_unitary_gates(2, 1, 2, rng))[0][1]
    if u2.shape[0] != 4:
        u2 = np.kron(G.H, u2)
    u3 = np.kron(G.H, u2)
    gl = [((0, 1), u2), ((1, 4, 5), u3), ((0, 4), u2)]
    f = oracle.fuse(gl, 6, 3)
    assert len(f) == 3
    assert np.max(np.abs(_op(6, f) - _op(6, gl))) < 1e-12
    del specs


def test_chain_of_single_qubit_gates():
    rng = np.random.default_rng(8)
    gl = [((2,), G.matrix("u3", tuple(rng.uniform(0, 6, 3)))) for _ in range(7)]
    f = oracle.fuse(gl, 3, 1)
    want = np.eye(2)
    for _, u in gl:
        want = u @ want
    assert len(f) == 1 and np.allclose(f[0][1], want, atol=1e-14)


def test_sort_targets_and_embed_against_kronecker():
    rng = np.random.default_rng(4)
    (spec,) = W.random_unitary_gates(6, 1, 3, rng)
    tg, u = G.gate_list([spec])[0]
    st, su = fusion.sort_targets(tg, u)
    assert np.allclose(brute.full_operator(6, st, su), brute.full_operator(6, tg, u))
    sup = tuple(sorted(set(st) | {5 - st[0]} | {0}))
    e = fusion.embed(su, st, sup)
    assert np.allclose(brute.full_operator(6, sup, e), brute.full_operator(6, st, su))


def test_precision_rule_printed_value():
    # Section 5.4: n = 20, g = 200 gives about 2.5e1 for the left-hand side of Eq. 12.
    v = precision.eps_round(20, 200)
    assert abs(v - 24.96) < 0.01
    assert float(f"{v:.1e}") == 25.0
    assert not precision.choose_c64(20, 200, 1e-6)
    assert precision.choose_c64(4, 10, 1e-3)          # 10 * 16 * 1.19e-7 = 1.9e-5
    # boundary: equality selects complex64
    g, n = 10, 4
    assert precision.choose_c64(n, g, precision.eps_round(n, g))
    assert precision.eps_round(20, 200, precision.EPS_MACH_F64) < 1e-6


def test_detour_check_is_load_bearing(monkeypatch):
    # Planted mistake in the oracle: without the detour check the contraction makes a
    # cycle, which the topological sort detects.
    rng = np.random.default_rng(2)
    u2 = np.kron(G.H, G.gate_list(W.random_unitary_gates(1, 1, 1, rng))[0][1])
    u3 = np.kron(G.H, u2)
    gl = [((0, 1), u2), ((1, 4, 5), u3), ((0, 4), u2)]
    monkeypatch.setattr(fusion.Dag, "other_path", lambda self, u, v: False)
    with pytest.raises(AssertionError):
        oracle.fuse(gl, 6, 3)
