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


# ----------------------------------------------------------- commutation-aware variant

def _diag_heavy(n, count, rng):
    """Random circuits where most gates are diagonal (CZ, CP, RZ, T, Z) or controlled
    (CNOT, Toffoli), with some dense ones (H, U3, random 2-qubit unitaries)."""
    gl = []
    for _ in range(count):
        r = rng.random()
        q = [int(x) for x in rng.choice(n, 3, replace=False)]
        if r < 0.25:
            gl.append(((q[0], q[1]), G.matrix("cp", (float(rng.uniform(0, 6)),))))
        elif r < 0.33:
            gl.append(((q[0],), G.matrix("rz", (float(rng.uniform(0, 6)),))))
        elif r < 0.4:
            gl.append(((q[0],), G.matrix(str(rng.choice(["t", "z"])))))
        elif r < 0.5:
            gl.append(((q[0], q[1]), G.matrix("cz")))
        elif r < 0.65:
            gl.append(((q[0], q[1]), G.matrix("cnot")))
        elif r < 0.7:
            gl.append(((q[0], q[1], q[2]), G.matrix("toffoli")))
        elif r < 0.85:
            gl.append(((q[0],), G.matrix("h")))
        else:
            gl.append(((q[0], q[1]), G.gate_list(W.random_unitary_gates(2, 1, 2, rng, exact_k=True,
                                                                       targets=(0, 1)))[0][1]))
    return gl


def test_diagonal_on_qubit():
    assert fusion.diagonal_on(G.matrix("cnot"), 0) and not fusion.diagonal_on(G.matrix("cnot"), 1)
    assert fusion.diagonal_on(G.matrix("cz"), 0) and fusion.diagonal_on(G.matrix("cz"), 1)
    assert not fusion.diagonal_on(G.matrix("swap"), 0) and not fusion.diagonal_on(G.H, 0)
    assert fusion.diagonal_on(G.matrix("toffoli"), 1) and not fusion.diagonal_on(G.matrix("toffoli"), 2)


def test_commuting_gates_fuse_around_a_blocker():
    """CP(0,1), CP(1,2), CP(0,1)': Algorithm 2 keeps three gates at width 2 (the middle
    gate separates the two CP(0,1) on qubit 1); all three commute, so the commutation-
    aware variant fuses the outer two.  With an H on qubit 1 in between they no longer
    commute and stay apart."""
    a, b, c = (G.matrix("cp", (t,)) for t in (0.3, 0.5, 0.7))
    gl = [((0, 1), a), ((1, 2), b), ((0, 1), c)]
    assert len(oracle.fuse(gl, 3, 2)) == 3
    f = oracle.fuse(gl, 3, 2, commute=True)
    assert [t for t, _ in f] == [(0, 1), (1, 2)]
    assert np.array_equal(np.diag(f[0][1]), np.diag(c @ a))
    blocked = [((0, 1), a), ((1,), G.H), ((1, 2), b), ((0, 1), c)]
    f2 = oracle.fuse(blocked, 3, 2, commute=True)
    assert np.max(np.abs(_op(3, f2) - _op(3, blocked))) < 1e-13
    assert not any(t == (0, 1) and np.allclose(u, c @ a) for t, u in f2)


@pytest.mark.parametrize("qmax", [2, 3, 4, 5])
@pytest.mark.parametrize("seed", range(4))
def test_commutation_fused_equals_unfused(qmax, seed):
    # Any topological order of the commutation DAG gives the same product (Eq. 10).
    rng = np.random.default_rng(300 + 10 * qmax + seed)
    n = 7
    gl = _diag_heavy(n, 40, rng)
    fused = oracle.fuse(gl, n, qmax, commute=True)
    assert all(len(t) <= max(qmax, 3) for t, _ in fused)
    assert np.max(np.abs(_op(n, fused) - _op(n, gl))) < 1e-12
    assert len(fused) <= len(oracle.fuse(gl, n, qmax)) + 3


def test_commutation_dag_edges_are_needed(monkeypatch):
    # Planted mistake in the oracle: calling every gate diagonal on every qubit drops the
    # edges that order H against the phases around it, and the fused product changes.
    rng = np.random.default_rng(4)
    dense = G.gate_list(W.random_unitary_gates(3, 1, 2, rng, exact_k=True, targets=(0, 2)))[0][1]
    gl = [((0, 1), G.matrix("cp", (0.4,))), ((0, 2), dense), ((0, 1), G.matrix("cp", (1.1,)))]
    good = oracle.fuse(gl, 3, 2, commute=True)
    assert len(good) == 3
    assert np.max(np.abs(_op(3, good) - _op(3, gl))) < 1e-13
    monkeypatch.setattr(fusion, "diagonal_on", lambda u, j: True)
    bad = oracle.fuse(gl, 3, 2, commute=True)
    assert np.max(np.abs(_op(3, bad) - _op(3, gl))) > 0.1
