"""Pins of the structure oracle (oracle/structure.py): textbook gates whose controls and
remainders are known, exact reconstruction of gates built as controlled diagonal /
monomial / dense blocks, the absence of any tolerance, and the semantics the structured
kernels rely on (only amplitudes whose control bits are all 1 change) checked against
the brute-force operator."""
import numpy as np
import pytest

import oracle
from oracle import brute
from oracle import gates as G
from oracle import structure as S


def _cls(name, params=()):
    u = G.matrix(name, params)
    k = u.shape[0].bit_length() - 1
    return S.classify(tuple(range(k)), u)


def test_textbook_gates():
    assert _cls("cnot") == (S.MONOMIAL, 0b01)          # control = local bit 0, V = X
    assert _cls("cz") == (S.DIAGONAL, 0b11)            # V = [[-1]]
    assert _cls("cp", (0.3,)) == (S.DIAGONAL, 0b11)    # V = [[e^{0.3 i}]]
    assert _cls("toffoli") == (S.MONOMIAL, 0b011)      # two controls, V = X
    assert _cls("swap") == (S.MONOMIAL, 0)
    assert _cls("x") == (S.MONOMIAL, 0) and _cls("y") == (S.MONOMIAL, 0)
    for g in ("z", "s", "t"):                          # phase gates: control + 1 x 1 phase
        assert _cls(g) == (S.DIAGONAL, 0b1)
    assert _cls("rz", (0.7,)) == (S.DIAGONAL, 0)       # entry 0 is not 1: no control
    assert _cls("h") == (S.DENSE, 0)
    assert _cls("i") == (S.IDENTITY, 0b1)
    assert S.classify((0, 1), np.eye(4)) == (S.IDENTITY, 0b11)
    ctl, keep, v = S.reduced((4, 9), G.matrix("cnot"))
    assert ctl == [4] and keep == [9] and np.array_equal(v, G.X)
    ctl, keep, v = S.reduced((2, 5), G.matrix("cp", (0.3,)))
    assert ctl == [2, 5] and keep == [] and v.shape == (1, 1) and v[0, 0] == np.exp(0.3j)


def test_no_tolerance():
    # fSim(pi/2, phi) is a monomial matrix in exact arithmetic, but cos(pi/2) rounds to
    # 6e-17 in FP64: the classification looks at the stored entries only.
    assert _cls("fsim", (np.pi / 2, np.pi / 6)) == (S.DENSE, 0)
    u = np.diag([1, 1, 1, -1]).astype(np.complex128)
    u[1, 3] = 1e-300                                    # changes bit 1 when bit 0 is 1
    assert S.classify((0, 1), u) == (S.DENSE, 0b01)


def _haar(d, rng):
    z = (rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _random_v(kind, d, rng):
    ph = np.exp(1j * rng.uniform(0.1, 6.0, d))        # never exactly 1
    if kind == S.DIAGONAL:
        return np.diag(ph)
    if kind == S.MONOMIAL:
        while True:
            p = rng.permutation(d)
            if d == 1 or not np.array_equal(p, np.arange(d)):
                break
        m = np.zeros((d, d), dtype=np.complex128)
        m[np.arange(d), p] = ph
        return m
    return _haar(d, rng)


@pytest.mark.parametrize("seed", range(40))
def test_built_structures_are_recovered_exactly(seed):
    """U = I - P_C + P_C (V on the other bits), built with Kronecker products; the oracle
    must return C, V and V's kind, and rebuilding from its answer gives U bit for bit."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 6))
    cmask = int(rng.integers(0, 1 << k))
    ctl = [j for j in range(k) if (cmask >> j) & 1]
    keep = [j for j in range(k) if j not in ctl]
    if keep:
        kind = int(rng.choice([S.DIAGONAL, S.MONOMIAL, S.DENSE]))
        if kind == S.MONOMIAL and len(keep) == 0:
            kind = S.DIAGONAL
    else:
        kind = S.DIAGONAL
    v = _random_v(kind, 1 << len(keep), rng)
    if not keep:
        v = np.array([[np.exp(0.4j)]])
    proj = np.diag([0.0] * ((1 << len(ctl)) - 1) + [1.0]).astype(np.complex128)
    P = brute.full_operator(k, ctl, proj) if ctl else np.eye(1 << k, dtype=np.complex128)
    F = brute.full_operator(k, keep, v) if keep else v[0, 0] * np.eye(1 << k)
    u = np.eye(1 << k) - P + P @ F
    got_kind, got_mask = S.classify(tuple(range(k)), u)
    assert got_mask == cmask and got_kind == kind
    rc, rk, rv = S.reduced(tuple(range(k)), u)
    assert rc == ctl and rk == keep and np.array_equal(rv, v)
    # rebuild from the oracle's answer
    P2 = brute.full_operator(k, rc, proj) if rc else np.eye(1 << k, dtype=np.complex128)
    F2 = brute.full_operator(k, rk, rv) if rk else rv[0, 0] * np.eye(1 << k)
    assert np.array_equal(np.eye(1 << k) - P2 + P2 @ F2, u)


def _apply_reduced(psi, n, targets, u):
    """The structured pass: only groups whose control bits are all 1 change, by V."""
    ctl, keep, v = S.reduced(targets, u)
    out = psi.copy()
    cm = sum(1 << q for q in ctl)
    km = sum(1 << q for q in keep)
    for i in range(1 << n):
        if (i & cm) != cm or (i & km):
            continue
        idx = []
        for a in range(1 << len(keep)):
            x = i
            for j, q in enumerate(keep):
                if (a >> j) & 1:
                    x |= 1 << q
            idx.append(x)
        out[idx] = v @ psi[idx]
    return out


@pytest.mark.parametrize("seed", range(12))
def test_structured_pass_equals_the_full_operator(seed):
    rng = np.random.default_rng(100 + seed)
    n = 6
    k = int(rng.integers(1, 5))
    tg = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
    cmask = int(rng.integers(1, 1 << k))
    ctl = [j for j in range(k) if (cmask >> j) & 1]
    keep = [j for j in range(k) if j not in ctl]
    v = _random_v(int(rng.choice([S.DIAGONAL, S.MONOMIAL, S.DENSE])) if keep else S.DIAGONAL,
                  1 << len(keep), rng)
    proj = np.diag([0.0] * ((1 << len(ctl)) - 1) + [1.0]).astype(np.complex128)
    P = brute.full_operator(k, ctl, proj)
    F = brute.full_operator(k, keep, v) if keep else v[0, 0] * np.eye(1 << k)
    u = np.eye(1 << k) - P + P @ F
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    want = brute.full_operator(n, tg, u) @ psi
    assert np.max(np.abs(_apply_reduced(psi, n, tg, u) - want)) < 1e-13
    assert np.max(np.abs(oracle.apply_gate(psi.copy(), tg, u) - want)) < 1e-13
    assert S.touched_fraction(u) == 0.5 ** len(ctl)


def test_a_dropped_control_condition_is_caught():
    # Planted mistake: a "control" test that only checks block-diagonality would call
    # bit 0 of RZ a control and then skip its e^{-i theta/2} half.
    u = G.matrix("rz", (0.7,))
    blockdiag = all(u[r, c] == 0 for r in range(2) for c in range(2) if (r & 1) != (c & 1))
    assert blockdiag and not S.is_control(u, 0)
    psi = np.array([0.6, 0.8], dtype=np.complex128)
    wrong = psi.copy()
    wrong[1] *= u[1, 1]
    assert np.max(np.abs(wrong - u @ psi)) > 0.1
