"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and its
host-only entry points (gate library, sv_fuse, the precision rule, argument checks)
agree with the oracle.  No GPU call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from oracle import gates as OG
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "sv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sv_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(svlib):
    lib = ctypes.CDLL(svlib.LIB_PATH)
    declared = _declared_symbols()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(svlib.EXPORTS)


def test_gate_library_matches_oracle(svlib):
    rng = np.random.default_rng(0)
    for name, npar in [("i", 0), ("x", 0), ("y", 0), ("z", 0), ("h", 0), ("s", 0), ("t", 0),
                       ("rx", 1), ("ry", 1), ("rz", 1), ("u3", 3), ("sqrtx", 0), ("sqrty", 0),
                       ("sqrtw", 0), ("cnot", 0), ("cz", 0), ("swap", 0), ("toffoli", 0),
                       ("fsim", 2), ("cp", 1)]:
        for dagger in (False, True):
            p = tuple(rng.uniform(-7, 7, npar))
            got = svlib.sv_gate_matrix(name, p, dagger)
            want = OG.matrix(name, p, dagger)
            assert np.max(np.abs(got - want)) < 1e-15, name
    (spec,) = W.random_unitary_gates(5, 1, 3, rng)
    u = OG.matrix("unitary", (), False, spec.matrix)
    assert np.array_equal(svlib.sv_gate_matrix("unitary", matrix=spec.matrix), u)
    assert np.array_equal(svlib.sv_gate_matrix("unitary", dagger=True, matrix=spec.matrix),
                          u.conj().T)


def _compare_fusion(svlib, specs, n, k):
    want = oracle.fuse(OG.gate_list(specs), n, k)
    c = svlib.sv_fuse(svlib.gates_from_specs(specs), n, k)
    assert len(c) == len(want)
    for i, (tw, uw) in enumerate(want):
        tg, ug = svlib.sv_circuit_gate(c, i)
        assert tg == tuple(tw), (i, tg, tw)                  # schedule: bit-exact
        assert np.max(np.abs(ug - uw)) < 1e-12               # FP64 products
    return len(want)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5])
def test_fusion_matches_oracle_random(svlib, k):
    rng = np.random.default_rng(40 + k)
    for n in (3, 6, 9):
        _compare_fusion(svlib, W.random_unitary_gates(n, 60, 3, rng), n, k)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_fusion_matches_oracle_qft_brickwork_24q(svlib, k):
    _, specs = W.qft_brickwork(24, 40)
    assert len(specs) == 2192
    _compare_fusion(svlib, specs, 24, k)


@pytest.mark.parametrize("n,k", [(30, 4), (30, 5), (33, 5), (32, 3)])
def test_fusion_matches_oracle_grid(svlib, n, k):
    _compare_fusion(svlib, W.grid_random(n, 24), n, k)


def test_fusion_matches_oracle_other_families(svlib):
    for k in (1, 2, 3, 5):
        _compare_fusion(svlib, W.brickwork(12, 20), 12, k)
        _compare_fusion(svlib, W.hea(18, 6, seed=1), 18, k)
        _compare_fusion(svlib, W.qft(20, swaps=False), 20, k)


def test_precision_rule_matches_oracle(svlib):
    from oracle import precision
    for n, g, tol in [(20, 200, 1e-6), (4, 10, 1e-3), (16, 49, 1.0), (30, 1014, 1e3)]:
        dt, e = svlib.sv_choose_dtype(n, g, tol)
        assert e == pytest.approx(precision.eps_round(n, g), rel=1e-15)
        assert (dt == svlib.SV_C64) == precision.choose_c64(n, g, tol)


def test_argument_errors_are_reported(svlib):
    h = svlib.sv_gate_matrix("h")
    with pytest.raises(svlib.SvError) as e:
        svlib.sv_fuse([((0, 0), np.eye(4))], 4, 2)
    assert e.value.status == 1 and "repeated" in str(e.value)
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse([((5,), h)], 4, 2)                    # target >= n
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse([((0, 1, 2, 3, 4, 5), np.eye(64))], 8, 2)   # k > 5
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse([((0,), h)], 4, 6)                    # max_k > 5
    with pytest.raises(svlib.SvError):
        svlib.sv_gate_matrix("rx", ())                      # missing angle
    with pytest.raises(svlib.SvError):
        svlib.sv_alloc(0)                                   # n out of range, no GPU call
    with pytest.raises(svlib.SvError):
        svlib.sv_alloc(35)


def test_fuse_like_equals_fuse(svlib):
    # Algorithm 2's decisions depend on the qubits only: replaying them on new angles
    # gives exactly what a fresh fusion gives.
    for n, k in ((16, 4), (22, 4), (12, 5), (9, 2)):
        pat = svlib.sv_fuse(svlib.gates_from_specs(W.hea(n, 6, seed=1)), n, k)
        for seed in (2, 3):
            gl = svlib.gates_from_specs(W.hea(n, 6, seed=seed))
            a = svlib.sv_fuse(gl, n, k)
            b = svlib.sv_fuse_like(pat, gl)
            assert len(a) == len(b)
            for i in range(len(a)):
                ta, ua = svlib.sv_circuit_gate(a, i)
                tb, ub = svlib.sv_circuit_gate(b, i)
                assert ta == tb and np.array_equal(ua, ub)
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse_like(pat, svlib.gates_from_specs(W.brickwork(9, 2)))


def test_density_fusion_matches_density_oracle(svlib):
    """sv_fuse_density's fused 2n-qubit schedule, applied by the state-vector oracle to
    vec(|0><0|), gives vec(rho) of the density-matrix oracle (host only)."""
    from oracle import density as D
    rng = np.random.default_rng(77)
    for n, p, k in ((2, 0.01, 2), (3, 0.05, 4), (4, 0.2, 5), (3, 0.0, 3), (4, 0.1, 0)):
        specs = W.random_unitary_gates(n, 8, 2, rng) if n > 2 else W.bell()
        c = svlib.sv_fuse_density(svlib.gates_from_specs(specs), n, p, k)
        nf, n2 = svlib.sv_circuit_size(c)
        assert n2 == 2 * n
        v = oracle.basis(2 * n, 0)
        for i in range(nf):
            tg, u = svlib.sv_circuit_gate(c, i)
            v = oracle.apply_gate(v, tg, u)
        rho = D.run(n, OG.gate_list(specs), p)
        assert np.max(np.abs(v - D.vec(rho))) < 1e-13, (n, p, k)
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse_density(svlib.gates_from_specs(W.bell()), 18, 0.01, 4)   # 2n > 34
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse_density(svlib.gates_from_specs(W.bell()), 2, 1.5, 4)


def _structured_gate(rng, k):
    """A k-qubit gate I - P_C + P_C (V on the rest) with a random control set C and a
    random diagonal / monomial / dense V (Kronecker construction, as in the oracle pins)."""
    from oracle import brute
    cmask = int(rng.integers(0, 1 << k))
    ctl = [j for j in range(k) if (cmask >> j) & 1]
    keep = [j for j in range(k) if j not in ctl]
    d = 1 << len(keep)
    ph = np.exp(1j * rng.uniform(0.1, 6.0, d))
    kind = int(rng.integers(0, 3))
    if kind == 0:
        v = np.diag(ph)
    elif kind == 1:
        v = np.zeros((d, d), dtype=np.complex128)
        v[np.arange(d), rng.permutation(d)] = ph
    else:
        z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
        v = np.linalg.qr(z)[0]
    proj = np.diag([0.0] * ((1 << len(ctl)) - 1) + [1.0]).astype(np.complex128)
    P = brute.full_operator(k, ctl, proj) if ctl else np.eye(1 << k, dtype=np.complex128)
    F = brute.full_operator(k, keep, v) if keep else v[0, 0] * np.eye(1 << k)
    return np.eye(1 << k) - P + P @ F


def test_gate_structure_matches_oracle(svlib):
    """sv_gate_structure (controls in the caller's target order, the reduced gate's kind)
    against oracle/structure.py on textbook gates, built structured gates with shuffled
    targets, and the fused gates of QFT / brickwork circuits."""
    from oracle import structure as OS
    cases = [((0,), OG.matrix(g, p)) for g, p in [("x", ()), ("z", ()), ("h", ()), ("rz", (0.4,)),
                                                    ("t", ()), ("i", ())]]
    cases += [((3, 1), OG.matrix(g, p)) for g, p in [("cnot", ()), ("cz", ()), ("cp", (0.9,)),
                                                       ("swap", ()), ("fsim", (0.3, 0.2))]]
    cases.append(((5, 0, 2), OG.matrix("toffoli")))
    rng = np.random.default_rng(17)
    for _ in range(60):
        k = int(rng.integers(1, 6))
        tg = tuple(int(q) for q in rng.permutation(8)[:k])
        cases.append((tg, _structured_gate(rng, k)))
    for specs, n in [(W.qft(10), 10), (W.brickwork(8, 6, seed=3), 8)]:
        for k in (2, 3, 5):
            cases += [(tuple(t), u) for t, u in oracle.fuse(OG.gate_list(specs), n, k)]
    kinds = set()
    for tg, u in cases:
        got = svlib.sv_gate_structure(tg, u)
        assert got == OS.classify(tg, u), (tg, got)
        kinds.add(got[0])
    assert kinds == {svlib.SV_STRUCT_DENSE, svlib.SV_STRUCT_DIAGONAL, svlib.SV_STRUCT_MONOMIAL,
                     svlib.SV_STRUCT_IDENTITY}


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_commutation_fusion_matches_oracle(svlib, k):
    """sv_fuse_ex(SV_FUSE_COMMUTE): the schedule (targets, in order) bit-exact against
    the oracle's commutation-aware Algorithm 2, the products to 1e-12."""
    cases = [(W.phase_heavy(7, 60, seed=k), 7), (W.qft(10), 10), (W.qaoa(9, 2, 14, seed=k), 9),
             (W.brickwork(8, 6, seed=3), 8), (W.hea(8, 2, seed=4), 8)]
    for specs, n in cases:
        want = oracle.fuse(OG.gate_list(specs), n, k, commute=True)
        c = svlib.sv_fuse_ex(svlib.gates_from_specs(specs), n, k, svlib.SV_FUSE_COMMUTE)
        assert len(c) == len(want)
        for i, (tw, uw) in enumerate(want):
            tg, ug = svlib.sv_circuit_gate(c, i)
            assert tg == tuple(tw), (i, tg, tw)
            assert np.max(np.abs(ug - uw)) < 1e-12


def test_commutation_fuse_like_checks_structure(svlib):
    n = 6
    specs = W.phase_heavy(n, 40, seed=11)
    pattern = svlib.sv_fuse_ex(svlib.gates_from_specs(specs), n, 3, svlib.SV_FUSE_COMMUTE)
    # a parameter sweep that keeps every gate's diagonal qubits replays exactly
    sweep = [s if s.name not in ("cp", "rz") else W.GateSpec(s.name, s.qubits, (s.params[0] + 0.5,))
             for s in specs]
    direct = svlib.sv_fuse_ex(svlib.gates_from_specs(sweep), n, 3, svlib.SV_FUSE_COMMUTE)
    like = svlib.sv_fuse_like(pattern, svlib.gates_from_specs(sweep))
    assert len(like) == len(direct)
    for i in range(len(direct)):
        a, b = svlib.sv_circuit_gate(like, i), svlib.sv_circuit_gate(direct, i)
        assert a[0] == b[0] and np.array_equal(a[1], b[1])
    # a CZ turned into a CNOT on the same qubits commutes differently: refused
    i = next(j for j, s in enumerate(specs) if s.name == "cz")
    changed = list(specs)
    changed[i] = W.GateSpec("cnot", specs[i].qubits)
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse_like(pattern, svlib.gates_from_specs(changed))
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse_ex(svlib.gates_from_specs(specs), n, 3, 2)


def test_new_entry_points_validate_arguments(svlib):
    """Host-only argument checks of sv_gate_structure and sv_fuse_ex (no GPU call)."""
    import ctypes
    lib = ctypes.CDLL(svlib.LIB_PATH)
    h = OG.matrix("h")
    with pytest.raises(svlib.SvError):
        svlib.sv_gate_structure((0, 0), np.eye(4))             # repeated target
    with pytest.raises(svlib.SvError):
        svlib.sv_gate_structure((0, 1, 2, 3, 4, 5), np.eye(64))  # wider than 5
    assert lib.sv_gate_structure(None, None, None) != 0         # null gate
    gl = [((0,), h), ((1,), h)]
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse_ex(gl, 2, 6, svlib.SV_FUSE_COMMUTE)      # max_k > 5
    with pytest.raises(svlib.SvError):
        svlib.sv_fuse_ex(gl, 1, 2, svlib.SV_FUSE_COMMUTE)      # target >= n
    c = svlib.sv_fuse_ex(gl, 2, 0, svlib.SV_FUSE_COMMUTE)      # max_k = 0: unfused
    assert len(c) == 2
    # either output of sv_gate_structure may be NULL
    ga = svlib.GateArray([((0, 1), OG.matrix("cz"))])
    kind = ctypes.c_uint32()
    assert lib.sv_gate_structure(ga.arr, ctypes.byref(kind), None) == 0 and kind.value == svlib.SV_STRUCT_DIAGONAL


def _tile_low_bits(u):
    """Largest L with L + #{targets >= L} <= 12 (the two-gate pass's tile of 2^12)."""
    for L in range(12, -1, -1):
        if L + sum(1 for t in u if t >= L) <= 12:
            return L
    return -1


@pytest.mark.parametrize("case", ["grid14", "random15", "qft_brickwork13", "random16_k3"])
def test_pass_plan_pairs_commuting_gates_within_one_tile(svlib, case):
    """The two-gate pass plan (sv_plan_passes, SV_POLICY_TWO_GATE_PASSES): every gate once; each pair fits one
    2^12-amplitude tile with segments of at least 2^5 amplitudes; two gates that share a
    qubit keep their schedule order (so only commuting gates are reordered, Eq. 8's DAG);
    only dense gates without controls are paired; and the oracle's state after the gates in
    plan order equals its state after the schedule."""
    sv = svlib
    rng = np.random.default_rng(4242)
    if case == "grid14":
        n, specs = 14, W.grid_random(14, 8)
    elif case == "random15":
        n, specs = 15, W.random_unitary_gates(15, 60, 5, rng)
    elif case == "qft_brickwork13":
        n, (_, specs) = 13, W.qft_brickwork(13, 6)
    else:
        n, specs = 16, W.random_unitary_gates(16, 80, 3, rng)
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, 5 if case != "random16_k3" else 3)
    nf, _ = sv.sv_circuit_size(c)
    gates = [sv.sv_circuit_gate(c, i) for i in range(nf)]
    plan = sv.sv_plan_passes(c)
    order = [g for a, b in plan for g in ((a,) if b < 0 else (a, b))]
    assert sorted(order) == list(range(nf))
    pairs = [(a, b) for a, b in plan if b >= 0]
    assert len(pairs) >= 1
    for a, b in pairs:
        assert _tile_low_bits(set(gates[a][0]) | set(gates[b][0])) >= 5
        for g in (a, b):
            kind, ctrl = sv.sv_gate_structure(gates[g][0], gates[g][1])
            assert kind == sv.SV_STRUCT_DENSE and ctrl == 0
    pos = {g: i for i, g in enumerate(order)}
    for i in range(nf):
        for j in range(i + 1, nf):
            if set(gates[i][0]) & set(gates[j][0]):
                assert pos[i] < pos[j], (i, j)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 = v / np.linalg.norm(v)
    ref = oracle.run(psi0, gates)
    got = oracle.run(psi0, [gates[g] for g in order])
    assert np.max(np.abs(got - ref)) <= 1e-12
    # no pairs by default or without tensor cores; every dense gate is a candidate with DENSE_ONLY
    P = sv.SV_POLICY_TWO_GATE_PASSES
    assert sv.sv_plan_passes(c, 0) == [(i, -1) for i in range(nf)]
    assert len(sv.sv_plan_passes(c, P | sv.SV_POLICY_DENSE_ONLY)) <= len(plan)
    assert sv.sv_plan_passes(c, P | sv.SV_POLICY_NO_TENSOR_CORES) == [(i, -1) for i in range(nf)]


def test_pass_plan_skips_only_gates_on_other_qubits(svlib):
    """A pair partner is taken from further on only past gates on other qubits: g0 on
    5..9 pairs with g2 on 5..8 and 15 (g1 on 10..14 shares no qubit with g2); when g1
    also acts on qubit 15, g2 must wait and no pair forms; gates whose union needs more
    than the tile's bits (L < 5) stay apart."""
    sv = svlib
    rng = np.random.default_rng(99)
    n = 16

    def plan(tsets):
        specs = [W.GateSpec("unitary", t, (), False, W.haar_unitary(1 << len(t), rng)) for t in tsets]
        c = sv.sv_fuse(sv.gates_from_specs(specs), n, 0)
        return sv.sv_plan_passes(c)

    assert plan([(5, 6, 7, 8, 9), (10, 11, 12, 13, 14), (5, 6, 7, 8, 15)]) == [(0, 2), (1, -1)]
    assert plan([(5, 6, 7, 8, 9), (10, 11, 12, 13, 15), (5, 6, 7, 8, 15)]) == [(0, -1), (1, -1), (2, -1)]
    assert plan([(5, 6, 7, 8, 9), (10, 11, 12, 13, 14)]) == [(0, -1), (1, -1)]
    assert plan([(0, 1, 2, 3, 4), (0, 9, 13, 14, 15)]) == [(0, 1)]
    assert plan([(3,), (7, 9)]) == [(0, 1)]


def test_plan_passes_validates_arguments(svlib):
    """sv_plan_passes: null arguments and a too-small output capacity are reported (host)."""
    import ctypes
    lib = ctypes.CDLL(svlib.LIB_PATH)
    rng = np.random.default_rng(5)
    specs = W.random_unitary_gates(14, 6, 5, rng)
    c = svlib.sv_fuse(svlib.gates_from_specs(specs), 14, 0)
    first = (ctypes.c_uint32 * 6)()
    second = (ctypes.c_int32 * 6)()
    npasses = ctypes.c_size_t()
    P = svlib.SV_POLICY_TWO_GATE_PASSES
    assert lib.sv_plan_passes(None, P, first, second, 6, ctypes.byref(npasses)) != 0
    assert lib.sv_plan_passes(ctypes.c_void_p(c.handle), P, None, second, 6, ctypes.byref(npasses)) != 0
    assert lib.sv_plan_passes(ctypes.c_void_p(c.handle), P, first, second, 6, None) != 0
    assert lib.sv_plan_passes(ctypes.c_void_p(c.handle), P, first, second, 0, ctypes.byref(npasses)) != 0
    assert npasses.value >= 1                      # the count is reported even when cap is short
    assert lib.sv_plan_passes(ctypes.c_void_p(c.handle), P, first, second, 6, ctypes.byref(npasses)) == 0
    assert 1 <= npasses.value <= 6
