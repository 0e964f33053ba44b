"""GPU parity of the structure-aware passes (controls skipped, diagonal and monomial
remainders, controlled dense remainders) through the C ABI, against the CPU oracle and
against the same gates forced through the dense kernels (SV_POLICY_DENSE_ONLY).

Tolerances as for every pass: complex128 within 1e-12 max-abs, complex64 within 1e-5
max-abs.  Amplitudes whose control bits are not all 1 must come back bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle import gates as OG
from oracle import structure as OS
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


def _torch():
    import torch
    return torch


def _structured(rng, k, kind=None, cmask=None):
    """I - P_C + P_C (V on the other bits): random controls C, V diagonal / monomial / dense."""
    if cmask is None:
        cmask = int(rng.integers(0, 1 << k))
    ctl = [j for j in range(k) if (cmask >> j) & 1]
    keep = [j for j in range(k) if j not in ctl]
    d = 1 << len(keep)
    kind = int(rng.integers(0, 3)) if kind is None else kind
    ph = np.exp(1j * rng.uniform(0.1, 6.0, d))
    if not keep or kind == 0:
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


def _state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def _apply(sv, n, dtype, tg, u, psi0, policy=0):
    s = sv.sv_alloc(n, dtype, stream=_torch().cuda.current_stream())
    sv.sv_set_policy(s, policy)
    sv.sv_set_state(s, psi0)
    sv.sv_apply_gate(s, tg, u)
    out = sv.sv_get_state(s).astype(np.complex128)
    s.free()
    return out


LAYOUTS = [(0, 1, 2, 3, 4), (1, 3, 6, 9, 12), (8, 12, 13, 15, 16), (0, 5, 11, 16, 17), (2, 4, 7, 10, 14)]


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("seed", range(10))
def test_structured_gates_match_oracle_and_dense_path(gpu, dtype, seed):
    sv = gpu
    rng = np.random.default_rng(500 + seed)
    n = 18
    psi0 = _state(n, rng)
    for k in range(1, 6):
        lay = LAYOUTS[(seed + k) % len(LAYOUTS)]
        tg = tuple(int(q) for q in rng.permutation(lay[:k]))
        for kind in (0, 1, 2):
            u = _structured(rng, k, kind)
            want = oracle.apply_gate(psi0.copy(), tg, u)
            got = _apply(sv, n, dtype, tg, u, psi0)
            err = float(np.max(np.abs(got - want)))
            assert err <= TOL[dtype], (k, tg, kind, OS.classify(tg, u), err)
            dense = _apply(sv, n, dtype, tg, u, psi0, policy=sv.SV_POLICY_DENSE_ONLY)
            assert float(np.max(np.abs(dense - want))) <= TOL[dtype]
            # untouched amplitudes (a control bit 0) come back bit for bit when the
            # structure-aware pass runs (complex128 takes a dense remainder only with
            # fewer targets than controls)
            ctl, keep, _ = OS.reduced(tg, u)
            structured = OS.kind(OS.reduced(tg, u)[2]) != OS.DENSE or (
                ctl and (dtype == 0 or len(keep) < len(ctl)))
            if ctl and structured:
                cm = sum(1 << q for q in ctl)
                idx = np.arange(1 << n)
                off = (idx & cm) != cm
                base = psi0.astype(np.complex64 if dtype == 0 else np.complex128).astype(np.complex128)
                assert np.array_equal(got[off], base[off])


@pytest.mark.parametrize("dtype", [0, 1])
def test_textbook_structured_gates(gpu, dtype):
    sv = gpu
    rng = np.random.default_rng(7)
    n = 14
    psi0 = _state(n, rng)
    cases = [((3, 9), OG.matrix("cnot")), ((9, 3), OG.matrix("cnot")), ((0, 13), OG.matrix("cz")),
             ((6, 1), OG.matrix("cp", (0.77,))), ((2, 11), OG.matrix("swap")),
             ((12, 0, 5), OG.matrix("toffoli")), ((4,), OG.matrix("x")), ((0,), OG.matrix("t")),
             ((7,), OG.matrix("rz", (1.3,))), ((10,), OG.matrix("y")), ((1, 2), np.eye(4)),
             ((0, 1), OG.matrix("fsim", (np.pi / 2, np.pi / 6)))]
    for tg, u in cases:
        want = oracle.apply_gate(psi0.copy(), tg, u)
        got = _apply(sv, n, dtype, tg, u, psi0)
        assert float(np.max(np.abs(got - want))) <= TOL[dtype], (tg, OS.classify(tg, u))


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [5, 7])
def test_small_states_all_controls(gpu, dtype, n):
    """Degenerate sizes: the whole state is one group, or the controlled subspace is a
    single amplitude (k = n with every bit a control but one)."""
    sv = gpu
    rng = np.random.default_rng(n)
    psi0 = _state(n, rng)
    k = 5
    tg = tuple(int(q) for q in rng.permutation(n)[:k])
    for cmask in (0b11111, 0b11110, 0b01111, 0b10101):
        for kind in (0, 1, 2):
            u = _structured(rng, k, kind, cmask)
            want = oracle.apply_gate(psi0.copy(), tg, u)
            got = _apply(sv, n, dtype, tg, u, psi0)
            assert float(np.max(np.abs(got - want))) <= TOL[dtype], (cmask, kind)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("k", [3, 5])
def test_qft_circuit_structure_vs_dense(gpu, dtype, k):
    """QFT-16 of a basis state, fused: the structure-aware schedule against the oracle's
    unfused state, with fewer algorithmic bytes than the dense schedule."""
    sv = gpu
    n, x = 16, 0x5A3C
    ref = oracle.simulate(n, W.qft(n), x)
    c = sv.sv_fuse(sv.gates_from_specs(W.qft(n)), n, k)
    reps = {}
    for policy in (0, sv.SV_POLICY_DENSE_ONLY):
        s = sv.sv_alloc(n, dtype, stream=_torch().cuda.current_stream())
        sv.sv_set_policy(s, policy)
        sv.sv_set_basis(s, x)
        reps[policy] = sv.sv_apply_circuit(s, c)
        psi = sv.sv_get_state(s).astype(np.complex128)
        s.free()
        assert float(np.max(np.abs(psi - ref))) <= TOL[dtype]
    # every fused gate is applied once either way (dense gates may share a pass)
    assert (reps[0]["passes"] + reps[0]["paired_passes"] ==
            reps[sv.SV_POLICY_DENSE_ONLY]["passes"] + reps[sv.SV_POLICY_DENSE_ONLY]["paired_passes"])
    assert reps[0]["bytes"] < 0.8 * reps[sv.SV_POLICY_DENSE_ONLY]["bytes"]


@pytest.mark.parametrize("dtype", [0, 1])
def test_qft_30q_closed_form_sampled(gpu, dtype):
    """Full size: QFT-30 of |x> fused at k = 5, as the QFT workload runs it; sampled
    amplitudes against 2^(-n/2) exp(2 pi i x y / 2^n), to 1e-4 (complex64) and 1e-9
    (complex128) of their modulus, and the norm."""
    torch = _torch()
    sv = gpu
    n, x = 30, 0x2B5D1C37
    c = sv.sv_fuse(sv.gates_from_specs(W.qft(n)), n, 5)
    buf = torch.empty(1 << n, dtype=torch.complex64 if dtype == 0 else torch.complex128, device="cuda")
    s = sv.sv_alloc(n, dtype, dev_buf=buf, stream=torch.cuda.current_stream())
    sv.sv_set_basis(s, x)
    sv.sv_apply_circuit(s, c)
    sv.sv_sync(s)
    rng = np.random.default_rng(30)
    ys = np.concatenate([[0, 1, (1 << n) - 1], rng.integers(0, 1 << n, 4000)])
    got = buf[torch.as_tensor(ys, device="cuda")].cpu().numpy().astype(np.complex128)
    ph = np.array([((x * int(y)) % (1 << n)) / float(1 << n) for y in ys])
    want = np.exp(2j * math.pi * ph) * 2.0 ** (-n / 2)
    rel = np.max(np.abs(got - want)) / 2.0 ** (-n / 2)
    assert rel <= (1e-4 if dtype == 0 else 1e-9), rel
    assert abs(sv.sv_norm(s) - 1.0) <= (1e-5 if dtype == 0 else 1e-12)
    s.free()
    del buf
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("k", [3, 5])
def test_commutation_fused_circuits(gpu, dtype, k):
    """Circuits fused with SV_FUSE_COMMUTE (reordered commuting gates) run on the
    structure-aware passes: the state equals the oracle's unfused one."""
    sv = gpu
    for specs, n in ((W.phase_heavy(16, 200, seed=21), 16), (W.qaoa(15, 3, 30, seed=22), 15),
                     (W.qft(14), 14)):
        x = 0x1234 & ((1 << n) - 1)
        ref = oracle.simulate(n, specs, x)
        c = sv.sv_fuse_ex(sv.gates_from_specs(specs), n, k, sv.SV_FUSE_COMMUTE)
        s = sv.sv_alloc(n, dtype, stream=_torch().cuda.current_stream())
        sv.sv_set_basis(s, x)
        sv.sv_apply_circuit(s, c)
        psi = sv.sv_get_state(s).astype(np.complex128)
        s.free()
        assert float(np.max(np.abs(psi - ref))) <= TOL[dtype]
