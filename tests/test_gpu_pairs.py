"""Two fused gates in one HBM pass (complex64, tensor cores, SV_POLICY_TWO_GATE_PASSES):
every tile layout the pass can take -- targets in the bank-selecting bits, high targets
moved as 256-byte segments, gates narrower than 5 qubits widened inside the tile, one tile
per CTA and several -- against the oracle, and whole fused circuits with and without
pairing."""
import numpy as np
import pytest

import oracle
from oracle import gates as OG
import workloads as W

pytestmark = pytest.mark.gpu


def _state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex64)


def _apply(sv, n, psi0, c, policy):
    import torch
    s = sv.sv_alloc(n, 0, stream=torch.cuda.current_stream())
    sv.sv_set_policy(s, policy)
    sv.sv_set_state(s, psi0)
    rep = sv.sv_apply_circuit(s, c)
    sv.sv_sync(s)
    out = sv.sv_get_state(s).astype(np.complex128)
    s.free()
    return out, rep


def _check(out, ref):
    err = float(np.max(np.abs(out - ref)))
    f = abs(np.vdot(ref, out)) ** 2 / np.vdot(out, out).real
    assert err <= 1e-5 and 1 - f <= 1e-6, (err, 1 - f)
    return err


PAIRS = [
    (13, (0, 1, 2, 3, 4), (8, 9, 10, 11, 12), True),          # one tile per CTA, L = 7
    (16, (0, 1, 2, 3, 4), (0, 1, 2, 3, 5), True),             # contiguous, bank targets in both
    (16, (8, 9, 10, 11, 12), (9, 10, 11, 13, 14), True),      # L = 5: 128 segments of 256 B
    (16, (0, 1, 10, 11, 12), (2, 3, 13, 14, 15), True),       # L = 6, bank targets in both
    (16, (3,), (7, 9), True),                                 # widths 1 and 2 widened
    (16, (0, 5, 10, 15), (1, 6, 11, 13, 14), True),           # width 4 with width 5
    (16, (1, 2, 3), (2, 3, 4, 5, 6), True),                   # overlapping, bank targets
    (16, (6, 7, 8, 9, 10), (4, 5, 6, 7, 8), True),            # bank-free first, low second
    (16, (4, 5, 6, 7, 8), (11, 12, 13, 14, 15), False),       # union too wide: two passes
    (21, (0, 1, 2, 3, 4), (16, 17, 18, 19, 20), True),        # several tiles per CTA
    (21, (2, 6, 15, 17, 20), (3, 6, 15, 18, 20), True),       # L = 8, bank targets
    (21, (13, 14, 15, 16, 17), (16, 17, 18, 19), True),       # L = 5, several tiles per CTA
]


@pytest.mark.parametrize("case", range(len(PAIRS)))
def test_pair_layouts_against_oracle(gpu, case):
    sv = gpu
    n, t0, t1, paired = PAIRS[case]
    rng = np.random.default_rng(7000 + case)
    specs = [W.GateSpec("unitary", t, (), False, W.haar_unitary(1 << len(t), rng)) for t in (t0, t1)]
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, 0)
    assert sv.sv_plan_passes(c) == ([(0, 1)] if paired else [(0, -1), (1, -1)])
    psi0 = _state(n, rng)
    ref = oracle.run(psi0.astype(np.complex128), OG.gate_list(specs))
    out, rep = _apply(sv, n, psi0, c, sv.SV_POLICY_TWO_GATE_PASSES)
    assert rep["paired_passes"] == (1 if paired else 0)
    assert rep["passes"] == (1 if paired else 2)
    e2 = _check(out, ref)
    one, rep1 = _apply(sv, n, psi0, c, 0)
    assert rep1["paired_passes"] == 0 and rep1["passes"] == 2
    e1 = _check(one, ref)
    # the pair computes each gate exactly as the single-gate kernels do
    assert e2 <= 4 * max(e1, 1e-7)


@pytest.mark.parametrize("family", ["grid20", "qft_brickwork18", "random17"])
def test_paired_circuits_against_oracle(gpu, family):
    """Fused circuits (k = 5) with two-gate passes against the oracle and against the same
    schedule one gate per pass; pairing applies every gate once and cuts passes."""
    sv = gpu
    import torch
    rng = np.random.default_rng(321)
    x = 0
    if family == "grid20":
        n, specs = 20, W.grid_random(20, 12)
    elif family == "qft_brickwork18":
        n = 18
        x, specs = W.qft_brickwork(n, 8)
    else:
        n, specs = 17, W.random_unitary_gates(17, 120, 5, rng)
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, 5)
    nf, _ = sv.sv_circuit_size(c)
    ref = oracle.simulate(n, specs, x=x)
    outs = {}
    P = sv.SV_POLICY_TWO_GATE_PASSES
    for policy in (P, 0):
        s = sv.sv_alloc(n, 0, stream=torch.cuda.current_stream())
        sv.sv_set_policy(s, policy)
        sv.sv_set_basis(s, x)
        rep = sv.sv_apply_circuit(s, c)
        outs[policy] = sv.sv_get_state(s).astype(np.complex128)
        s.free()
        assert rep["passes"] + rep["paired_passes"] == nf
        if policy == P:
            assert rep["paired_passes"] >= 1
            assert rep["passes"] == len(sv.sv_plan_passes(c))
        _check(outs[policy], ref)
    assert float(np.max(np.abs(outs[P] - outs[0]))) <= 2e-5


def test_paired_norm_over_many_passes(gpu):
    """Pairs of width-5 unitaries keep the norm of a 17-qubit state within 1e-6 over 300
    gates (the exact-slice products stay unbiased inside a pair too)."""
    sv = gpu
    import torch
    rng = np.random.default_rng(88)
    n = 17
    specs = W.random_unitary_gates(n, 300, 5, rng, exact_k=True)
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, 0)
    s = sv.sv_alloc(n, 0, stream=torch.cuda.current_stream())
    sv.sv_set_policy(s, sv.SV_POLICY_TWO_GATE_PASSES)
    sv.sv_set_basis(s, 777)
    rep = sv.sv_apply_circuit(s, c)
    assert rep["paired_passes"] >= 30
    assert abs(sv.sv_norm(s) - 1.0) < 1e-6
    ref = oracle.simulate(n, specs, x=777)
    _check(sv.sv_get_state(s).astype(np.complex128), ref)
    s.free()
