"""Tensor-core (tcgen05, exact FP16 slices) path for fused k = 4, 5 complex64 gates, against the
oracle and against the CUDA-core kernels on the same inputs."""
import numpy as np
import pytest

import oracle
from oracle import gates as OG
import workloads as W

pytestmark = pytest.mark.gpu


def _state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex64)


def _run(sv, n, psi0, gl, policy):
    import torch
    s = sv.sv_alloc(n, 0, stream=torch.cuda.current_stream())
    sv.sv_set_policy(s, policy)
    sv.sv_set_state(s, psi0)
    for tg, u in gl:
        sv.sv_apply_gate(s, tg, u)
    out = sv.sv_get_state(s).astype(np.complex128)
    s.free()
    return out


@pytest.mark.parametrize("k", [4, 5])
def test_tc_matches_oracle_and_cuda_cores(gpu, k):
    sv = gpu
    rng = np.random.default_rng(500 + k)
    for n in (k + 7, 14, 17):
        for tg in (tuple(range(k)), tuple(range(n - k, n)), None,
                   tuple(rng.choice(n, k, replace=False)), (0,) + tuple(range(n - k + 1, n))):
            specs = W.random_unitary_gates(n, 3, k, rng, exact_k=True, targets=tg)
            psi0 = _state(n, rng)
            ref = oracle.run(psi0.astype(np.complex128), OG.gate_list(specs))
            gl = sv.gates_from_specs(specs)
            tc = _run(sv, n, psi0, gl, 0)
            cc = _run(sv, n, psi0, gl, sv.SV_POLICY_NO_TENSOR_CORES)
            err_tc = np.max(np.abs(tc - ref))
            err_cc = np.max(np.abs(cc - ref))
            assert err_tc <= 1e-5 and err_cc <= 1e-5, (n, tg, err_tc, err_cc)
            f = abs(np.vdot(ref, tc)) ** 2 / np.vdot(tc, tc).real
            assert 1 - f <= 1e-6
            # the exact-slice products keep FP32-level accuracy, like the FP32 FMA path
            assert err_tc <= 8 * max(err_cc, 1e-7)


def test_tc_norm_is_preserved_over_many_passes(gpu):
    """The exact-slice products make tensor-core errors unbiased: 400 random width-5
    unitaries keep the norm within 1e-6 (a truncating split loses ~1e-6 per pass)."""
    sv = gpu
    import torch
    rng = np.random.default_rng(77)
    n = 16
    specs = W.random_unitary_gates(n, 400, 5, rng, exact_k=True)
    s = sv.sv_alloc(n, 0, stream=torch.cuda.current_stream())
    sv.sv_set_basis(s, 12345)
    for tg, u in sv.gates_from_specs(specs):
        sv.sv_apply_gate(s, tg, u)
    assert abs(sv.sv_norm(s) - 1.0) < 1e-6
    ref = oracle.simulate(n, specs, x=12345)
    psi = sv.sv_get_state(s).astype(np.complex128)
    assert np.max(np.abs(psi - ref)) < 1e-5
    assert 1 - abs(np.vdot(ref, psi)) ** 2 < 1e-6
    s.free()


def test_tc_variants_edge_layouts(gpu):
    """The width-5 kernel variants at their boundaries: one two-subtile tile (n = 13), the
    one-subtile kernel at n = 12, width-4 gates widened to width 5, and the XOR member order
    with one to four targets in the bank bits, against the oracle."""
    sv = gpu
    rng = np.random.default_rng(5150)
    cases = [(13, (8, 9, 10, 11, 12)), (13, (0, 1, 2, 3, 4)), (13, (5, 6, 7, 8, 9)),
             (12, (7, 8, 9, 10, 11)), (14, (0, 6, 9, 12, 13)), (14, (0, 1, 7, 10, 13)),
             (14, (0, 1, 2, 10, 13)), (15, (1, 2, 3, 4, 14)),
             (13, (9, 10, 11, 12)), (14, (0, 1, 2, 3)), (12, (4, 5, 6, 7))]
    for n, tg in cases:
        specs = W.random_unitary_gates(n, 2, len(tg), rng, exact_k=True, targets=tg)
        psi0 = _state(n, rng)
        ref = oracle.run(psi0.astype(np.complex128), OG.gate_list(specs))
        got = _run(sv, n, psi0, sv.gates_from_specs(specs), 0)
        assert np.max(np.abs(got - ref)) <= 1e-5, (n, tg)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_narrow_gates_route_to_the_tensor_cores_from_13_qubits(gpu, k):
    """complex64 gates narrower than 4 qubits run on the width-5 tensor-core kernel (widened
    by identity qubits) on states of at least 13 qubits, and on the CUDA cores below; both
    against the oracle, with targets among the shared-memory bank bits 0-3 included."""
    sv = gpu
    import torch
    rng = np.random.default_rng(9000 + k)
    for n in (12, 13, 16):
        for tg in (tuple(range(k)), tuple(range(n - k, n)), (0,) + tuple(range(n - k + 1, n)), None):
            specs = W.random_unitary_gates(n, 6, k, rng, exact_k=True, targets=tg)
            psi0 = _state(n, rng)
            ref = oracle.run(psi0.astype(np.complex128), OG.gate_list(specs))
            c = sv.sv_fuse(sv.gates_from_specs(specs), n, k)
            s = sv.sv_alloc(n, 0, stream=torch.cuda.current_stream())
            sv.sv_set_state(s, psi0)
            rep = sv.sv_apply_circuit(s, c)
            got = sv.sv_get_state(s).astype(np.complex128)
            s.free()
            assert rep["passes"] >= 1
            assert rep["tc_passes"] == (rep["passes"] if n >= 13 else 0), (n, tg, rep)
            assert np.max(np.abs(got - ref)) <= 1e-5, (n, tg)
            f = abs(np.vdot(ref, got)) ** 2 / np.vdot(got, got).real
            assert 1 - f <= 1e-6
