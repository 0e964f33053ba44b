"""Tensor-core path for complex128 gates of up to four qubits (six exact FP16 digits per
operand, exact level sums, integer recombination), against the oracle and against the
FP64 CUDA-core kernels on the same inputs."""
import numpy as np
import pytest

import oracle
from oracle import gates as OG
import workloads as W

pytestmark = pytest.mark.gpu


def _state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def _run(sv, n, psi0, gl, policy):
    import torch
    s = sv.sv_alloc(n, 1, stream=torch.cuda.current_stream())
    sv.sv_set_policy(s, policy)
    sv.sv_set_state(s, psi0.astype(np.complex128))
    for tg, u in gl:
        sv.sv_apply_gate(s, tg, u)
    out = sv.sv_get_state(s)
    s.free()
    return out


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_tc64_matches_oracle_and_fp64_cores(gpu, k):
    sv = gpu
    rng = np.random.default_rng(600 + k)
    for n in (11, 13, 17):
        for tg in (tuple(range(k)), tuple(range(n - k, n)), None,
                   tuple(rng.choice(n, k, replace=False)), (0,) + tuple(range(n - k + 1, n)),
                   tuple(range(5, 5 + k))):
            specs = W.random_unitary_gates(n, 3, k, rng, exact_k=True, targets=tg)
            psi0 = _state(n, rng)
            ref = oracle.run(psi0.copy(), OG.gate_list(specs))
            gl = sv.gates_from_specs(specs)
            tc = _run(sv, n, psi0, gl, 0)
            cc = _run(sv, n, psi0, gl, sv.SV_POLICY_NO_TENSOR_CORES)
            err_tc = np.max(np.abs(tc - ref))
            err_cc = np.max(np.abs(cc - ref))
            assert err_tc <= 1e-14 and err_cc <= 1e-14, (n, tg, err_tc, err_cc)
            # FP64-class accuracy: within a small factor of the FP64 FMA kernels
            assert err_tc <= 64 * max(err_cc, 1e-17), (n, tg, err_tc, err_cc)


def test_tc64_mixed_magnitudes_and_non_unitary(gpu):
    """Amplitudes spread over many binades in one group, and a non-unitary matrix with
    large entries: the error stays below 2^-46 of (largest amplitude x largest entry)."""
    sv = gpu
    rng = np.random.default_rng(611)
    n = 12
    psi0 = _state(n, rng) * np.exp2(rng.integers(-40, 0, 1 << n))
    psi0[rng.integers(0, 1 << n, 300)] = 0.0
    m = (rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))) * 250.0
    for tg in ((0, 1, 2, 3), (2, 5, 9, 11), (8, 9, 10, 11)):
        gl = [(tg, m)]
        ref = oracle.run(psi0.copy(), [(tuple(tg), m)])
        tc = _run(sv, n, psi0, gl, 0)
        bound = 2.0 ** -46 * np.max(np.abs(psi0)) * 2 * np.max(np.abs(m)) * 2 + 1e-300
        assert np.max(np.abs(tc - ref)) <= bound + 4 * np.spacing(np.max(np.abs(ref)))


def test_tc64_norm_is_preserved_over_many_passes(gpu):
    """400 random width-4 unitaries in complex128 keep the norm to 1e-12 and the state
    within 1e-12 of the oracle."""
    sv = gpu
    import torch
    rng = np.random.default_rng(612)
    n = 16
    specs = W.random_unitary_gates(n, 400, 4, rng, exact_k=True)
    s = sv.sv_alloc(n, 1, stream=torch.cuda.current_stream())
    sv.sv_set_basis(s, 4321)
    for tg, u in sv.gates_from_specs(specs):
        sv.sv_apply_gate(s, tg, u)
    assert abs(sv.sv_norm(s) - 1.0) < 1e-12
    ref = oracle.simulate(n, specs, x=4321)
    psi = sv.sv_get_state(s)
    assert np.max(np.abs(psi - ref)) < 1e-12
    s.free()
