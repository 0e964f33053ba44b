"""Noisy simulation with density matrices on the GPU (sv_fuse_density + sv_apply_circuit +
sv_density_probs) against the density-matrix oracle, the paper's Table 8, and the
invariants of a density matrix at 15 qubits (a 30-qubit vector)."""
import os

import numpy as np
import pytest

import oracle
from oracle import density as D
from oracle import gates as OG
import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _torch():
    import torch
    return torch


def _run(sv, n, specs, p, k, dtype):
    torch = _torch()
    c = sv.sv_fuse_density(sv.gates_from_specs(specs), n, p, k)
    s = sv.sv_alloc(2 * n, dtype, stream=torch.cuda.current_stream())
    sv.sv_set_basis(s, 0)
    sv.sv_apply_circuit(s, c)
    return s


@pytest.mark.parametrize("dtype", [0, 1])
def test_density_matrix_matches_oracle(gpu, dtype):
    sv = gpu
    rng = np.random.default_rng(1301 + dtype)
    tol = 1e-5 if dtype == 0 else 1e-12
    for n, p, k, ng in ((2, 0.01, 4, 6), (4, 0.03, 4, 14), (6, 0.01, 5, 20), (7, 0.1, 3, 16)):
        specs = W.random_unitary_gates(n, ng, 2, rng)
        s = _run(sv, n, specs, p, k, dtype)
        v = sv.sv_get_state(s).astype(np.complex128)
        rho = D.run(n, OG.gate_list(specs), p)
        assert np.max(np.abs(v - D.vec(rho))) < tol, (n, p, k)
        pr = sv.sv_density_probs(s)
        assert np.max(np.abs(pr - D.probs(rho))) < tol
        s.free()


@pytest.mark.parametrize("dtype", [0, 1])
def test_table8_on_the_gpu(gpu, dtype):
    sv = gpu
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "noise_table8.txt"))
            if l.strip() and not l.startswith("#")]
    for name, n, f_msle, _, t_msle, _ in rows:
        n = int(n)
        specs = W.bell() if n == 2 else W.ghz(n)
        ideal = D.probs(D.run(n, OG.gate_list(specs), 0.0))
        s = _run(sv, n, specs, 0.01, 4, dtype)
        pr = sv.sv_density_probs(s).astype(np.float64)
        s.free()
        f, t = D.classical_fidelity(pr, ideal), D.tvd(pr, ideal)
        fo, to = D.noisy_vs_ideal(n, OG.gate_list(specs), 0.01)
        assert abs(f - fo) < (1e-6 if dtype == 0 else 1e-12) and abs(t - to) < (1e-6 if dtype == 0 else 1e-12)
        assert abs(f - float(f_msle)) <= 0.006 and abs(t - float(t_msle)) <= 0.006


def test_density_15q_invariants(gpu):
    """GHZ-15 with p = 0.01 on a 2^30-entry density vector (complex128, 16 GiB): unit trace,
    nonnegative populations, the two GHZ outcomes equally likely and most likely, and the
    population lost to the other outcomes close to its first-order value 2(n-1)(2p/3)."""
    sv = gpu
    torch = _torch()
    n, p = 15, 0.01
    s = _run(sv, n, W.ghz(n), p, 4, 1)
    pr = sv.sv_density_probs(s)
    s.free()
    torch.cuda.empty_cache()
    assert abs(pr.sum() - 1.0) < 1e-12
    assert pr.min() > -1e-15
    top = np.argsort(pr)[::-1][:2]
    assert set(int(t) for t in top) == {0, (1 << n) - 1}
    assert abs(pr[0] - pr[-1]) < 1e-12
    lost = 1.0 - pr[0] - pr[-1]
    first_order = 2 * (n - 1) * (2 * p / 3)
    assert 0.85 * first_order < lost < first_order
