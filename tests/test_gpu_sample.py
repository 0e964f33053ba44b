"""Measurement sampling on the GPU (sv_sample) against the oracle's sampling: the same
indices, bit for bit, on seeded states of both precisions (single block, several blocks,
several chunks), plus distribution checks at 30 qubits."""
import numpy as np
import pytest

import oracle
from oracle import gates as OG
from oracle import sampling as OS
import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _state(n, rng, zeros=0.0):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    if zeros:
        v[rng.random(1 << n) < zeros] = 0.0
    v[0] = 1.0 if not np.any(v) else v[0]
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("dtype", [0, 1])
def test_samples_match_oracle_bit_for_bit(gpu, dtype):
    sv = gpu
    rng = np.random.default_rng(1201 + dtype)
    for n, zeros in ((1, 0.0), (5, 0.3), (6, 0.0), (13, 0.5), (19, 0.2), (20, 0.0)):
        psi = _state(n, rng, zeros).astype(np.complex64 if dtype == 0 else np.complex128)
        s = sv.sv_alloc(n, dtype, stream=_torch().cuda.current_stream())
        sv.sv_set_state(s, psi)
        seed = int(rng.integers(0, 2 ** 63))
        nshots = 3000
        got = sv.sv_sample(s, seed, nshots)
        want = OS.sample(oracle.probs_in_precision(psi), seed, nshots)
        assert np.array_equal(got, want), (n, zeros, int(np.sum(got != want)))
        s.free()


def test_sample_edge_cases(gpu):
    sv = gpu
    torch = _torch()
    s = sv.sv_alloc(12, 0, stream=torch.cuda.current_stream())
    sv.sv_set_basis(s, 2077)
    assert np.all(sv.sv_sample(s, 5, 1000) == 2077)          # a basis state
    assert sv.sv_sample(s, 5, 0).size == 0
    sv.sv_set_state(s, np.zeros(1 << 12, dtype=np.complex64))
    with pytest.raises(sv.SvError):
        sv.sv_sample(s, 5, 10)                                # zero norm
    s.free()
    # device output equals host output
    s = sv.sv_alloc(16, 1, stream=torch.cuda.current_stream())
    sv.sv_set_state(s, _state(16, np.random.default_rng(3)))
    dev = torch.empty(5000, dtype=torch.int64, device="cuda")
    sv.sv_sample(s, 11, 5000, dev)
    assert np.array_equal(dev.cpu().numpy().astype(np.uint64), sv.sv_sample(s, 11, 5000))
    s.free()


def test_sample_30q_distribution(gpu):
    """2^30 outcomes: a uniform superposition over qubits 0..9 times |x> on the rest; and
    H on one qubit of a basis state (two outcomes, 50/50)."""
    scipy_stats = pytest.importorskip("scipy.stats")
    sv = gpu
    torch = _torch()
    n = 30
    x = (0b1011 << 26) | (1 << 20)
    s = sv.sv_alloc(n, 0, stream=torch.cuda.current_stream())
    sv.sv_set_basis(s, x)
    for q in range(10):
        sv.sv_apply_gate(s, (q,), OG.H)
    shots = sv.sv_sample(s, 2026, 200000)
    assert np.all((shots >> 10) == (x >> 10))
    counts = np.bincount((shots & 1023).astype(np.int64), minlength=1024)
    assert scipy_stats.chisquare(counts).pvalue > 1e-4
    s.free()
    torch.cuda.empty_cache()
