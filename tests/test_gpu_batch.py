"""Batched execution: many states of one width driven by circuits that share a fused
structure (a parameter sweep), per-state matrices, L2 chunks and CUDA-graph replay."""
import numpy as np
import pytest

import oracle
from oracle import gates as OG
import workloads as W

pytestmark = pytest.mark.gpu


def _family(n, count, seed, layers=3):
    rng = np.random.default_rng(seed)
    return [W.hea(n, layers, rng=rng) for _ in range(count)]


@pytest.mark.parametrize("dtype,k", [(0, 2), (0, 3), (0, 4), (1, 3)])
def test_batch_matches_oracle(gpu, dtype, k):
    sv = gpu
    import torch
    n, count = 9, 12
    fam = _family(n, count, 10 + k)
    circs = [sv.sv_fuse(sv.gates_from_specs(f), n, k) for f in fam]
    b = sv.sv_batch_alloc(n, dtype, count, stream=torch.cuda.current_stream())
    sv.sv_batch_set_basis(b, 5)
    rep = sv.sv_batch_apply(b, circs, chunk_states=5)     # 3 chunks, ragged last one
    assert rep["chunk_states"] == 5 and rep["launches"] == 3 * len(circs[0])
    tol = 1e-5 if dtype == 0 else 1e-12
    xs, zs, cs = W.zz_chain(n)
    zz = sv.sv_batch_expect(b, xs, zs, cs)
    for i, f in enumerate(fam):
        ref = oracle.simulate(n, f, x=5)
        psi = sv.sv_batch_get_state(b, i).astype(np.complex128)
        assert np.max(np.abs(psi - ref)) < tol, i
        assert abs(zz[i] - oracle.expect(ref, xs, zs, cs)) < 10 * tol
    b.free()


def test_batch_graph_replay_with_new_parameters(gpu):
    sv = gpu
    import torch
    n, count = 10, 8
    b = sv.sv_batch_alloc(n, 0, count, stream=torch.cuda.current_stream())
    for rnd in range(3):
        fam = _family(n, count, 100 + rnd)
        circs = [sv.sv_fuse(sv.gates_from_specs(f), n, 3) for f in fam]
        sv.sv_batch_set_basis(b, 0)
        rep = sv.sv_batch_apply(b, circs)
        assert rep["graph_reused"] == (1 if rnd > 0 else 0)
        for i in (0, count - 1):
            ref = oracle.simulate(n, fam[i])
            assert np.max(np.abs(sv.sv_batch_get_state(b, i) - ref)) < 1e-5
    # direct launches give the same states as the graph
    fam = _family(n, count, 7)
    circs = [sv.sv_fuse(sv.gates_from_specs(f), n, 3) for f in fam]
    sv.sv_batch_set_basis(b, 0)
    sv.sv_batch_apply(b, circs, no_graph=True)
    direct = sv.sv_batch_get_state(b, 3)
    sv.sv_batch_set_basis(b, 0)
    sv.sv_batch_apply(b, circs)
    assert np.array_equal(direct, sv.sv_batch_get_state(b, 3))
    b.free()


def test_batch_rejects_mismatched_structure(gpu):
    sv = gpu
    n = 8
    b = sv.sv_batch_alloc(n, 0, 2)
    c1 = sv.sv_fuse(sv.gates_from_specs(W.hea(n, 2, seed=1)), n, 2)
    c2 = sv.sv_fuse(sv.gates_from_specs(W.brickwork(n, 2)), n, 2)
    with pytest.raises(sv.SvError) as e:
        sv.sv_batch_apply(b, [c1, c2])
    assert e.value.status == 1
    b.free()


def test_batch_tune_picks_and_caches(gpu):
    sv = gpu
    import torch
    n, count = 14, 16
    b = sv.sv_batch_alloc(n, 0, count, stream=torch.cuda.current_stream())
    gl = sv.gates_from_specs(W.hea(n, 6, seed=3))
    r = sv.sv_batch_tune(b, gl, 1, 4)
    assert 1 <= r["best_k"] <= 4 and r["cached"] == 0
    assert all(v > 0 for v in r["ms"].values())
    assert r["best_ms"] == min(r["ms"].values())
    r2 = sv.sv_batch_tune(b, gl, 1, 4)
    assert r2["cached"] == 1 and r2["best_k"] == r["best_k"]
    assert r2["tile_bits"] == r["tile_bits"] and r["tile_bits"] in (0, 10, 11, 12, 13)
    # the states were reset to |0...0>
    assert sv.sv_batch_get_state(b, 0)[0] == 1
    b.free()


@pytest.mark.parametrize("dtype", [0, 1])
def test_batch_tile_sizes_give_identical_states(gpu, dtype):
    """The CUDA-core batched passes at every tile size the tuner may choose (2^10..2^13
    amplitudes per CTA): each group's arithmetic is the same, so the states agree bit for
    bit across tile sizes and with the oracle."""
    sv = gpu
    import torch
    n, count = 15, 6
    fam = [W.hea(n, 3, seed=40 + i) for i in range(count)]
    circs = [sv.sv_fuse(sv.gates_from_specs(f), n, 3) for f in fam]
    b = sv.sv_batch_alloc(n, dtype, count, stream=torch.cuda.current_stream())
    states = {}
    for tb in (0, 10, 11, 12, 13):
        sv.sv_batch_set_basis(b, 0)
        rep = sv.sv_batch_apply(b, circs, tile_bits=tb, no_tensor_cores=True)
        assert rep["tile_bits"] == (tb or (12 if dtype == 0 else 11))
        states[tb] = [sv.sv_batch_get_state(b, i) for i in range(count)]
    for tb in (10, 11, 12, 13):
        assert all(np.array_equal(a, z) for a, z in zip(states[0], states[tb])), tb
    tol = 1e-5 if dtype == 0 else 1e-12
    for i, f in enumerate(fam):
        assert np.max(np.abs(states[13][i].astype(np.complex128) - oracle.simulate(n, f))) < tol
    with pytest.raises(sv.SvError):
        sv.sv_batch_apply(b, circs, tile_bits=9)
    b.free()


@pytest.mark.parametrize("n", [12, 14])
@pytest.mark.parametrize("k", [4, 5])
def test_batch_tensor_cores_match_oracle(gpu, n, k):
    """complex64 width-4/5 gates of a batch run on the tensor cores (width 4 widened by an
    identity qubit in the kernel, B built per state on the device): each state against
    the oracle, and against the CUDA-core batched path.  Small states and a chunk size
    that is not a multiple of anything make CTAs' tile ranges cross state boundaries (a
    12-qubit state is one tile)."""
    import torch
    sv = gpu
    count = 23
    specs = [W.hea(n, 3, seed=300 + i) for i in range(count)]
    circs = [sv.sv_fuse(sv.gates_from_specs(sp), n, k) for sp in specs]
    assert any(len(sv.sv_circuit_gate(circs[0], g)[0]) == k for g in range(len(circs[0])))
    outs = {}
    for no_tc in (False, True):
        b = sv.sv_batch_alloc(n, 0, count, stream=torch.cuda.current_stream())
        sv.sv_batch_apply(b, circs, chunk_states=7, no_tensor_cores=no_tc)
        sv.sv_batch_sync(b)
        outs[no_tc] = [sv.sv_batch_get_state(b, i).astype(np.complex128) for i in range(count)]
        b.free()
    for i in range(count):
        ref = oracle.simulate(n, specs[i])
        for no_tc in (False, True):
            err = float(np.max(np.abs(outs[no_tc][i] - ref)))
            assert err <= 1e-5, (i, no_tc, err)
        assert float(np.max(np.abs(outs[False][i] - outs[True][i]))) <= 2e-6


@pytest.mark.parametrize("k", [4, 5])
def test_batch_tensor_cores_rebuild_b_across_states(gpu, k):
    """Many small states in one chunk: each CTA's tile range crosses several states, so
    the producer rebuilds B mid-launch and reuses both B sets.  Every state against the
    CUDA-core batched path; a sample against the oracle."""
    import torch
    sv = gpu
    n, count = 13, 400            # 2 tiles per state, 800 tiles over 152 CTAs
    rng = np.random.default_rng(77 + k)
    specs = [W.hea(n, 2, rng=rng) for _ in range(count)]
    circs = [sv.sv_fuse(sv.gates_from_specs(sp), n, k) for sp in specs]
    outs = {}
    for no_tc in (False, True):
        b = sv.sv_batch_alloc(n, 0, count, stream=torch.cuda.current_stream())
        sv.sv_batch_apply(b, circs, l2_bytes=1 << 40, no_tensor_cores=no_tc)
        sv.sv_batch_sync(b)
        outs[no_tc] = np.stack([sv.sv_batch_get_state(b, i) for i in range(count)]).astype(np.complex128)
        b.free()
    diff = np.max(np.abs(outs[False] - outs[True]), axis=1)
    assert float(diff.max()) <= 2e-6, int(diff.argmax())
    for i in list(range(0, count, 37)) + [count - 1]:
        ref = oracle.simulate(n, specs[i])
        assert float(np.max(np.abs(outs[False][i] - ref))) <= 1e-5, i
