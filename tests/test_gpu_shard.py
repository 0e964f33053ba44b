"""Global-qubit sharding on one GPU: the pack/unpack kernels against their index
definition, and a state sharded over 2, 4 and 8 ranks run as threads of one process
(ThreadComm: host barriers, device copies between the ranks' staging buffers; no kernel
waits on another rank) against the oracle and the unsharded path."""
import threading

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


def _half(n, bit, value):
    e = np.arange(1 << (n - 1), dtype=np.int64)
    return ((e >> bit) << (bit + 1)) | (value << bit) | (e & ((1 << bit) - 1))


@pytest.mark.parametrize("dtype", [0, 1])
def test_pack_unpack_match_the_index_definition(gpu, dtype):
    sv = gpu
    import torch
    n = 13
    rng = np.random.default_rng(21 + dtype)
    npdt = np.complex64 if dtype == 0 else np.complex128
    psi = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(npdt)
    s = sv.sv_alloc(n, dtype, stream=torch.cuda.current_stream())
    esz = 8 if dtype == 0 else 16
    for bit in (0, 1, 3, 12):
        for value in (0, 1):
            for off, cnt in ((0, 1 << (n - 1)), (3, 101), (64, 500), ((1 << (n - 1)) - 7, 7)):
                sv.sv_set_state(s, psi)
                idx = _half(n, bit, value)[off:off + cnt]
                dst = torch.zeros(esz * cnt, dtype=torch.uint8, device="cuda")
                sv.sv_shard_pack(s, bit, value, off, cnt, dst)
                torch.cuda.synchronize()
                got = dst.cpu().numpy().view(npdt)
                assert np.array_equal(got, psi[idx]), (bit, value, off, cnt)
                new = (rng.normal(size=cnt) + 1j * rng.normal(size=cnt)).astype(npdt)
                src = torch.from_numpy(new.view(np.uint8).copy()).cuda()
                sv.sv_shard_unpack(s, bit, value, off, cnt, src)
                want = psi.copy()
                want[idx] = new
                assert np.array_equal(sv.sv_get_state(s), want), (bit, value, off, cnt)
    with pytest.raises(sv.SvError):
        sv.sv_shard_pack(s, n, 0, 0, 1, dst)                      # bit >= n
    with pytest.raises(sv.SvError):
        sv.sv_shard_pack(s, 0, 0, 1 << (n - 1), 1, dst)           # beyond the half
    s.free()


def _run_sharded(sv, world, n, dtype, k, chunk, x, specs):
    import torch
    from paper_2604_03816_gb300.shard import GpuShard, ShardedState, ThreadComm, ThreadHub
    hub = ThreadHub(world)
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, k)
    g = world.bit_length() - 1
    out = [None] * world
    errors = []
    xs, zs, cs = W.zz_chain(n)
    top, top2 = 1 << (n - 1), 1 << (n - 2)
    terms = (list(xs) + [0, 0b11, top, top | top2 | 1], list(zs) + [top | 1, 0b10, top2, top | 0b110],
             list(cs) + [0.5, -0.25, 0.8, -0.6])   # Z and X/Y on the top qubits too

    def worker(r):
        try:
            torch.cuda.set_device(0)
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                local = GpuShard(n - g, dtype, stream=stream, chunk=chunk)
                st = ShardedState(n, dtype, ThreadComm(hub, r), local)
                st.set_basis(x)
                rep = st.apply_circuit(c)
                out[r] = {"rep": rep, "state": st.get_state(), "norm": st.norm(),
                          "expect": st.expect(*terms), "topk": st.topk(16),
                          "bytes": st.exchanged_bytes}
                local.free()
        except BaseException as e:          # noqa: BLE001 -- reported below
            errors.append(e)
            hub.barrier.abort()

    threads = [threading.Thread(target=worker, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(600)
    assert not errors, errors
    return out, terms


@pytest.mark.parametrize("world,n,dtype,k,chunk", [(2, 20, 0, 5, 1 << 26), (4, 20, 0, 5, 1 << 12),
                                                   (4, 18, 1, 4, 1 << 10), (8, 17, 1, 5, 1 << 26),
                                                   (2, 22, 1, 5, 1 << 14)])
def test_sharded_state_on_thread_ranks(gpu, world, n, dtype, k, chunk):
    sv = gpu
    import torch
    specs = W.grid_random(n, 8)
    x = 12345 % (1 << n)
    ref = oracle.simulate(n, specs, x=x)
    out, terms = _run_sharded(sv, world, n, dtype, k, chunk, x, specs)
    # the same circuit unsharded on the GPU
    s = sv.sv_alloc(n, dtype, stream=torch.cuda.current_stream())
    sv.sv_set_basis(s, x)
    sv.sv_apply_circuit(s, sv.sv_fuse(sv.gates_from_specs(specs), n, k))
    whole = sv.sv_get_state(s).astype(np.complex128)
    s.free()
    want_e = oracle.expect(ref, *terms)
    for r in out:
        psi = r["state"].astype(np.complex128)
        assert np.max(np.abs(psi - ref)) <= TOL[dtype]
        assert np.max(np.abs(psi - whole)) <= TOL[dtype]
        if dtype == 0:
            f = abs(np.vdot(ref, psi)) ** 2 / np.vdot(psi, psi).real
            assert 1 - f <= 1e-6
        assert abs(r["norm"] - 1.0) <= 10 * TOL[dtype]
        assert abs(r["expect"] - want_e) <= 10 * TOL[dtype] * len(terms[0])
        assert oracle.topk_valid(r["topk"][0], oracle.probs(ref), 16, 10 * TOL[dtype])
        assert r["rep"]["exchanges"] > 0 and r["bytes"] > 0
