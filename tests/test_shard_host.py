"""Global-qubit sharding on the CPU: the planner's steps and the executor's exchange and
reductions, against the oracle.

* The plan (sv_shard_plan_*, host code of the library) is replayed on a full state vector:
  a segment's gates act on bit positions, an exchange of local position p with global
  bit j is the swap of index bits p and L + j; the final vector must be the oracle's
  state of the unsharded circuit, and the plan must end in the identity layout.
* The executor (paper_2604_03816_gb300.shard.ShardedState) runs on 2 and 4 gloo ranks
  (processes) with TorchComm; each rank's local part is the oracle applied to its shard
  (test infrastructure standing in for a GPU).  The gathered state, norm, Pauli
  expectations (ZZ chain, Z on the top qubits, X/Y on local and on top qubits) and top-k
  must equal the oracle's on the whole state.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import gates as OG


def _replay_plan(sv, plan, n, g, psi):
    L = n - g
    for kind, p, j, seg in plan.steps():
        if kind == sv.SV_SHARD_APPLY:
            for i in range(len(seg)):
                tg, u = sv.sv_circuit_gate(seg, i)
                assert max(tg) < L                       # only local positions
                oracle.apply_gate(psi, tg, u)
        else:
            assert p < L and j < g
            idx = np.arange(psi.size, dtype=np.int64)
            a, b = (idx >> p) & 1, (idx >> (L + j)) & 1
            swapped = idx ^ ((a ^ b) << p) ^ ((a ^ b) << (L + j))
            psi[swapped] = psi.copy()
    return psi


@pytest.mark.parametrize("n,g,k,dtype", [(10, 1, 3, 0), (10, 2, 4, 0), (11, 3, 5, 0),
                                         (12, 2, 5, 1), (9, 4, 3, 1)])
def test_plan_replayed_on_the_full_state(svlib, n, g, k, dtype):
    sv = svlib
    rng = np.random.default_rng(100 * n + g)
    specs = W.random_unitary_gates(n, 40, min(k, 3), rng)
    x = int(rng.integers(0, 1 << n))
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, k)
    plan = sv.sv_shard_plan_create(c, g, dtype)
    nsteps, nex, nswap = plan.info()
    assert nex > 0                                  # gates on the top qubits need exchanges
    psi = _replay_plan(sv, plan, n, g, oracle.basis(n, x))
    ref = oracle.simulate(n, specs, x=x)
    assert np.max(np.abs(psi - ref)) < 1e-12


def test_plan_grid_circuit_and_limits(svlib):
    sv = svlib
    n = 12
    specs = W.grid_random(n, 6)
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, 5)
    for g in (0, 1, 3, 7):
        plan = sv.sv_shard_plan_create(c, g, 0)
        _, nex, _ = plan.info()
        assert (nex == 0) == (g == 0)
        psi = _replay_plan(sv, plan, n, g, oracle.basis(n, 0))
        assert np.max(np.abs(psi - oracle.simulate(n, specs))) < 1e-12
    with pytest.raises(sv.SvError):
        sv.sv_shard_plan_create(c, 8, 0)               # 4 local qubits < a width-5 gate
    with pytest.raises(sv.SvError):
        sv.sv_shard_plan_create(c, n, 0)


# ------------------------------------------------------------------ executor on gloo ranks

class OracleShard:
    """A rank's 2^L amplitudes on the CPU, gates applied by the oracle (test only)."""

    def __init__(self, sv, L, chunk):
        self.sv, self.L, self.chunk = sv, L, chunk
        self.psi = np.zeros(1 << L, dtype=np.complex128)

    def _half(self, bit, value):
        e = np.arange(1 << (self.L - 1), dtype=np.int64)
        return ((e >> bit) << (bit + 1)) | (value << bit) | (e & ((1 << bit) - 1))

    def set_basis(self, x):
        self.psi[:] = 0
        self.psi[x] = 1

    def set_zero(self):
        self.psi[:] = 0

    def apply(self, seg):
        for i in range(len(seg)):
            tg, u = self.sv.sv_circuit_gate(seg, i)
            oracle.apply_gate(self.psi, tg, u)
        return {"passes": len(seg)}

    def outgoing(self, bit, value, off, cnt):
        import torch
        idx = self._half(bit, value)[off:off + cnt]
        return torch.from_numpy(self.psi[idx].view(np.float64).copy())

    def incoming(self, cnt):
        import torch
        return torch.empty(2 * cnt, dtype=torch.float64)

    def store(self, bit, value, off, cnt, src):
        idx = self._half(bit, value)[off:off + cnt]
        self.psi[idx] = src.numpy().view(np.complex128)

    def norm(self):
        return oracle.norm(self.psi)

    def expect(self, xs, zs, cs):
        return oracle.expect(self.psi, xs, zs, cs)

    def topk(self, k):
        return oracle.topk(oracle.probs(self.psi), k)

    def get_state(self):
        return self.psi.copy()


def _rank_main(rank, world, port, n, k, out_dir):
    import torch.distributed as dist
    from paper_2604_03816_gb300 import sv
    from paper_2604_03816_gb300.shard import ShardedState, TorchComm
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        specs = W.grid_random(n, 6) + W.random_unitary_gates(n, 12, 2, np.random.default_rng(7))
        c = sv.sv_fuse(sv.gates_from_specs(specs), n, k)
        comm = TorchComm()
        L = n - (world.bit_length() - 1)
        st = ShardedState(n, 1, comm, OracleShard(sv, L, chunk=16))
        st.set_basis(37)
        rep = st.apply_circuit(c)
        terms = _terms(n)
        res = {"state": st.get_state(), "norm": st.norm(), "expect": st.expect(*terms),
               "topk": st.topk(10), "rep": rep, "bytes": st.exchanged_bytes}
        # the layout is back to the identity after the swaps of the expectation
        res["state_after"] = st.get_state()
        with pytest.raises(ValueError):
            st.expect([1 << n], [0], [1.0])            # qubit >= n
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([res], dtype=object))
    finally:
        dist.destroy_process_group()


def _terms(n):
    """ZZ chain, Z on the top qubits, X/Y on local and on top qubits (one and two of
    them, with Z and Y mixed in)."""
    xs, zs, cs = W.zz_chain(n)
    top, top2 = 1 << (n - 1), 1 << (n - 2)
    return (list(xs) + [0, 0, 0b101, top, top | 0b10, top | top2, top2 | 1],
            list(zs) + [top | top2, top, 0b110, 0, top | 0b1, top2 | 0b100, top2 | top],
            list(cs) + [0.5, -1.25, 0.75, 0.3, -0.7, 1.1, 0.45])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world,n,k", [(2, 12, 4), (4, 11, 3)])
def test_executor_on_gloo_ranks_matches_the_oracle(svlib, world, n, k):
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), n, k, d), nprocs=world,
                           join=True, start_method="spawn")
        res = [np.load(os.path.join(d, f"rank{r}.npy"), allow_pickle=True)[0] for r in range(world)]
    specs = W.grid_random(n, 6) + W.random_unitary_gates(n, 12, 2, np.random.default_rng(7))
    ref = oracle.simulate(n, specs, x=37)
    want_e = oracle.expect(ref, *_terms(n))
    want_i, want_p = oracle.topk(oracle.probs(ref), 10)
    for r in res:
        assert np.max(np.abs(r["state"] - ref)) < 1e-12
        assert np.max(np.abs(r["state_after"] - ref)) < 1e-12
        assert abs(r["norm"] - 1.0) < 1e-12
        assert abs(r["expect"] - want_e) < 1e-12
        assert np.array_equal(r["topk"][0], want_i)
        assert np.allclose(r["topk"][1], want_p, rtol=0, atol=1e-14)
        assert r["rep"]["exchanges"] > 0 and r["bytes"] > 0
    assert len({r["rep"]["exchanges"] for r in res}) == 1      # one plan on every rank
