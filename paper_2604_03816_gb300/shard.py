"""One state vector over 2^g processes: the executor of a shard plan (sv_shard_plan_*).

Rank r holds the amplitudes r 2^L .. (r + 1) 2^L - 1 (L = n - g) as an ordinary L-qubit
state on its own GPU.  Every rank walks the same plan: segments of gates on local qubits
are applied by the library's passes, and each swap of a local bit position p with a
global bit j is an exchange of half a shard with the partner rank r ^ 2^j, moved in
chunks through staging buffers (sv_shard_pack -> send/recv -> sv_shard_unpack; when p is
the top local bit the outgoing half is contiguous and is sent from the state itself).
Reductions finish with one FP64 sum over the ranks.  The paper runs on one device and
names multi-device partitioning as future work (Sections 10-11).

The transport is a `comm` object:
  * TorchComm -- torch.distributed point-to-point (NCCL between GPUs, one process each;
    gloo between CPU processes);
  * ThreadComm -- ranks as threads of one process on one GPU, the exchange a device copy
    between their staging buffers after a host barrier (for testing the path on a single
    GPU: no kernel of one rank waits on another rank's kernels).
The local part is a GpuShard (the C ABI on the current CUDA device); the executor itself
holds no arithmetic.
"""
from __future__ import annotations

import threading
from typing import List, Sequence, Tuple

import numpy as np

from . import sv


# --------------------------------------------------------------------------- transports

class TorchComm:
    """Exchanges and sums over torch.distributed (NCCL for CUDA tensors, gloo for CPU ones)."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.torch = torch
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        self.device = device if device is not None else ("cuda" if dist.get_backend() == "nccl" else "cpu")

    def exchange(self, send, recv, partner: int) -> None:
        """recv <- the partner's send (same size), while the partner receives ours."""
        ops = [self.dist.P2POp(self.dist.isend, send, partner),
               self.dist.P2POp(self.dist.irecv, recv, partner)]
        for req in self.dist.batch_isend_irecv(ops):
            req.wait()

    def sum(self, value: float) -> float:
        t = self.torch.tensor([value], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t)
        return float(t.item())

    def allgather(self, obj) -> list:
        out = [None] * self.world
        self.dist.all_gather_object(out, obj)
        return out


class ThreadHub:
    """Shared by the ThreadComm of every rank of one process."""

    def __init__(self, world: int):
        self.world = world
        self.barrier = threading.Barrier(world)
        self.slots = [None] * world


class ThreadComm:
    """Ranks as threads of one process (one GPU): host barriers order the ranks, a device
    copy on the receiving rank's stream moves the data."""

    def __init__(self, hub: ThreadHub, rank: int):
        self.hub, self.rank, self.world = hub, rank, hub.world

    def exchange(self, send, recv, partner: int) -> None:
        import torch
        torch.cuda.current_stream().synchronize()      # this rank's send buffer is final
        self.hub.slots[self.rank] = send
        self.hub.barrier.wait()
        recv.copy_(self.hub.slots[partner])
        torch.cuda.current_stream().synchronize()      # copied before the partner reuses it
        self.hub.barrier.wait()

    def allgather(self, obj) -> list:
        self.hub.slots[self.rank] = obj
        self.hub.barrier.wait()
        out = list(self.hub.slots)
        self.hub.barrier.wait()
        return out

    def sum(self, value: float) -> float:
        vals = self.allgather(value)
        total = 0.0
        for v in vals:                   # rank order: the same sum on every rank
            total += v
        return total


# --------------------------------------------------------------------------- local part

class GpuShard:
    """This rank's 2^L amplitudes as an sv_state in a torch-owned device buffer, plus two
    staging buffers of `chunk` amplitudes."""

    def __init__(self, L: int, dtype: int, stream=None, chunk: int = 1 << 26):
        import torch
        self.torch = torch
        self.L, self.dtype = L, dtype
        self.esize = 8 if dtype == sv.SV_C64 else 16
        self.chunk = min(chunk, 1 << max(L - 1, 0))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.buf = torch.empty(self.esize << L, dtype=torch.uint8, device="cuda")
        self.state = sv.sv_alloc(L, dtype, dev_buf=self.buf, stream=self.stream)
        self.sendbuf = torch.empty(self.esize * self.chunk, dtype=torch.uint8, device="cuda")
        self.recvbuf = torch.empty(self.esize * self.chunk, dtype=torch.uint8, device="cuda")

    def set_basis(self, x: int) -> None:
        sv.sv_set_basis(self.state, x)

    def set_zero(self) -> None:
        sv.sv_set_zero(self.state)

    def apply(self, seg: sv.Circuit) -> dict:
        return sv.sv_apply_circuit(self.state, seg)

    def outgoing(self, bit: int, value: int, off: int, cnt: int):
        """The cnt amplitudes off.. of the half (bit = value), as a device tensor."""
        if bit == self.L - 1:           # that half is contiguous: send from the state itself
            base = (value << (self.L - 1)) + off
            return self.buf[base * self.esize:(base + cnt) * self.esize]
        dst = self.sendbuf[:cnt * self.esize]
        sv.sv_shard_pack(self.state, bit, value, off, cnt, dst)
        return dst

    def incoming(self, cnt: int):
        return self.recvbuf[:cnt * self.esize]

    def store(self, bit: int, value: int, off: int, cnt: int, src) -> None:
        sv.sv_shard_unpack(self.state, bit, value, off, cnt, src)

    def norm(self) -> float:
        return sv.sv_norm(self.state)

    def expect(self, xs, zs, cs) -> float:
        return sv.sv_expect(self.state, xs, zs, cs) if len(xs) else 0.0

    def topk(self, k: int):
        return sv.sv_topk(self.state, k)

    def get_state(self) -> np.ndarray:
        return sv.sv_get_state(self.state)

    def free(self) -> None:
        self.state.free()


# --------------------------------------------------------------------------- executor

class ShardedState:
    """An n-qubit state over comm.world = 2^g ranks; every rank constructs one and makes
    the same calls in the same order."""

    def __init__(self, n: int, dtype: int, comm, local):
        world = comm.world
        g = world.bit_length() - 1
        if (1 << g) != world:
            raise ValueError("the number of ranks must be a power of two")
        self.n, self.g, self.L, self.dtype = n, g, n - g, dtype
        self.comm, self.local, self.rank = comm, local, comm.rank
        self.exchanged_bytes = 0
        self.exchanges = 0

    # ---- initialisation
    def set_basis(self, x: int) -> None:
        if x >> self.n:
            raise ValueError("x >= 2^n")
        if (x >> self.L) == self.rank:
            self.local.set_basis(x & ((1 << self.L) - 1))
        else:
            self.local.set_zero()

    # ---- gates
    def apply_circuit(self, circuit: sv.Circuit) -> dict:
        plan = sv.sv_shard_plan_create(circuit, self.g, self.dtype)
        passes = 0
        for kind, p, j, seg in plan.steps():
            if kind == sv.SV_SHARD_APPLY:
                passes += self.local.apply(seg)["passes"]
            else:
                self._exchange(p, j)
        nsteps, nex, nswap = plan.info()
        return {"passes": passes, "exchanges": nex, "swap_passes": nswap, "steps": nsteps}

    def _exchange(self, p: int, j: int) -> None:
        partner = self.rank ^ (1 << j)
        value = 1 - ((self.rank >> j) & 1)     # the half this rank gives away (and refills)
        half = 1 << (self.L - 1)
        chunk = self.local.chunk
        for off in range(0, half, chunk):
            cnt = min(chunk, half - off)
            send = self.local.outgoing(p, value, off, cnt)
            recv = self.local.incoming(cnt)
            self.comm.exchange(send, recv, partner)
            self.local.store(p, value, off, cnt, recv)
            self.exchanged_bytes += 2 * cnt * (8 if self.dtype == sv.SV_C64 else 16)
        self.exchanges += 1

    # ---- reductions (the layout is the identity after every apply_circuit)
    def norm(self) -> float:
        return self.comm.sum(self.local.norm())

    def _local_terms(self, terms):
        """Terms with no X/Y on the top qubits as this rank's terms: Z on a top qubit
        contributes the sign of the rank's bit there."""
        lo = (1 << self.L) - 1
        xs, zs, cs = [], [], []
        for x, z, c in terms:
            sign = -1.0 if bin((z >> self.L) & self.rank).count("1") & 1 else 1.0
            xs.append(x)
            zs.append(z & lo)
            cs.append(sign * c)
        return xs, zs, cs

    def expect(self, xmask: Sequence[int], zmask: Sequence[int], coef: Sequence[float]) -> float:
        """sum_t coef[t] <P_t> for Pauli strings on any qubits.  Terms are grouped by their
        X/Y part on the top qubits; a group that flips top qubits has each of them swapped
        into a local position the group does not flip (one exchange each, as in a plan),
        is summed on the shards with its masks relabelled, and the same exchanges swap the
        qubits back.  One FP64 sum over the ranks at the end."""
        L = self.L
        lo = (1 << L) - 1
        groups = {}
        for x, z, c in zip(xmask, zmask, coef):
            if (x | z) >> self.n:
                raise ValueError("a Pauli mask names a qubit >= n")
            groups.setdefault(x >> L, []).append((x, z, c))
        total = 0.0
        for gx in sorted(groups):
            terms = groups[gx]
            if gx == 0:
                total += self.local.expect(*self._local_terms(terms))
                continue
            js = [j for j in range(self.g) if (gx >> j) & 1]
            flipped = 0
            for x, _, _ in terms:
                flipped |= x & lo
            free = [p for p in range(L - 1, -1, -1) if not (flipped >> p) & 1]
            if len(free) < len(js):
                raise ValueError("too few local qubits outside the terms' X/Y part to swap the "
                                 "top qubits in")
            swaps = list(zip(free[:len(js)], js))
            for p, j in swaps:
                self._exchange(p, j)
            mapped = []
            for x, z, c in terms:
                for p, j in swaps:                    # qubit L + j now at p, qubit p at L + j
                    q = L + j
                    bxq, bzq, bxp, bzp = (x >> q) & 1, (z >> q) & 1, (x >> p) & 1, (z >> p) & 1
                    keep = ~((1 << q) | (1 << p))
                    x = (x & keep) | (bxq << p) | (bxp << q)
                    z = (z & keep) | (bzq << p) | (bzp << q)
                mapped.append((x, z, c))
            total += self.local.expect(*self._local_terms(mapped))
            for p, j in reversed(swaps):
                self._exchange(p, j)
        return self.comm.sum(total)

    def topk(self, k: int) -> Tuple[np.ndarray, np.ndarray]:
        """The k most probable outcomes over all ranks, ties to the lower index."""
        idx, p = self.local.topk(k)
        mine = [(float(pp), int(i) + (self.rank << self.L)) for i, pp in zip(idx, p)]
        allc = [c for part in self.comm.allgather(mine) for c in part]
        allc.sort(key=lambda t: (-t[0], t[1]))
        best = allc[:min(k, 1 << self.n)]
        return (np.array([i for _, i in best], dtype=np.uint64),
                np.array([pp for pp, _ in best], dtype=np.float64))

    def get_state(self) -> np.ndarray:
        """The whole state on every rank (small n only: for tests)."""
        parts = self.comm.allgather(self.local.get_state())
        return np.concatenate(parts)
