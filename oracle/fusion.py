"""Oracle for DAG-based gate fusion (test infrastructure only; see oracle/__init__.py).

Follows Section 5 of the paper in its own order:

* DAG construction (Section 5.1, Eq. 8): one vertex per gate; scanning the gates in
  order with a map from each qubit to the last gate that acted on it, an edge (u, v) is
  added for every qubit of v whose last gate is u.  So |E| <= sum_v |q(v)|.
* Fusion (Section 5.2, Algorithm 2, Eq. 9): repeat sweeps until a sweep changes
  nothing; each sweep takes the vertices in topological order and, for each vertex v,
  tries its predecessors u.  u and v fuse when (1) (u, v) is an edge, (2)
  |q(u) | q(v)| <= q_max^fuse and (3) u is v's only route on the qubits they share.
  The fused gate replaces u with U_fused = U_v . U_u on q(u) | q(v); v's edges move to
  u and v is removed.  The sweep then moves on to the next vertex.

Readings where the paper is silent or ambiguous:

* Condition (3) is read as "contracting the edge (u, v) keeps the graph acyclic": there
  is no other directed path from u to v.  This implies the printed condition (no other
  predecessor of v acts on the qubits of u after u) and also rules out longer detours.
* Topological order: Kahn's algorithm that always takes the ready vertex with the
  smallest id.  A vertex starts with its gate's index as id; a fused vertex keeps the
  id of u, the predecessor that absorbed v.
* Predecessors of v are tried in ascending order of |q(u) | q(v)| (the narrowest fused
  gate first, which leaves room for later contractions), ties by ascending id.  The
  paper's loop over "each predecessor" leaves the order open.
* A fused gate's qubits are sorted ascending and each factor is embedded on the union
  with identities on the other qubits before the product.
* q_max^fuse = 0 means no fusion: the gates come back unchanged (targets sorted).

The output is the list of surviving vertices in the same topological order.

Commutation-aware variant (``commute=True``; the paper's fusion has no commutativity
analysis and names it as future work, Sections 10-11):

* Two gates commute when, on every qubit they share, both are diagonal in that qubit
  (the gate's matrix never changes the qubit's bit) -- a sufficient condition.
* DAG: for each qubit, scanning the gates in order, a gate that is not diagonal on it
  gets an edge from every gate on it since (and including) the last such gate, and a
  gate diagonal on it gets an edge from that last non-diagonal gate only.  Two gates
  with no path between them then commute, so every topological order gives the same
  product.
* Fusion: Algorithm 2 as above; after v's predecessors, the sweep also tries the
  vertices that share a qubit with v, are placed before v in the sweep's topological
  order and are not its predecessors, in ascending id, contracting one when there is no
  path from it to v (the two commute, so U_fused = U_v . U_u is the product in either
  order); both groups in the same order as the predecessors above.
"""
from __future__ import annotations

import heapq
from typing import Dict, List, Sequence, Set, Tuple

import numpy as np


def sort_targets(targets: Sequence[int], u: np.ndarray) -> Tuple[Tuple[int, ...], np.ndarray]:
    """Same operator with its targets listed in ascending order.

    The operator is fixed by u[loc_out][loc_in] with loc = sum_j bit(targets[j]) 2^j;
    relabelling local bits permutes rows and columns alike."""
    k = len(targets)
    order = sorted(range(k), key=lambda j: targets[j])      # new bit j <- old bit order[j]
    new_t = tuple(targets[j] for j in order)
    d = 1 << k
    perm = np.zeros(d, dtype=np.int64)                       # perm[new_idx] = old_idx
    for new_idx in range(d):
        old = 0
        for j in range(k):
            if (new_idx >> j) & 1:
                old |= 1 << order[j]
        perm[new_idx] = old
    return new_t, u[np.ix_(perm, perm)].copy()


def embed(u: np.ndarray, qa: Sequence[int], qs: Sequence[int]) -> np.ndarray:
    """Operator u on sorted qubits qa, as a matrix on the sorted superset qs (identity
    on qs minus qa)."""
    pos = [qs.index(q) for q in qa]
    m = len(qs)
    d = 1 << m
    r = np.arange(d)
    ex = np.zeros(d, dtype=np.int64)
    amask = 0
    for j, p in enumerate(pos):
        ex |= ((r >> p) & 1) << j
        amask |= 1 << p
    rest = r & ~amask
    same = rest[:, None] == rest[None, :]
    return np.where(same, u[ex[:, None], ex[None, :]], 0.0 + 0.0j)


class Dag:
    def __init__(self, gates: Sequence[Tuple[Sequence[int], np.ndarray]], n: int):
        self.q: Dict[int, Tuple[int, ...]] = {}
        self.u: Dict[int, np.ndarray] = {}
        self.preds: Dict[int, Set[int]] = {}
        self.succs: Dict[int, Set[int]] = {}
        last = [-1] * n
        for i, (tg, u) in enumerate(gates):
            st, su = sort_targets(tuple(tg), np.asarray(u, dtype=np.complex128))
            self.q[i], self.u[i] = st, su
            self.preds[i], self.succs[i] = set(), set()
            for qb in st:
                if last[qb] >= 0:
                    self.preds[i].add(last[qb])
                    self.succs[last[qb]].add(i)
                last[qb] = i

    def topo_order(self) -> List[int]:
        indeg = {v: len(p) for v, p in self.preds.items()}
        ready = [v for v, d in indeg.items() if d == 0]
        heapq.heapify(ready)
        out = []
        while ready:
            v = heapq.heappop(ready)
            out.append(v)
            for w in self.succs[v]:
                indeg[w] -= 1
                if indeg[w] == 0:
                    heapq.heappush(ready, w)
        assert len(out) == len(self.preds), "cycle in fusion DAG"
        return out

    def other_path(self, u: int, v: int) -> bool:
        """Is there a directed path u -> ... -> v other than the edge (u, v)?"""
        stack = [w for w in self.succs[u] if w != v]
        seen = set(stack)
        while stack:
            w = stack.pop()
            if w == v:
                return True
            for x in self.succs[w]:
                if x not in seen:
                    seen.add(x)
                    stack.append(x)
        return False

    def contract(self, u: int, v: int) -> None:
        qs = tuple(sorted(set(self.q[u]) | set(self.q[v])))
        # Eq. 9: U_fused = U_v . U_u (u first, v second)
        self.u[u] = embed(self.u[v], self.q[v], qs) @ embed(self.u[u], self.q[u], qs)
        self.q[u] = qs
        for w in self.preds[v]:
            if w != u:
                self.succs[w].discard(v)
                self.succs[w].add(u)
                self.preds[u].add(w)
        for w in self.succs[v]:
            self.preds[w].discard(v)
            self.preds[w].add(u)
            self.succs[u].add(w)
        self.succs[u].discard(v)
        del self.preds[v], self.succs[v], self.q[v], self.u[v]


def diagonal_on(u: np.ndarray, j: int) -> bool:
    """True when the matrix never changes local bit j: u[r][c] = 0 whenever bit j of r
    differs from bit j of c."""
    d = u.shape[0]
    for r in range(d):
        for c in range(d):
            if ((r >> j) & 1) != ((c >> j) & 1) and u[r, c] != 0:
                return False
    return True


class CommutingDag(Dag):
    """The DAG of the commutation-aware variant (see the module docstring)."""

    def __init__(self, gates: Sequence[Tuple[Sequence[int], np.ndarray]], n: int):
        self.q, self.u, self.preds, self.succs = {}, {}, {}, {}
        last_nondiag = [-1] * n
        diag_since = [[] for _ in range(n)]   # gates diagonal on the qubit since then
        for i, (tg, u) in enumerate(gates):
            st, su = sort_targets(tuple(tg), np.asarray(u, dtype=np.complex128))
            self.q[i], self.u[i] = st, su
            self.preds[i], self.succs[i] = set(), set()
            for j, qb in enumerate(st):
                if diagonal_on(su, j):
                    deps = [last_nondiag[qb]] if last_nondiag[qb] >= 0 else []
                    diag_since[qb].append(i)
                else:
                    deps = list(diag_since[qb])
                    if last_nondiag[qb] >= 0:
                        deps.append(last_nondiag[qb])
                    last_nondiag[qb] = i
                    diag_since[qb] = []
                for p in deps:
                    self.preds[i].add(p)
                    self.succs[p].add(i)

    def any_path(self, u: int, v: int) -> bool:
        """Is there a directed path u -> ... -> v?"""
        stack = list(self.succs[u])
        seen = set(stack)
        while stack:
            w = stack.pop()
            if w == v:
                return True
            for x in self.succs[w]:
                if x not in seen:
                    seen.add(x)
                    stack.append(x)
        return False


def fuse(gates: Sequence[Tuple[Sequence[int], np.ndarray]], n: int, qmax: int,
         commute: bool = False) -> List[Tuple[Tuple[int, ...], np.ndarray]]:
    """Algorithm 2 (commutation-aware with commute=True).  Returns [(sorted targets, U)]
    in topological order."""
    dag = CommutingDag(gates, n) if commute else Dag(gates, n)
    changed = qmax > 0
    while changed:
        changed = False
        order = dag.topo_order()
        pos = {v: i for i, v in enumerate(order)}
        for v in order:
            if v not in dag.preds:            # absorbed earlier in this sweep
                continue
            def width_then_id(u):
                return (len(set(dag.q[u]) | set(dag.q[v])), u)
            cands = sorted(dag.preds[v], key=width_then_id)
            if commute:
                cands += sorted((w for w in dag.preds if w != v and w not in dag.preds[v]
                                 and pos[w] < pos[v] and set(dag.q[w]) & set(dag.q[v])),
                                key=width_then_id)
            for u in cands:
                if len(set(dag.q[u]) | set(dag.q[v])) > qmax:
                    continue
                if u in dag.preds[v]:
                    if dag.other_path(u, v):
                        continue
                elif dag.any_path(u, v):
                    continue
                dag.contract(u, v)
                changed = True
                break
    return [(dag.q[v], dag.u[v]) for v in dag.topo_order()]
