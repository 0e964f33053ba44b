"""Seeded synthetic circuit generators shared by the tests, the benchmark and smoke().

This module draws random numbers and lays gates out on qubits.  It holds none of the
simulation method's arithmetic: a gate is a symbolic record (a name from the paper's
canonical gate set, Eq. 4, its qubits, its angles).  Each side -- the CPU oracle and the
CUDA library -- builds the matrices from those records with its own gate library.  The
one exception is the "unitary" gate of the Table 3 workload (a Haar-random SU(2) element),
whose entries are themselves the random input, drawn here from normal deviates.

Seeds are fixed per workload: seed = 20261203 + 1000 * family + index.

Circuit families (all little-endian: qubit t is bit t of the amplitude index, Eq. 3):

* ``brickwork``  -- U3 on every qubit, then CZ on (i, i+1), even i in even layers and
  odd i in odd layers.  12 qubits x 20 layers = 240 U3 + 110 CZ.
* ``qft_brickwork`` -- QFT on a seeded basis state, then layers of U3 on every qubit
  followed by a CNOT ladder (i, i+1), i = 0..n-2 in order.
* ``grid_random`` -- Sycamore-style random circuit: per cycle one gate from
  {sqrtX, sqrtY, sqrtW} on every qubit, then fSim(pi/2, pi/6) on one of four edge
  classes of a 2-D grid (cycling A, B, C, D).
* ``hea`` -- hardware-efficient ansatz: RY then RZ on every qubit, then a CNOT ladder.
* ``table3_random`` -- 10 n Haar-random single-qubit gates on uniformly chosen qubits
  (the workload of the paper's Table 3).
* ``serving_stream`` -- Poisson arrivals of brickwork circuits of mixed width, depth and
  precision.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 20261203


def seed_for(family: int, index: int = 0) -> int:
    return SEED_BASE + 1000 * family + index


@dataclass(frozen=True)
class GateSpec:
    """One gate: canonical name, qubits (matrix local bit j <-> qubits[j]), angles."""

    name: str
    qubits: Tuple[int, ...]
    params: Tuple[float, ...] = ()
    dagger: bool = False
    matrix: Optional[Tuple[complex, ...]] = field(default=None, compare=False)

    def adjoint(self) -> "GateSpec":
        return GateSpec(self.name, self.qubits, self.params, not self.dagger, self.matrix)


# Gate names and arities understood by both gate libraries.
GATE_ARITY = {
    "i": 1, "x": 1, "y": 1, "z": 1, "h": 1, "s": 1, "t": 1,
    "rx": 1, "ry": 1, "rz": 1, "u3": 1,
    "sqrtx": 1, "sqrty": 1, "sqrtw": 1,
    "cnot": 2, "cz": 2, "swap": 2, "cp": 2, "fsim": 2,
    "toffoli": 3,
}
GATE_NPARAMS = {"rx": 1, "ry": 1, "rz": 1, "u3": 3, "cp": 1, "fsim": 2}


def mirror(gates: Sequence[GateSpec]) -> List[GateSpec]:
    """C followed by C^dagger (reversed order, each gate adjoint): returns any input state."""
    return list(gates) + [g.adjoint() for g in reversed(gates)]


# --------------------------------------------------------------------------- small circuits

def bell() -> List[GateSpec]:
    return [GateSpec("h", (0,)), GateSpec("cnot", (0, 1))]


def ghz(n: int) -> List[GateSpec]:
    return [GateSpec("h", (0,))] + [GateSpec("cnot", (i, i + 1)) for i in range(n - 1)]


def qft(n: int, swaps: bool = True) -> List[GateSpec]:
    """QFT with the most significant qubit first; the final swaps reverse the bit order."""
    gates: List[GateSpec] = []
    for j in range(n - 1, -1, -1):
        gates.append(GateSpec("h", (j,)))
        for k in range(j - 1, -1, -1):
            gates.append(GateSpec("cp", (k, j), (math.pi / 2 ** (j - k),)))
    if swaps:
        for i in range(n // 2):
            gates.append(GateSpec("swap", (i, n - 1 - i)))
    return gates


# --------------------------------------------------------------------------- families

def brickwork(n: int = 12, layers: int = 20, seed: Optional[int] = None,
              two_qubit: str = "cz") -> List[GateSpec]:
    rng = np.random.default_rng(seed_for(1) if seed is None else seed)
    gates: List[GateSpec] = []
    for layer in range(layers):
        ang = rng.uniform(0.0, 2.0 * math.pi, size=(n, 3))
        for q in range(n):
            gates.append(GateSpec("u3", (q,), tuple(float(a) for a in ang[q])))
        for i in range(layer % 2, n - 1, 2):
            gates.append(GateSpec(two_qubit, (i, i + 1)))
    return gates


def qft_brickwork(n: int = 24, layers: int = 40, seed: Optional[int] = None):
    """Returns (x, gates): the seeded basis state |x> and QFT + U3/CNOT-ladder layers."""
    rng = np.random.default_rng(seed_for(2) if seed is None else seed)
    x = int(rng.integers(0, 2 ** n))
    gates = qft(n)
    for _ in range(layers):
        ang = rng.uniform(0.0, 2.0 * math.pi, size=(n, 3))
        for q in range(n):
            gates.append(GateSpec("u3", (q,), tuple(float(a) for a in ang[q])))
        for i in range(n - 1):
            gates.append(GateSpec("cnot", (i, i + 1)))
    return x, gates


def grid_shape(n: int) -> Tuple[int, int]:
    """(rows, cols): cols = ceil(sqrt(n)), row-major, last row possibly partial."""
    cols = int(math.ceil(math.sqrt(n)))
    rows = (n + cols - 1) // cols
    return rows, cols


def grid_edges(n: int, cls: str) -> List[Tuple[int, int]]:
    """Edge classes A/B: horizontal with even/odd left column; C/D: vertical with
    even/odd top row."""
    rows, cols = grid_shape(n)
    edges = []
    for q in range(n):
        r, c = divmod(q, cols)
        if cls in "AB":
            if c + 1 < cols and q + 1 < n and (c % 2 == (0 if cls == "A" else 1)):
                edges.append((q, q + 1))
        else:
            if q + cols < n and (r % 2 == (0 if cls == "C" else 1)):
                edges.append((q, q + cols))
    return edges


def grid_random(n: int = 30, cycles: int = 24, seed: Optional[int] = None) -> List[GateSpec]:
    rng = np.random.default_rng(seed_for(3, n) if seed is None else seed)
    names = ("sqrtx", "sqrty", "sqrtw")
    fsim = (math.pi / 2, math.pi / 6)
    gates: List[GateSpec] = []
    for cyc in range(cycles):
        pick = rng.integers(0, 3, size=n)
        for q in range(n):
            gates.append(GateSpec(names[int(pick[q])], (q,)))
        for a, b in grid_edges(n, "ABCD"[cyc % 4]):
            gates.append(GateSpec("fsim", (a, b), fsim))
    return gates


def hea(n: int, layers: int = 6, rng: Optional[np.random.Generator] = None,
        seed: Optional[int] = None) -> List[GateSpec]:
    if rng is None:
        rng = np.random.default_rng(seed_for(4) if seed is None else seed)
    gates: List[GateSpec] = []
    for _ in range(layers):
        th = rng.uniform(-math.pi, math.pi, size=n)
        ph = rng.uniform(-math.pi, math.pi, size=n)
        for q in range(n):
            gates.append(GateSpec("ry", (q,), (float(th[q]),)))
            gates.append(GateSpec("rz", (q,), (float(ph[q]),)))
        for i in range(n - 1):
            gates.append(GateSpec("cnot", (i, i + 1)))
    return gates


def hea_batch(count: int = 512, widths: Sequence[int] = (16, 18, 20, 22), layers: int = 6,
              seed: Optional[int] = None) -> List[Tuple[int, List[GateSpec]]]:
    """count circuits of width drawn uniformly from `widths`, each with its own angles."""
    rng = np.random.default_rng(seed_for(4) if seed is None else seed)
    w = rng.choice(np.asarray(widths), size=count)
    return [(int(wi), hea(int(wi), layers, rng=rng)) for wi in w]


def zz_chain(n: int):
    """Open-chain sum_{i=0}^{n-2} Z_i Z_{i+1} as (xmask, zmask, coef) lists."""
    xs = [0] * (n - 1)
    zs = [(1 << i) | (1 << (i + 1)) for i in range(n - 1)]
    cs = [1.0] * (n - 1)
    return xs, zs, cs


def haar_su2(rng: np.random.Generator) -> Tuple[complex, ...]:
    """Haar-random SU(2) element from a uniformly random unit quaternion."""
    v = rng.normal(size=4)
    v = v / np.linalg.norm(v)
    a = complex(v[0], v[3])
    b = complex(v[2], v[1])
    # [[a, -conj(b)], [b, conj(a)]], row-major
    return (a, -b.conjugate(), b, a.conjugate())


def table3_random(n: int, seed: Optional[int] = None) -> List[GateSpec]:
    rng = np.random.default_rng(seed_for(6, n) if seed is None else seed)
    gates = []
    for _ in range(10 * n):
        q = int(rng.integers(0, n))
        gates.append(GateSpec("unitary", (q,), (), False, haar_su2(rng)))
    return gates


def haar_unitary(d: int, rng: np.random.Generator) -> Tuple[complex, ...]:
    """Haar-random d x d unitary: the Q factor of a complex Gaussian matrix with the
    phases of R's diagonal folded in."""
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    q = q * (np.diagonal(r) / np.abs(np.diagonal(r)))
    return tuple(complex(c) for c in q.ravel())


def random_unitary_gates(n: int, count: int, kmax: int, rng: np.random.Generator,
                         exact_k: bool = False, targets: Optional[Sequence[int]] = None
                         ) -> List[GateSpec]:
    """Random dense k-qubit gates (k <= kmax, or k = kmax with exact_k) on random,
    unsorted distinct targets (or on the given targets, in the given order).  Used for
    parity cases over every target set."""
    gates = []
    for _ in range(count):
        if targets is not None:
            tg = tuple(int(t) for t in targets)
        else:
            k = kmax if exact_k else int(rng.integers(1, kmax + 1))
            k = min(k, n)
            tg = tuple(int(t) for t in rng.choice(n, size=k, replace=False))
        gates.append(GateSpec("unitary", tg, (), False, haar_unitary(1 << len(tg), rng)))
    return gates


def phase_heavy(n: int, count: int, seed: Optional[int] = None) -> List[GateSpec]:
    """Random circuits dominated by diagonal and controlled gates (CP, RZ, T, Z, CZ, CNOT,
    Toffoli) with some dense ones (H, random 2-qubit unitaries), on random qubits: inputs
    where commutation and gate structure matter."""
    rng = np.random.default_rng(seed_for(7, n) if seed is None else seed)
    gates: List[GateSpec] = []
    for _ in range(count):
        r = rng.random()
        q = tuple(int(x) for x in rng.choice(n, size=min(3, n), replace=False))
        if r < 0.25 and n >= 2:
            gates.append(GateSpec("cp", q[:2], (float(rng.uniform(0, 2 * math.pi)),)))
        elif r < 0.33:
            gates.append(GateSpec("rz", q[:1], (float(rng.uniform(0, 2 * math.pi)),)))
        elif r < 0.4:
            gates.append(GateSpec(str(rng.choice(["t", "z"])), q[:1]))
        elif r < 0.5 and n >= 2:
            gates.append(GateSpec("cz", q[:2]))
        elif r < 0.65 and n >= 2:
            gates.append(GateSpec("cnot", q[:2]))
        elif r < 0.7 and n >= 3:
            gates.append(GateSpec("toffoli", q[:3]))
        elif r < 0.85 or n < 2:
            gates.append(GateSpec("h", q[:1]))
        else:
            gates.append(GateSpec("unitary", q[:2], (), False, haar_unitary(4, rng)))
    return gates


def qaoa(n: int, layers: int = 3, edges: int = 24, seed: Optional[int] = None) -> List[GateSpec]:
    """QAOA-style layers: exp(-i gamma Z_a Z_b) on `edges` random pairs in random order
    (diag(e^{-i g}, e^{i g}, e^{i g}, e^{-i g})), then RX(beta) on every qubit."""
    rng = np.random.default_rng(seed_for(8, n) if seed is None else seed)
    gates: List[GateSpec] = []
    for _ in range(layers):
        g = float(rng.uniform(0, math.pi))
        pairs = set()
        while len(pairs) < min(edges, n * (n - 1) // 2):
            a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
            pairs.add((min(a, b), max(a, b)))
        order = sorted(pairs)
        rng.shuffle(order)
        zz = (complex(math.cos(g), -math.sin(g)), 0j, 0j, 0j,
              0j, complex(math.cos(g), math.sin(g)), 0j, 0j,
              0j, 0j, complex(math.cos(g), math.sin(g)), 0j,
              0j, 0j, 0j, complex(math.cos(g), -math.sin(g)))
        for a, b in order:
            gates.append(GateSpec("unitary", (a, b), (), False, zz))
        beta = float(rng.uniform(0, math.pi))
        for q in range(n):
            gates.append(GateSpec("rx", (q,), (beta,)))
    return gates


@dataclass
class Request:
    arrival_s: float
    width: int
    depth: int
    dtype: str          # "c64" or "c128"
    gates: List[GateSpec]


def serving_stream(rate_hz: float, duration_s: float, seed: Optional[int] = None,
                   width_range=(10, 30), depth_range=(10, 60), frac_c64: float = 0.7,
                   max_requests: Optional[int] = None) -> List[Request]:
    """Poisson arrivals of brickwork circuits of width ~ U{10..30}, depth ~ U{10..60}:
    the arrivals within duration_s, at most max_requests of them."""
    rng = np.random.default_rng(seed_for(5, int(rate_hz)) if seed is None else seed)
    t = 0.0
    out: List[Request] = []
    i = 0
    while max_requests is None or i < max_requests:
        t += float(rng.exponential(1.0 / rate_hz))
        if t > duration_s:
            break
        w = int(rng.integers(width_range[0], width_range[1] + 1))
        d = int(rng.integers(depth_range[0], depth_range[1] + 1))
        dt = "c64" if rng.uniform() < frac_c64 else "c128"
        out.append(Request(t, w, d, dt, brickwork(w, d, seed=int(rng.integers(0, 2**31)))))
        i += 1
    return out
