"""Structure of a gate matrix: control qubits, and a diagonal or monomial remainder --
oracle side.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper densifies every fused gate and lists the missing structure and commutativity
analysis among the limits of its fusion (Section 10) and its future work (Section 11).
The library's structure-aware application rests on these exact definitions, taken on
the FP64 entries of U (2^k x 2^k, local bit j <-> targets[j]):

* local bit j is a CONTROL of U when U never changes bit j (U[r][c] = 0 whenever bit j
  of r differs from bit j of c) and U is the identity on the half where bit j is 0
  (U[r][c] = [r == c] whenever bit j of r and of c is 0);
* the REDUCED gate V is U restricted to the rows and columns whose control bits are all
  1, on the remaining targets in their order; with the controls C,
  U = (I - P_C) + P_C (V (x) I_C) where P_C projects on "every control bit is 1";
* V is DIAGONAL when all its off-diagonal entries are 0, MONOMIAL when every row and
  every column has exactly one nonzero entry (a permutation with phases), else DENSE;
  a 1 x 1 V equal to 1 is the IDENTITY (U = I).

Plain loops over the matrix entries; no tolerance anywhere.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

DENSE, DIAGONAL, MONOMIAL, IDENTITY = 0, 1, 2, 3


def is_control(u: np.ndarray, j: int) -> bool:
    d = u.shape[0]
    for r in range(d):
        for c in range(d):
            br, bc = (r >> j) & 1, (c >> j) & 1
            if br != bc and u[r, c] != 0:
                return False
            if br == 0 and bc == 0 and u[r, c] != (1.0 if r == c else 0.0):
                return False
    return True


def controls(u: np.ndarray) -> List[int]:
    k = u.shape[0].bit_length() - 1
    return [j for j in range(k) if is_control(u, j)]


def reduced(targets: Sequence[int], u: np.ndarray) -> Tuple[List[int], List[int], np.ndarray]:
    """(control qubits, remaining targets, V)."""
    u = np.asarray(u, dtype=np.complex128)
    ctl = controls(u)
    k = len(targets)
    keep = [j for j in range(k) if j not in ctl]
    cmask = sum(1 << j for j in ctl)
    idx = []                                  # V's index a -> U's index with controls 1
    for a in range(1 << len(keep)):
        x = cmask
        for i, j in enumerate(keep):
            if (a >> i) & 1:
                x |= 1 << j
        idx.append(x)
    v = u[np.ix_(idx, idx)].copy()
    return [targets[j] for j in ctl], [targets[j] for j in keep], v


def kind(v: np.ndarray) -> int:
    d = v.shape[0]
    if d == 1 and v[0, 0] == 1.0:
        return IDENTITY
    nz = v != 0
    if all(not nz[r, c] for r in range(d) for c in range(d) if r != c):
        return DIAGONAL
    if all(nz[r, :].sum() == 1 for r in range(d)) and all(nz[:, c].sum() == 1 for c in range(d)):
        return MONOMIAL
    return DENSE


def classify(targets: Sequence[int], u: np.ndarray) -> Tuple[int, int]:
    """(kind, control mask over local bits)."""
    u = np.asarray(u, dtype=np.complex128)
    ctl = controls(u)
    _, _, v = reduced(targets, u)
    return kind(v), sum(1 << j for j in ctl)


def touched_fraction(u: np.ndarray) -> float:
    """Share of the amplitudes a structure-aware pass reads: those whose control bits are
    all 1 (none for the identity)."""
    k = u.shape[0].bit_length() - 1
    ctl = controls(np.asarray(u, dtype=np.complex128))
    return 0.0 if len(ctl) == k and u[-1, -1] == 1.0 else 0.5 ** len(ctl)
