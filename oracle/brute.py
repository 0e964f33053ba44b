"""Brute-force Kronecker forms (test infrastructure only; see oracle/__init__.py).

An implementation independent of the oracle's amplitude loops, used to pin them at
n <= 10: a k-qubit gate becomes the full 2^n x 2^n operator of Eq. 3,
I_{2^{n-t-1}} (x) U (x) I_{2^t}, generalised to several (unsorted) targets by building
U (x) I on the "targets first" tensor axes and permuting the axes back.  Pauli strings
become Kronecker products of 2 x 2 matrices.  numpy's kron, transpose and matmul are the
only steps.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import gates as G


def full_operator(n: int, targets: Sequence[int], u: np.ndarray) -> np.ndarray:
    """2^n x 2^n operator of gate u on targets (local bit j <-> targets[j])."""
    k = len(targets)
    rest = [q for q in range(n) if q not in targets]
    # Operator on the ordering (targets[0], ..., targets[k-1], rest...) with the first
    # listed qubit least significant: kron puts its first factor most significant.
    op = np.kron(np.eye(1 << (n - k), dtype=np.complex128), np.asarray(u, np.complex128))
    order = list(targets) + rest              # local qubit position p -> physical qubit
    # As a tensor with 2n axes, numpy's C order lists the most significant bit first.
    t = op.reshape([2] * (2 * n))
    # axis a (0..n-1) of the row index is local bit n-1-a; move it to physical bit.
    src_to_phys = [order[n - 1 - a] for a in range(n)]
    perm_rows = [src_to_phys.index(n - 1 - a) for a in range(n)]
    perm = perm_rows + [n + p for p in perm_rows]
    return t.transpose(perm).reshape(1 << n, 1 << n)


def circuit_operator(n: int, gates) -> np.ndarray:
    """U_m ... U_1 (Eq. 10) for [(targets, U)]."""
    m = np.eye(1 << n, dtype=np.complex128)
    for tg, u in gates:
        m = full_operator(n, tg, u) @ m
    return m


def pauli_operator(n: int, xmask: int, zmask: int) -> np.ndarray:
    """Kronecker product of per-qubit I/X/Y/Z; qubit 0 is the last (least significant)
    factor."""
    op = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        x, z = (xmask >> q) & 1, (zmask >> q) & 1
        p = G.I2 if not x and not z else G.X if x and not z else G.Z if z and not x else G.Y
        op = np.kron(op, p)
    return op
