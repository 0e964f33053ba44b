"""Density-matrix simulation with single-qubit depolarizing noise after every gate
(Section 9.5, Table 8) -- oracle side.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

rho is a 2^n x 2^n complex128 matrix, rho[r, c] with qubit t = bit t of r and of c.
* A gate U on targets T maps rho -> E(U) rho E(U)^dagger with E(U) the full operator
  (identities elsewhere, Eq. 3).
* The depolarizing channel with probability p on qubit q maps
  rho -> (1 - p) rho + (p / 3) (X_q rho X_q + Y_q rho Y_q + Z_q rho Z_q);
  the noisy circuit applies it to every target of a gate right after the gate.
* The outcome distribution is p(x) = Re rho[x, x]; against a reference distribution q:
  classical fidelity F_cl = (sum_x sqrt(p(x) q(x)))^2 and TVD = (1/2) sum_x |p(x) - q(x)|.

Plain dense matrices (n <= 10): the point is being obviously correct.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np

from . import brute

X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def pure(psi: np.ndarray) -> np.ndarray:
    """|psi><psi|."""
    return np.outer(psi, np.conj(psi))


def apply_gate(rho: np.ndarray, n: int, targets: Sequence[int], u: np.ndarray) -> np.ndarray:
    e = brute.full_operator(n, targets, u)
    return e @ rho @ e.conj().T


def depolarize(rho: np.ndarray, n: int, q: int, p: float) -> np.ndarray:
    out = (1.0 - p) * rho
    for P in (X, Y, Z):
        e = brute.full_operator(n, (q,), P)
        out = out + (p / 3.0) * (e @ rho @ e.conj().T)
    return out


def run(n: int, gate_list, p: float, rho0: np.ndarray = None) -> np.ndarray:
    """The noisy circuit from rho0 (default |0..0><0..0|): each gate, then the channel on
    each of its targets."""
    rho = rho0.copy() if rho0 is not None else pure(np.eye(1 << n, dtype=np.complex128)[0])
    for targets, u in gate_list:
        rho = apply_gate(rho, n, targets, u)
        if p:
            for q in targets:
                rho = depolarize(rho, n, q, p)
    return rho


def probs(rho: np.ndarray) -> np.ndarray:
    return np.real(np.diag(rho)).copy()


def classical_fidelity(p: np.ndarray, q: np.ndarray) -> float:
    return float(np.sum(np.sqrt(np.clip(p, 0, None) * np.clip(q, 0, None))) ** 2)


def tvd(p: np.ndarray, q: np.ndarray) -> float:
    return float(0.5 * np.sum(np.abs(p - q)))


def noisy_vs_ideal(n: int, gate_list, p: float) -> Tuple[float, float]:
    """(F_cl, TVD) of the noisy circuit's distribution against the noiseless one."""
    pn = probs(run(n, gate_list, p))
    pi = probs(run(n, gate_list, 0.0))
    return classical_fidelity(pn, pi), tvd(pn, pi)


def vec(rho: np.ndarray) -> np.ndarray:
    """rho as the 2n-qubit vector v[r + 2^n c] = rho[r, c] (row bits low, column bits high)."""
    return np.ascontiguousarray(rho.T).reshape(-1)
