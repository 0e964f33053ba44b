"""Oracle gate library (test infrastructure only; see oracle/__init__.py).

Matrices of the paper's canonical gate set G (Eq. 4) in complex128, written from the
definitions:

* R_a(theta) = exp(-i theta A / 2) for A in {X, Y, Z} (Eq. 4);
* U3 is "the general single-qubit gate with three Euler angles" (Eq. 4, no formula
  printed); read as the OpenQASM 2 form
  [[cos(t/2), -e^{i l} sin(t/2)], [e^{i p} sin(t/2), e^{i(p+l)} cos(t/2)]];
* gates outside G are full unitaries (Eq. 4): sqrt(P) = ((1+i) I + (1-i) P) / 2 for
  P in {X, Y, W = (X+Y)/sqrt2}; fSim(theta, phi); CP(phi) = diag(1, 1, 1, e^{i phi}).

Multi-qubit matrices use the convention of the gate record: matrix local bit j belongs
to qubits[j] (local index = sum_j bit(qubits[j]) 2^j).  CNOT(c, t) flips t when c = 1:
local index c + 2 t, so it swaps local states 1 and 3.  Toffoli(c1, c2, t) swaps local
states 3 and 7.
"""
from __future__ import annotations

import math

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
T = np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=np.complex128)
W = (X + Y) / math.sqrt(2.0)


def rot(pauli: np.ndarray, theta: float) -> np.ndarray:
    """exp(-i theta P / 2) = cos(theta/2) I - i sin(theta/2) P, valid because P^2 = I."""
    return math.cos(theta / 2) * I2 - 1j * math.sin(theta / 2) * pauli


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def sqrt_pauli(p: np.ndarray) -> np.ndarray:
    return ((1 + 1j) * I2 + (1 - 1j) * p) / 2


def perm_matrix(d: int, swaps) -> np.ndarray:
    m = np.eye(d, dtype=np.complex128)
    for a, b in swaps:
        m[[a, b]] = m[[b, a]]
    return m


def fsim(theta: float, phi: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)


def matrix(name: str, params=(), dagger: bool = False, explicit=None) -> np.ndarray:
    """Matrix of one gate record (name, params); adjoint when dagger."""
    p = tuple(params)
    if name == "i":
        m = I2.copy()
    elif name == "x":
        m = X.copy()
    elif name == "y":
        m = Y.copy()
    elif name == "z":
        m = Z.copy()
    elif name == "h":
        m = H.copy()
    elif name == "s":
        m = S.copy()
    elif name == "t":
        m = T.copy()
    elif name == "rx":
        m = rot(X, p[0])
    elif name == "ry":
        m = rot(Y, p[0])
    elif name == "rz":
        m = rot(Z, p[0])
    elif name == "u3":
        m = u3(p[0], p[1], p[2])
    elif name == "sqrtx":
        m = sqrt_pauli(X)
    elif name == "sqrty":
        m = sqrt_pauli(Y)
    elif name == "sqrtw":
        m = sqrt_pauli(W)
    elif name == "cnot":
        m = perm_matrix(4, [(1, 3)])
    elif name == "cz":
        m = np.diag([1, 1, 1, -1]).astype(np.complex128)
    elif name == "swap":
        m = perm_matrix(4, [(1, 2)])
    elif name == "cp":
        m = np.diag([1, 1, 1, np.exp(1j * p[0])]).astype(np.complex128)
    elif name == "fsim":
        m = fsim(p[0], p[1])
    elif name == "toffoli":
        m = perm_matrix(8, [(3, 7)])
    elif name == "unitary":
        e = np.asarray(explicit, dtype=np.complex128)
        d = int(round(math.sqrt(e.size)))
        m = e.reshape(d, d).copy()
    else:
        raise ValueError(f"unknown gate {name!r}")
    return m.conj().T.copy() if dagger else m


def gate_list(specs):
    """[(targets, U)] for a list of workloads.GateSpec records."""
    return [(tuple(g.qubits), matrix(g.name, g.params, g.dagger, g.matrix)) for g in specs]
