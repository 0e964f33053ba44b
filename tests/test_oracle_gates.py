"""Pins for the oracle's gate library (Eq. 4) against textbook identities and scipy."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import brute
from oracle import gates as G

NAMES_1Q = ["i", "x", "y", "z", "h", "s", "t", "sqrtx", "sqrty", "sqrtw"]
NAMES_2Q = ["cnot", "cz", "swap"]


def _all_matrices():
    out = [(n, G.matrix(n)) for n in NAMES_1Q + NAMES_2Q + ["toffoli"]]
    rng = np.random.default_rng(5)
    for _ in range(5):
        a, b, c = rng.uniform(-7, 7, size=3)
        out += [("rx", G.matrix("rx", (a,))), ("ry", G.matrix("ry", (a,))),
                ("rz", G.matrix("rz", (a,))), ("u3", G.matrix("u3", (a, b, c))),
                ("cp", G.matrix("cp", (a,))), ("fsim", G.matrix("fsim", (a, b)))]
    return out


@pytest.mark.parametrize("name,m", _all_matrices())
def test_unitary(name, m):
    assert np.allclose(m @ m.conj().T, np.eye(m.shape[0]), atol=1e-14)


@pytest.mark.parametrize("theta", [0.0, 0.3, -1.7, math.pi, 5.9])
def test_rotations_are_matrix_exponentials(theta):
    # Eq. 4: R_a(theta) = exp(-i theta A / 2); checked with scipy's expm.
    for name, p in (("rx", G.X), ("ry", G.Y), ("rz", G.Z)):
        want = scipy.linalg.expm(-1j * theta * p / 2)
        assert np.allclose(G.matrix(name, (theta,)), want, atol=1e-14)


def test_sqrt_gates_square_to_pauli():
    for name, p in (("sqrtx", G.X), ("sqrty", G.Y), ("sqrtw", G.W)):
        r = G.matrix(name)
        assert np.allclose(r @ r, p, atol=1e-15)
        assert np.allclose(scipy.linalg.sqrtm(p) @ scipy.linalg.sqrtm(p), p)


def test_u3_special_cases():
    # OpenQASM 2 reading of U3: known reductions fix the sign and phase conventions.
    assert np.allclose(G.u3(math.pi / 2, 0, math.pi), G.H, atol=1e-15)
    th = 0.77
    assert np.allclose(G.u3(th, -math.pi / 2, math.pi / 2), G.matrix("rx", (th,)), atol=1e-15)
    assert np.allclose(G.u3(th, 0, 0), G.matrix("ry", (th,)), atol=1e-15)
    assert np.allclose(G.u3(0, 0, math.pi / 2), G.S, atol=1e-15)
    assert np.allclose(G.u3(0, 0, math.pi / 4), G.T, atol=1e-15)
    assert np.allclose(G.u3(math.pi, 0, math.pi), G.X, atol=1e-15)


def test_two_qubit_conventions_on_basis_states():
    # local bit j <-> qubits[j]; CNOT(c=qubit0, t=qubit1) maps |c=1,t=0> = index 1 to 3.
    cn = brute.full_operator(2, (0, 1), G.matrix("cnot"))
    assert np.allclose(cn[:, 1], np.eye(4)[3])
    assert np.allclose(cn[:, 0], np.eye(4)[0])
    # swapped roles: control qubit 1, target qubit 0 maps index 2 to 3
    cn10 = brute.full_operator(2, (1, 0), G.matrix("cnot"))
    assert np.allclose(cn10[:, 2], np.eye(4)[3])
    # Toffoli flips the third qubit only when both controls are set
    tf = brute.full_operator(3, (0, 1, 2), G.matrix("toffoli"))
    assert np.allclose(tf[:, 3], np.eye(8)[7]) and np.allclose(tf[:, 1], np.eye(8)[1])
    # SWAP exchanges the two qubits
    sw = brute.full_operator(2, (0, 1), G.matrix("swap"))
    assert np.allclose(sw[:, 1], np.eye(4)[2])
    # CZ is the controlled Z; CP(pi) = CZ
    assert np.allclose(G.matrix("cp", (math.pi,)), G.matrix("cz"), atol=1e-15)


def test_fsim_structure():
    # fSim(theta, 0) acts as exp(-i theta X) on span{|01>, |10>} and as I elsewhere.
    th = 0.6
    f = G.fsim(th, 0.0)
    assert np.allclose(f[1:3, 1:3], scipy.linalg.expm(-1j * th * G.X))
    assert f[0, 0] == 1 and f[3, 3] == 1
    # the phi part is a controlled phase e^{-i phi} on |11>
    assert np.allclose(G.fsim(0.0, 0.4), np.diag([1, 1, 1, np.exp(-0.4j)]))


def test_dagger_is_inverse():
    rng = np.random.default_rng(1)
    a, b, c = rng.uniform(0, 6, size=3)
    for name, p in (("u3", (a, b, c)), ("fsim", (a, b)), ("sqrtw", ()), ("t", ())):
        m = G.matrix(name, p)
        md = G.matrix(name, p, dagger=True)
        assert np.allclose(md @ m, np.eye(m.shape[0]), atol=1e-14)
