"""Pins of the density-matrix oracle (oracle/density.py): the paper's Table 8 values,
closed forms of the depolarizing channel, the noiseless limit, and the invariants of a
density matrix (trace, Hermiticity, positivity)."""
import os

import numpy as np
import pytest

import oracle
from oracle import density as D
from oracle import gates as OG
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _table8():
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "noise_table8.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, n, f_msle, f_cirq, t_msle, t_cirq = line.split()
            rows.append((name, int(n), float(f_msle), float(f_cirq), float(t_msle), float(t_cirq)))
    return rows


@pytest.mark.parametrize("row", _table8(), ids=lambda r: r[0])
def test_table8_noise_values(row):
    """Exact F_cl and TVD of the model against the printed, shot-averaged values: within
    0.006 (about three standard errors of an 8192-shot estimate)."""
    name, n, f_msle, f_cirq, t_msle, t_cirq = row
    specs = W.bell() if n == 2 else W.ghz(n)
    f, t = D.noisy_vs_ideal(n, OG.gate_list(specs), 0.01)
    assert abs(f - f_msle) <= 0.006 and abs(f - f_cirq) <= 0.006
    assert abs(t - t_msle) <= 0.006 and abs(t - t_cirq) <= 0.006


def test_single_qubit_channel_closed_forms():
    rho0 = D.pure(np.array([1, 0], dtype=np.complex128))
    for p in (0.0, 0.01, 0.3, 0.75):
        r = D.depolarize(rho0, 1, 0, p)
        assert np.allclose(r, np.diag([1 - 2 * p / 3, 2 * p / 3]), atol=1e-15)
    # p = 3/4 takes any one-qubit state to I / 2
    rng = np.random.default_rng(1)
    v = rng.normal(size=2) + 1j * rng.normal(size=2)
    v /= np.linalg.norm(v)
    assert np.allclose(D.depolarize(D.pure(v), 1, 0, 0.75), np.eye(2) / 2, atol=1e-15)
    # on one qubit of two, the other qubit is untouched: |+><+| (x) |0><0| -> |+><+| (x) diag
    plus = np.array([1, 1], dtype=np.complex128) / np.sqrt(2)
    r = D.depolarize(D.pure(np.kron(np.array([1, 0]), plus)), 2, 1, 0.3)
    want = np.kron(np.diag([1 - 0.2, 0.2]), D.pure(plus))
    assert np.allclose(r, want, atol=1e-15)


def test_noiseless_limit_is_the_pure_state():
    rng = np.random.default_rng(2)
    n = 5
    specs = W.random_unitary_gates(n, 12, 3, rng)
    rho = D.run(n, OG.gate_list(specs), 0.0)
    psi = oracle.simulate(n, specs)
    assert np.max(np.abs(rho - D.pure(psi))) < 1e-13


def test_density_matrix_invariants():
    rng = np.random.default_rng(3)
    n = 4
    specs = W.random_unitary_gates(n, 15, 2, rng)
    rho = D.run(n, OG.gate_list(specs), 0.07)
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.max(np.abs(rho - rho.conj().T)) < 1e-14
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-13
    # noise lowers the purity
    assert np.real(np.trace(rho @ rho)) < 1 - 1e-3
    p = D.probs(rho)
    assert D.classical_fidelity(p, p) == pytest.approx(1.0) and D.tvd(p, p) == 0.0


def test_vectorised_layout():
    rho = np.arange(16).reshape(4, 4).astype(np.complex128)
    v = D.vec(rho)
    for r in range(4):
        for c in range(4):
            assert v[r + 4 * c] == rho[r, c]
