"""CPU oracle for the state-vector hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may
import, call, link or execute anything under oracle/.  The CUDA library never does, and
the oracle imports nothing from the library: the two share only the seeded input
generators in workloads/, which hold none of the method's arithmetic.

Contents (each function cites the passage it follows):

* sv_oracle.c  -- complex128 apply / norm / probabilities / Pauli expectation / inner
  product, plain loops (Eqs. 1-3, Eq. 10).
* gates.py     -- the canonical gate set G (Eq. 4) and the full-unitary gates.
* fusion.py    -- DAG construction and Algorithm 2 (Section 5.1-5.2, Eqs. 8-9).
* precision.py -- the a-priori precision rule (Eqs. 11-12).
* brute.py     -- Kronecker forms used to pin the loops at n <= 10 (Eq. 3).
* sampling.py  -- measurement sampling (the backend's third operation, Section 4.1): block
  prefix sums in a fixed order and SplitMix64 counters.
* density.py   -- density matrices with single-qubit depolarizing noise after every gate
  (Section 9.5, Table 8).
* structure.py -- control qubits and diagonal / monomial remainders of a gate matrix
  (the structure the paper's fusion leaves unused, Sections 10-11).

Parity status: apply, norm, probabilities, Pauli expectation, top-k, fusion and the
precision rule are all pinned by tests under tests/test_oracle_*.py (closed forms,
brute force, invariants and the paper's printed Eq. 12 value).  The fused gate counts
of the paper's Tables 4 and 7 are parity unpinned (their circuits are not specified).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Iterable, List, Sequence, Tuple

import numpy as np

from . import brute, density, fusion, gates, precision, sampling, structure  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sv_oracle.c with gcc (OpenMP) into oracle/_build/liborc.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.orc_apply.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp]
            lib.orc_apply.restype = ctypes.c_int
            lib.orc_norm.argtypes = [dp, ctypes.c_int]
            lib.orc_norm.restype = ctypes.c_double
            lib.orc_probs.argtypes = [dp, ctypes.c_int, dp]
            lib.orc_expect_pauli.argtypes = [dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                             dp, dp]
            lib.orc_inner.argtypes = [dp, dp, ctypes.c_int, dp, dp]
            lib.orc_set_basis.argtypes = [dp, ctypes.c_int, ctypes.c_uint64]
            lib.orc_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _nq(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and (1 << n) == psi.size
    return n


def num_threads() -> int:
    return _load().orc_num_threads()


def basis(n: int, x: int = 0) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().orc_set_basis(_dptr(psi.view(np.float64)), n, x)
    return psi


def apply_gate(psi: np.ndarray, targets: Sequence[int], u: np.ndarray) -> np.ndarray:
    """In place: one k-qubit gate, local bit j <-> targets[j] (Eq. 3)."""
    n = _nq(psi)
    k = len(targets)
    u = np.ascontiguousarray(np.asarray(u, dtype=np.complex128).reshape(1 << k, 1 << k))
    tg = (ctypes.c_int * k)(*targets)
    rc = _load().orc_apply(_dptr(psi.view(np.float64)), n, k, tg,
                           _dptr(u.view(np.float64)))
    if rc != 0:
        raise ValueError(f"bad gate targets {targets} for n={n}")
    return psi


def run(psi: np.ndarray, gate_list: Iterable[Tuple[Sequence[int], np.ndarray]]) -> np.ndarray:
    """In place: U_m ... U_1 |psi> (Eq. 10), one gate at a time, unfused."""
    for tg, u in gate_list:
        apply_gate(psi, tg, u)
    return psi


def simulate(n: int, specs, x: int = 0) -> np.ndarray:
    """|psi_out> for workloads.GateSpec records applied to |x>."""
    return run(basis(n, x), gates.gate_list(specs))


def norm(psi: np.ndarray) -> float:
    return _load().orc_norm(_dptr(psi.view(np.float64)), _nq(psi))


def probs(psi: np.ndarray) -> np.ndarray:
    p = np.empty(psi.size, dtype=np.float64)
    _load().orc_probs(_dptr(psi.view(np.float64)), _nq(psi), _dptr(p))
    return p


def expect_pauli(psi: np.ndarray, xmask: int, zmask: int) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().orc_expect_pauli(_dptr(psi.view(np.float64)), _nq(psi), xmask, zmask,
                             ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def expect(psi: np.ndarray, xs, zs, cs) -> float:
    """sum_t c_t <P_t> (real part; each Pauli string is Hermitian)."""
    return float(sum(c * expect_pauli(psi, x, z).real for x, z, c in zip(xs, zs, cs)))


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().orc_inner(_dptr(a.view(np.float64)), _dptr(b.view(np.float64)), _nq(a),
                      ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def fidelity(a: np.ndarray, b: np.ndarray) -> float:
    """|<a|b>|^2, the fidelity column of Table 3."""
    return abs(inner(a, b)) ** 2


def probs_in_precision(psi: np.ndarray) -> np.ndarray:
    """p_k = |alpha_k|^2 evaluated as fl(fl(re*re) + fl(im*im)) in the precision of psi
    (float32 for complex64).  Where a floating-point value decides an integer result
    (the top-k indices), the oracle takes that decision in the kernel's precision."""
    re, im = psi.real.copy(), psi.imag.copy()
    return re * re + im * im


def topk_valid(idx: np.ndarray, p_exact: np.ndarray, k: int, tol: float) -> bool:
    """True if idx (distinct indices) is a correct top-k of p_exact up to ties within
    tol: the j-th listed outcome has probability within tol of the j-th largest."""
    if len(set(int(i) for i in idx)) != len(idx):
        return False
    best = np.sort(p_exact)[::-1][: min(k, p_exact.size)]
    got = p_exact[np.asarray(idx, dtype=np.int64)]
    return len(idx) == best.size and bool(np.all(np.abs(got - best) <= tol))


def topk(p: np.ndarray, k: int) -> Tuple[np.ndarray, np.ndarray]:
    """The k largest probabilities, ties to the lower index (a stable sort on -p)."""
    order = np.argsort(-p, kind="stable")[:k]
    return order.astype(np.uint64), p[order]


def zz_chain_weight(n: int, k: np.ndarray) -> np.ndarray:
    """sum_{i<n-1} (-1)^{b_i(k) + b_{i+1}(k)} = (n-1) - 2 popcount((k ^ (k >> 1)) & (2^{n-1}-1))."""
    m = (k ^ (k >> 1)) & ((1 << (n - 1)) - 1)
    pc = np.zeros_like(m)
    for b in range(n - 1):
        pc += (m >> b) & 1
    return (n - 1) - 2 * pc


def fuse(gate_list, n: int, qmax: int, commute: bool = False):
    """Algorithm 2 (see oracle/fusion.py)."""
    return fusion.fuse(gate_list, n, qmax, commute)
