"""Thin Python binding of the C ABI in include/sv.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Device memory and streams
may come from PyTorch (a CUDA tensor's data_ptr and torch.cuda.current_stream()); all
computation happens in libsvgb300.so.  Importing this module fails loudly when the
library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsvgb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

SV_C64, SV_C128 = 0, 1
SV_MAX_K = 5
STATUS = {0: "SV_OK", 1: "SV_ERR_ARG", 2: "SV_ERR_OOM", 3: "SV_ERR_CUDA", 4: "SV_ERR_TIMEOUT",
          5: "SV_ERR_STATE"}
GATE_KINDS = {"i": 0, "x": 1, "y": 2, "z": 3, "h": 4, "s": 5, "t": 6, "rx": 7, "ry": 8, "rz": 9,
              "cnot": 10, "cz": 11, "swap": 12, "toffoli": 13, "u3": 14, "sqrtx": 15,
              "sqrty": 16, "sqrtw": 17, "fsim": 18, "cp": 19, "unitary": 20}

EXPORTS = ["sv_gate_matrix", "sv_alloc", "sv_free", "sv_info", "sv_set_basis", "sv_set_dtype",
           "sv_set_state",
           "sv_get_state", "sv_fuse", "sv_circuit_free", "sv_circuit_size", "sv_circuit_gate",
           "sv_choose_dtype", "sv_apply_circuit", "sv_apply_gate", "sv_norm", "sv_probs",
           "sv_expect", "sv_topk", "sv_sync", "sv_last_error", "sv_set_policy",
           "sv_expect_noalloc", "sv_plan_passes"]
EXPORTS += ["sv_fuse_like", "sv_sample", "sv_fuse_density", "sv_density_probs", "sv_gate_structure",
            "sv_fuse_ex", "sv_debug_fail_allocs", "sv_set_zero", "sv_shard_plan_create",
            "sv_shard_plan_free", "sv_shard_plan_info", "sv_shard_plan_step", "sv_shard_pack",
            "sv_shard_unpack"]
EXPORTS += ["sv_server_create", "sv_server_submit", "sv_server_poll", "sv_server_get_stats",
            "sv_server_destroy"]
EXPORTS += ["sv_batch_alloc", "sv_batch_free", "sv_batch_set_basis", "sv_batch_get_state",
            "sv_batch_apply", "sv_batch_expect", "sv_batch_sync", "sv_batch_tune"]
SV_POLICY_NO_TENSOR_CORES = 1
SV_POLICY_DENSE_ONLY = 2
SV_POLICY_STAGED_PROBS = 4
SV_POLICY_TWO_GATE_PASSES = 8
SV_FUSE_COMMUTE = 1
SV_STRUCT_DENSE, SV_STRUCT_DIAGONAL, SV_STRUCT_MONOMIAL, SV_STRUCT_IDENTITY = 0, 1, 2, 3
SV_SHARD_APPLY, SV_SHARD_SWAP = 0, 1


class SvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class sv_gate(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("targets", ctypes.c_uint32 * SV_MAX_K),
                ("u", ctypes.POINTER(ctypes.c_double))]


class sv_apply_opts(ctypes.Structure):
    _fields_ = [("adaptive", ctypes.c_uint32), ("drift_threshold", ctypes.c_double),
                ("drift_check_every", ctypes.c_uint32), ("timing", ctypes.c_uint32)]


class sv_apply_report(ctypes.Structure):
    _fields_ = [("dtype_used", ctypes.c_int32), ("promotions", ctypes.c_uint32),
                ("passes", ctypes.c_uint64), ("norm_before", ctypes.c_double),
                ("norm_after", ctypes.c_double), ("drift", ctypes.c_double),
                ("bytes", ctypes.c_uint64), ("apply_ms", ctypes.c_double),
                ("tc_passes", ctypes.c_uint64), ("max_k_used", ctypes.c_uint32),
                ("paired_passes", ctypes.c_uint64)]


class sv_batch_opts(ctypes.Structure):
    _fields_ = [("chunk_states", ctypes.c_uint32), ("l2_bytes", ctypes.c_size_t),
                ("no_graph", ctypes.c_uint32), ("timing", ctypes.c_uint32),
                ("no_tensor_cores", ctypes.c_uint32), ("tile_bits", ctypes.c_uint32)]


class sv_batch_report(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("bytes", ctypes.c_uint64), ("chunk_states", ctypes.c_uint32),
                ("graph_reused", ctypes.c_uint32), ("apply_ms", ctypes.c_double),
                ("tile_bits", ctypes.c_uint32)]


class sv_tune_result(ctypes.Structure):
    _fields_ = [("best_k", ctypes.c_uint32), ("l2_bytes", ctypes.c_size_t),
                ("best_ms", ctypes.c_double), ("ms", ctypes.c_double * (SV_MAX_K + 1)),
                ("cached", ctypes.c_uint32), ("tile_bits", ctypes.c_uint32)]


class sv_server_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_uint32),
                ("topk", ctypes.c_uint32), ("max_k", ctypes.c_uint32),
                ("fuse_threads", ctypes.c_uint32)]


class sv_server_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("dtype_used", ctypes.c_int32),
                ("n", ctypes.c_uint32), ("k", ctypes.c_uint32), ("passes", ctypes.c_uint64),
                ("idx", ctypes.c_uint64 * 64), ("p", ctypes.c_double * 64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class sv_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("queued", ctypes.c_uint64), ("active", ctypes.c_uint32),
                ("in_use_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("now", ctypes.c_double)]


_vp = ctypes.c_void_p
_u32, _u64, _i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)
_sig = {
    "sv_gate_matrix": [_u32, _dp, _u32, _i32, _dp, ctypes.POINTER(_u32)],
    "sv_alloc": [_u32, _i32, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)],
    "sv_free": [_vp],
    "sv_info": [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_i32), ctypes.POINTER(_vp)],
    "sv_set_basis": [_vp, _u64],
    "sv_set_dtype": [_vp, _i32],
    "sv_set_state": [_vp, _vp, _i32],
    "sv_get_state": [_vp, _vp, _i32],
    "sv_fuse": [ctypes.POINTER(sv_gate), ctypes.c_size_t, _u32, _u32, ctypes.POINTER(_vp)],
    "sv_fuse_ex": [ctypes.POINTER(sv_gate), ctypes.c_size_t, _u32, _u32, _u32, ctypes.POINTER(_vp)],
    "sv_fuse_density": [ctypes.POINTER(sv_gate), ctypes.c_size_t, _u32, ctypes.c_double, _u32,
                        ctypes.POINTER(_vp)],
    "sv_circuit_free": [_vp],
    "sv_fuse_like": [_vp, ctypes.POINTER(sv_gate), ctypes.c_size_t, ctypes.POINTER(_vp)],
    "sv_circuit_size": [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_u32)],
    "sv_circuit_gate": [_vp, ctypes.c_size_t, ctypes.POINTER(_u32), ctypes.POINTER(_u32), _dp],
    "sv_choose_dtype": [_u32, _u64, ctypes.c_double, ctypes.POINTER(_i32), _dp],
    "sv_apply_circuit": [_vp, _vp, ctypes.POINTER(sv_apply_opts), ctypes.POINTER(sv_apply_report)],
    "sv_apply_gate": [_vp, ctypes.POINTER(sv_gate)],
    "sv_gate_structure": [ctypes.POINTER(sv_gate), ctypes.POINTER(_u32), ctypes.POINTER(_u32)],
    "sv_norm": [_vp, _dp],
    "sv_probs": [_vp, _vp, _i32],
    "sv_expect": [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), _dp, ctypes.c_size_t, _dp],
    "sv_topk": [_vp, _u32, ctypes.POINTER(_u64), _dp],
    "sv_sample": [_vp, _u64, ctypes.c_size_t, ctypes.POINTER(_u64), ctypes.c_int],
    "sv_density_probs": [_vp, _vp, ctypes.c_int],
    "sv_sync": [_vp],
    "sv_set_policy": [_vp, _u32],
    "sv_debug_fail_allocs": [_u32],
    "sv_set_zero": [_vp],
    "sv_shard_plan_create": [_vp, _u32, _i32, ctypes.POINTER(_vp)],
    "sv_shard_plan_free": [_vp],
    "sv_shard_plan_info": [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_u64),
                           ctypes.POINTER(_u64)],
    "sv_shard_plan_step": [_vp, ctypes.c_size_t, ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                           ctypes.POINTER(_u32), ctypes.POINTER(_vp)],
    "sv_shard_pack": [_vp, _u32, _u32, _u64, _u64, _vp],
    "sv_shard_unpack": [_vp, _u32, _u32, _u64, _u64, _vp],
    "sv_server_create": [ctypes.POINTER(sv_server_config), ctypes.POINTER(_vp)],
    "sv_server_submit": [_vp, _u32, _i32, ctypes.POINTER(sv_gate), ctypes.c_size_t,
                         ctypes.POINTER(_u64)],
    "sv_server_poll": [_vp, ctypes.POINTER(sv_server_result), ctypes.c_size_t,
                       ctypes.POINTER(ctypes.c_size_t), _i32],
    "sv_server_get_stats": [_vp, ctypes.POINTER(sv_server_stats)],
    "sv_server_destroy": [_vp],
    "sv_batch_alloc": [_u32, _i32, _u32, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)],
    "sv_batch_free": [_vp],
    "sv_batch_set_basis": [_vp, _u64],
    "sv_batch_get_state": [_vp, _u32, _vp, _i32],
    "sv_batch_apply": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(sv_batch_opts),
                       ctypes.POINTER(sv_batch_report)],
    "sv_batch_expect": [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), _dp, ctypes.c_size_t, _dp],
    "sv_batch_sync": [_vp],
    "sv_batch_tune": [_vp, ctypes.POINTER(sv_gate), ctypes.c_size_t, _u32, _u32,
                      ctypes.POINTER(sv_tune_result)],
    "sv_plan_passes": [_vp, _u32, ctypes.POINTER(_u32), ctypes.POINTER(ctypes.c_int32), ctypes.c_size_t,
                       ctypes.POINTER(ctypes.c_size_t)],
    "sv_expect_noalloc": [_vp, _u32, _i32, ctypes.POINTER(_u64), ctypes.POINTER(_u64), _dp,
                          ctypes.c_size_t, _vp, _vp],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.sv_last_error.restype = ctypes.c_char_p
_lib.sv_last_error.argtypes = []


def sv_last_error() -> str:
    return _lib.sv_last_error().decode()


def _check(st: int) -> None:
    if st != 0:
        raise SvError(st, sv_last_error())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


# --------------------------------------------------------------------------- gates

def sv_gate_matrix(name: str, params: Sequence[float] = (), dagger: bool = False,
                   matrix=None) -> np.ndarray:
    """Matrix (complex128, 2^k x 2^k) of a gate of the canonical set, built by the library."""
    kind = GATE_KINDS[name]
    if name == "unitary":
        m = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128).ravel())
        p = m.view(np.float64)
    else:
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    out = np.zeros(2 * 1024, dtype=np.float64)
    k = _u32()
    _check(_lib.sv_gate_matrix(kind, _ptr(p) if p.size else None, p.size, int(bool(dagger)),
                               _ptr(out), ctypes.byref(k)))
    d = 1 << k.value
    return out[: 2 * d * d].view(np.complex128).reshape(d, d).copy()


class GateArray:
    """A ctypes array of sv_gate plus the matrices it points to (kept alive)."""

    def __init__(self, gates: Sequence[Tuple[Sequence[int], np.ndarray]]):
        self.mats = [np.ascontiguousarray(np.asarray(u, dtype=np.complex128)) for _, u in gates]
        self.arr = (sv_gate * max(1, len(gates)))()
        for i, ((tg, _), m) in enumerate(zip(gates, self.mats)):
            self.arr[i].k = len(tg)
            for j, t in enumerate(tg[:SV_MAX_K]):     # k > 5 is rejected by the library
                self.arr[i].targets[j] = int(t)
            self.arr[i].u = m.view(np.float64).ctypes.data_as(_dp)
        self.n = len(gates)


def gates_from_specs(specs) -> List[Tuple[Tuple[int, ...], np.ndarray]]:
    """[(targets, U)] for workloads.GateSpec records, matrices from the library."""
    return [(tuple(g.qubits), sv_gate_matrix(g.name, g.params, g.dagger, g.matrix)) for g in specs]


# --------------------------------------------------------------------------- circuits

class Circuit:
    """An sv_circuit handle; owned=False for circuits owned by another object (a shard
    plan's segments), which are not freed here."""

    def __init__(self, handle: int, owned: bool = True, keep=None):
        self.handle = handle
        self.owned = owned
        self.keep = keep

    def __del__(self):
        if getattr(self, "handle", None) and getattr(self, "owned", True):
            _lib.sv_circuit_free(self.handle)
        self.handle = None

    def __len__(self) -> int:
        return sv_circuit_size(self)[0]


def sv_fuse(gates, n: int, max_k: int) -> Circuit:
    """gates: [(targets, U)] or a prebuilt GateArray."""
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    h = _vp()
    _check(_lib.sv_fuse(ga.arr, ga.n, n, max_k, ctypes.byref(h)))
    return Circuit(h.value)


def sv_fuse_ex(gates, n: int, max_k: int, flags: int = 0) -> Circuit:
    """sv_fuse with SV_FUSE_* flags (SV_FUSE_COMMUTE: commutation-aware fusion)."""
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    h = _vp()
    _check(_lib.sv_fuse_ex(ga.arr, ga.n, n, max_k, flags, ctypes.byref(h)))
    return Circuit(h.value)


def sv_fuse_density(gates, n: int, p: float, max_k: int) -> Circuit:
    """The noisy circuit on the vectorised density matrix (2n qubits), fused."""
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    h = _vp()
    _check(_lib.sv_fuse_density(ga.arr, ga.n, n, p, max_k, ctypes.byref(h)))
    return Circuit(h.value)


def sv_density_probs(s: State, out=None):
    """Re rho[x, x] (float32 for C64, float64 for C128) of a vectorised density matrix."""
    n2, dt, _ = sv_info(s)
    if out is not None and hasattr(out, "data_ptr"):
        _check(_lib.sv_density_probs(s.handle, int(out.data_ptr()), 1 if out.is_cuda else 0))
        return out
    a = out if out is not None else np.empty(1 << (n2 // 2), dtype=np.float32 if dt == SV_C64 else np.float64)
    _check(_lib.sv_density_probs(s.handle, a.ctypes.data, 0))
    return a


def sv_fuse_like(pattern: Circuit, gates) -> Circuit:
    """gates: [(targets, U)] or a prebuilt GateArray, same qubits as the pattern's input."""
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    h = _vp()
    _check(_lib.sv_fuse_like(pattern.handle, ga.arr, ga.n, ctypes.byref(h)))
    return Circuit(h.value)


def sv_circuit_size(c: Circuit) -> Tuple[int, int]:
    nf, n = ctypes.c_size_t(), _u32()
    _check(_lib.sv_circuit_size(c.handle, ctypes.byref(nf), ctypes.byref(n)))
    return nf.value, n.value


def sv_circuit_gate(c: Circuit, i: int) -> Tuple[Tuple[int, ...], np.ndarray]:
    k = _u32()
    tg = (_u32 * SV_MAX_K)()
    _check(_lib.sv_circuit_gate(c.handle, i, ctypes.byref(k), tg, None))
    d = 1 << k.value
    u = np.zeros(2 * d * d, dtype=np.float64)
    _check(_lib.sv_circuit_gate(c.handle, i, ctypes.byref(k), tg, _ptr(u)))
    return tuple(int(tg[j]) for j in range(k.value)), u.view(np.complex128).reshape(d, d)


def sv_plan_passes(c: Circuit, policy: int = SV_POLICY_TWO_GATE_PASSES) -> List[Tuple[int, int]]:
    """The passes of the circuit on a complex64 state with these policy flags:
    [(first, second or -1)]."""
    nf, _ = sv_circuit_size(c)
    first = (_u32 * max(nf, 1))()
    second = (ctypes.c_int32 * max(nf, 1))()
    np_ = ctypes.c_size_t()
    _check(_lib.sv_plan_passes(c.handle, policy, first, second, max(nf, 1), ctypes.byref(np_)))
    return [(int(first[i]), int(second[i])) for i in range(np_.value)]


def sv_choose_dtype(n: int, g: int, eps_tol: float) -> Tuple[int, float]:
    out, e = _i32(), ctypes.c_double()
    _check(_lib.sv_choose_dtype(n, g, eps_tol, ctypes.byref(out), ctypes.byref(e)))
    return out.value, e.value


# --------------------------------------------------------------------------- states

class State:
    """An sv_state handle.  `keep` holds the caller buffer (e.g. a torch tensor) alive."""

    def __init__(self, handle: int, keep=None):
        self.handle = handle
        self.keep = keep

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.sv_free(self.handle)
            self.handle = None

    def free(self):
        if self.handle:
            _check(_lib.sv_free(self.handle))
            self.handle = None

    @property
    def info(self):
        return sv_info(self)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


def sv_alloc(n: int, dtype: int = SV_C64, dev_buf=None, nbytes: int = 0, stream=None) -> State:
    """dev_buf: None (library-owned), a CUDA torch tensor, or a raw device pointer."""
    keep, ptr = None, None
    if dev_buf is not None:
        if hasattr(dev_buf, "data_ptr"):
            keep, ptr = dev_buf, int(dev_buf.data_ptr())
            nbytes = nbytes or int(dev_buf.numel() * dev_buf.element_size())
        else:
            ptr = int(dev_buf)
    h = _vp()
    _check(_lib.sv_alloc(n, dtype, ptr, nbytes, _stream_ptr(stream), ctypes.byref(h)))
    return State(h.value, keep)


def sv_free(s: State) -> None:
    s.free()


def sv_info(s: State) -> Tuple[int, int, int]:
    n, dt, p = _u32(), _i32(), _vp()
    _check(_lib.sv_info(s.handle, ctypes.byref(n), ctypes.byref(dt), ctypes.byref(p)))
    return n.value, dt.value, p.value


def sv_set_basis(s: State, x: int) -> None:
    _check(_lib.sv_set_basis(s.handle, x))


def sv_set_dtype(s: State, dtype: int) -> None:
    _check(_lib.sv_set_dtype(s.handle, dtype))


def _np_dtype(dt: int):
    return np.complex64 if dt == SV_C64 else np.complex128


def sv_set_state(s: State, src) -> None:
    """src: numpy array (host) or CUDA torch tensor (device), in the state's dtype."""
    if hasattr(src, "data_ptr"):
        _check(_lib.sv_set_state(s.handle, int(src.data_ptr()), 1))
        return
    n, dt, _ = sv_info(s)
    a = np.ascontiguousarray(src, dtype=_np_dtype(dt))
    assert a.size == 1 << n
    _check(_lib.sv_set_state(s.handle, a.ctypes.data, 0))


def sv_get_state(s: State, out=None):
    """Host numpy copy (default) or into a CUDA torch tensor `out` (asynchronous)."""
    if out is not None and hasattr(out, "data_ptr"):
        _check(_lib.sv_get_state(s.handle, int(out.data_ptr()), 1))
        return out
    n, dt, _ = sv_info(s)
    a = out if out is not None else np.empty(1 << n, dtype=_np_dtype(dt))
    _check(_lib.sv_get_state(s.handle, a.ctypes.data, 0))
    return a


def sv_apply_circuit(s: State, c: Circuit, adaptive: bool = False, drift_threshold: float = 1e-6,
                     drift_check_every: int = 0, timing: bool = False) -> dict:
    opts = sv_apply_opts(int(bool(adaptive)), drift_threshold, drift_check_every,
                         int(bool(timing)))
    rep = sv_apply_report()
    _check(_lib.sv_apply_circuit(s.handle, c.handle, ctypes.byref(opts), ctypes.byref(rep)))
    return {"dtype_used": rep.dtype_used, "promotions": rep.promotions, "passes": rep.passes,
            "norm_before": rep.norm_before, "norm_after": rep.norm_after, "drift": rep.drift,
            "bytes": rep.bytes, "apply_ms": rep.apply_ms, "tc_passes": rep.tc_passes,
            "max_k_used": rep.max_k_used, "paired_passes": rep.paired_passes}


def sv_apply_gate(s: State, targets: Sequence[int], u: np.ndarray) -> None:
    ga = GateArray([(targets, u)])
    _check(_lib.sv_apply_gate(s.handle, ga.arr))


def sv_gate_structure(targets: Sequence[int], u: np.ndarray) -> Tuple[int, int]:
    """(SV_STRUCT_* kind of the reduced gate, control mask over the caller's targets)."""
    ga = GateArray([(targets, u)])
    kind, mask = _u32(), _u32()
    _check(_lib.sv_gate_structure(ga.arr, ctypes.byref(kind), ctypes.byref(mask)))
    return kind.value, mask.value


def sv_norm(s: State) -> float:
    out = ctypes.c_double()
    _check(_lib.sv_norm(s.handle, ctypes.byref(out)))
    return out.value


def sv_probs(s: State, out=None):
    """Host numpy array (float32 for C64, float64 for C128), or into a tensor (a CUDA
    tensor is written asynchronously; a CPU tensor, pinned or not, is host memory)."""
    if out is not None and hasattr(out, "data_ptr"):
        _check(_lib.sv_probs(s.handle, int(out.data_ptr()), 1 if out.is_cuda else 0))
        return out
    n, dt, _ = sv_info(s)
    a = out if out is not None else np.empty(1 << n, dtype=np.float32 if dt == SV_C64 else np.float64)
    _check(_lib.sv_probs(s.handle, a.ctypes.data, 0))
    return a


def sv_expect(s: State, xmask: Iterable[int], zmask: Iterable[int], coef: Iterable[float]) -> float:
    x = np.ascontiguousarray(np.asarray(list(xmask), dtype=np.uint64))
    z = np.ascontiguousarray(np.asarray(list(zmask), dtype=np.uint64))
    c = np.ascontiguousarray(np.asarray(list(coef), dtype=np.float64))
    assert x.size == z.size == c.size
    out = ctypes.c_double()
    u64p = ctypes.POINTER(_u64)
    _check(_lib.sv_expect(s.handle, x.ctypes.data_as(u64p), z.ctypes.data_as(u64p), _ptr(c),
                          x.size, ctypes.byref(out)))
    return out.value


def sv_expect_noalloc(psi, n: int, dtype: int, xmask: Iterable[int], zmask: Iterable[int],
                      coef: Iterable[float], out, stream=None) -> None:
    """psi: CUDA tensor (or device pointer) holding the state; out: CUDA float64 tensor
    (or device pointer) receiving sum_t c_t <P_t>.  Asynchronous; allocates nothing."""
    x = np.ascontiguousarray(np.asarray(list(xmask), dtype=np.uint64))
    z = np.ascontiguousarray(np.asarray(list(zmask), dtype=np.uint64))
    c = np.ascontiguousarray(np.asarray(list(coef), dtype=np.float64))
    assert x.size == z.size == c.size
    pp = int(psi.data_ptr()) if hasattr(psi, "data_ptr") else int(psi)
    op = int(out.data_ptr()) if hasattr(out, "data_ptr") else int(out)
    u64p = ctypes.POINTER(_u64)
    _check(_lib.sv_expect_noalloc(pp, n, dtype, x.ctypes.data_as(u64p), z.ctypes.data_as(u64p),
                                  _ptr(c), x.size, op, _stream_ptr(stream)))


def sv_topk(s: State, k: int = 64) -> Tuple[np.ndarray, np.ndarray]:
    n, _, _ = sv_info(s)
    m = min(k, 1 << n)
    idx = np.zeros(k, dtype=np.uint64)
    p = np.zeros(k, dtype=np.float64)
    _check(_lib.sv_topk(s.handle, k, idx.ctypes.data_as(ctypes.POINTER(_u64)), _ptr(p)))
    return idx[:m], p[:m]


def sv_sample(s: State, seed: int, nshots: int, out=None) -> np.ndarray:
    """nshots sampled outcome indices (uint64); into a CUDA tensor if given one."""
    if out is not None and hasattr(out, "data_ptr") and out.is_cuda:
        _check(_lib.sv_sample(s.handle, seed & ((1 << 64) - 1), nshots,
                              ctypes.cast(int(out.data_ptr()), ctypes.POINTER(_u64)), 1))
        return out
    a = np.empty(nshots, dtype=np.uint64)
    _check(_lib.sv_sample(s.handle, seed & ((1 << 64) - 1), nshots,
                          a.ctypes.data_as(ctypes.POINTER(_u64)), 0))
    return a


def sv_set_policy(s: State, flags: int) -> None:
    _check(_lib.sv_set_policy(s.handle, flags))


def sv_sync(s: State) -> None:
    _check(_lib.sv_sync(s.handle))


def sv_debug_fail_allocs(count: int) -> None:
    _check(_lib.sv_debug_fail_allocs(count))


def sv_set_zero(s: State) -> None:
    _check(_lib.sv_set_zero(s.handle))


# --------------------------------------------------------------------------- sharding

class ShardPlan:
    """An sv_shard_plan handle: the steps every rank of a sharded state runs."""

    def __init__(self, handle: int, circuit: Circuit):
        self.handle = handle
        self.circuit = circuit          # the plan reads nothing from it later; kept for clarity

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.sv_shard_plan_free(self.handle)
            self.handle = None

    def info(self) -> Tuple[int, int, int]:
        """(steps, exchanges, SWAP passes)."""
        ns, ex, ls = ctypes.c_size_t(), _u64(), _u64()
        _check(_lib.sv_shard_plan_info(self.handle, ctypes.byref(ns), ctypes.byref(ex), ctypes.byref(ls)))
        return ns.value, ex.value, ls.value

    def steps(self):
        """[(kind, local_bit, global_bit, segment Circuit or None)]."""
        out = []
        for i in range(self.info()[0]):
            kind, lb, gb, seg = _u32(), _u32(), _u32(), _vp()
            _check(_lib.sv_shard_plan_step(self.handle, i, ctypes.byref(kind), ctypes.byref(lb),
                                           ctypes.byref(gb), ctypes.byref(seg)))
            c = Circuit(seg.value, owned=False, keep=self) if kind.value == SV_SHARD_APPLY else None
            out.append((kind.value, lb.value, gb.value, c))
        return out


def sv_shard_plan_create(c: Circuit, g: int, dtype: int) -> ShardPlan:
    h = _vp()
    _check(_lib.sv_shard_plan_create(c.handle, g, dtype, ctypes.byref(h)))
    return ShardPlan(h.value, c)


def sv_shard_pack(s: State, bit: int, value: int, offset: int, count: int, dst) -> None:
    """dst: CUDA tensor (or device pointer) of at least count amplitudes."""
    p = int(dst.data_ptr()) if hasattr(dst, "data_ptr") else int(dst)
    _check(_lib.sv_shard_pack(s.handle, bit, value, offset, count, p))


def sv_shard_unpack(s: State, bit: int, value: int, offset: int, count: int, src) -> None:
    p = int(src.data_ptr()) if hasattr(src, "data_ptr") else int(src)
    _check(_lib.sv_shard_unpack(s.handle, bit, value, offset, count, p))


# --------------------------------------------------------------------------- batches

class Batch:
    def __init__(self, handle: int, n: int, dtype: int, count: int, keep=None):
        self.handle, self.n, self.dtype, self.count, self.keep = handle, n, dtype, count, keep

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.sv_batch_free(self.handle)
            self.handle = None

    def free(self):
        if self.handle:
            _check(_lib.sv_batch_free(self.handle))
            self.handle = None


def sv_batch_alloc(n: int, dtype: int, count: int, dev_buf=None, nbytes: int = 0,
                   stream=None) -> Batch:
    keep, ptr = None, None
    if dev_buf is not None:
        keep, ptr = dev_buf, int(dev_buf.data_ptr())
        nbytes = nbytes or int(dev_buf.numel() * dev_buf.element_size())
    h = _vp()
    _check(_lib.sv_batch_alloc(n, dtype, count, ptr, nbytes, _stream_ptr(stream), ctypes.byref(h)))
    return Batch(h.value, n, dtype, count, keep)


def sv_batch_free(b: Batch) -> None:
    b.free()


def sv_batch_set_basis(b: Batch, x: int) -> None:
    _check(_lib.sv_batch_set_basis(b.handle, x))


def sv_batch_get_state(b: Batch, i: int) -> np.ndarray:
    a = np.empty(1 << b.n, dtype=_np_dtype(b.dtype))
    _check(_lib.sv_batch_get_state(b.handle, i, a.ctypes.data, 0))
    return a


def sv_batch_apply(b: Batch, circuits: Sequence[Circuit], chunk_states: int = 0,
                   l2_bytes: int = 0, no_graph: bool = False, timing: bool = False,
                   no_tensor_cores: bool = False, tile_bits: int = 0) -> dict:
    arr = (_vp * len(circuits))(*[c.handle for c in circuits])
    assert len(circuits) == b.count
    opts = sv_batch_opts(chunk_states, l2_bytes, int(bool(no_graph)), int(bool(timing)),
                         int(bool(no_tensor_cores)), tile_bits)
    rep = sv_batch_report()
    _check(_lib.sv_batch_apply(b.handle, arr, ctypes.byref(opts), ctypes.byref(rep)))
    return {"passes": rep.passes, "launches": rep.launches, "bytes": rep.bytes,
            "chunk_states": rep.chunk_states, "graph_reused": rep.graph_reused,
            "apply_ms": rep.apply_ms, "tile_bits": rep.tile_bits}


def sv_batch_expect(b: Batch, xmask, zmask, coef) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(list(xmask), dtype=np.uint64))
    z = np.ascontiguousarray(np.asarray(list(zmask), dtype=np.uint64))
    c = np.ascontiguousarray(np.asarray(list(coef), dtype=np.float64))
    out = np.zeros(b.count, dtype=np.float64)
    u64p = ctypes.POINTER(_u64)
    _check(_lib.sv_batch_expect(b.handle, x.ctypes.data_as(u64p), z.ctypes.data_as(u64p), _ptr(c),
                                x.size, _ptr(out)))
    return out


def sv_batch_sync(b: Batch) -> None:
    _check(_lib.sv_batch_sync(b.handle))


def sv_batch_tune(b: Batch, gates: Sequence[Tuple[Sequence[int], np.ndarray]], kmin: int = 1,
                  kmax: int = 4) -> dict:
    ga = GateArray(gates)
    r = sv_tune_result()
    _check(_lib.sv_batch_tune(b.handle, ga.arr, ga.n, kmin, kmax, ctypes.byref(r)))
    return {"best_k": r.best_k, "l2_bytes": r.l2_bytes, "best_ms": r.best_ms,
            "ms": {k: r.ms[k] for k in range(kmin, kmax + 1)}, "cached": r.cached,
            "tile_bits": r.tile_bits}


# --------------------------------------------------------------------------- serving

class Server:
    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.sv_server_destroy(self.handle)
            self.handle = None

    def destroy(self):
        if self.handle:
            _check(_lib.sv_server_destroy(self.handle))
            self.handle = None


def sv_server_create(budget_bytes: int = 0, max_slots: int = 0, topk: int = 0, max_k: int = 0,
                     fuse_threads: int = 0) -> Server:
    cfg = sv_server_config(budget_bytes, max_slots, topk, max_k, fuse_threads)
    h = _vp()
    _check(_lib.sv_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return Server(h.value)


def sv_server_submit(srv: Server, n: int, dtype: int, gates) -> int:
    """gates: a GateArray (prebuilt) or [(targets, U)]."""
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    rid = _u64()
    _check(_lib.sv_server_submit(srv.handle, n, dtype, ga.arr, ga.n, ctypes.byref(rid)))
    return rid.value


def _result_dict(r: sv_server_result) -> dict:
    k = r.k
    return {"id": r.id, "status": r.status, "dtype_used": r.dtype_used, "n": r.n, "k": k,
            "passes": r.passes, "idx": np.array(r.idx[:k], dtype=np.uint64),
            "p": np.array(r.p[:k], dtype=np.float64), "t_submit": r.t_submit,
            "t_admit": r.t_admit, "t_done": r.t_done}


def sv_server_poll(srv: Server, cap: int = 256, wait_ms: int = 0) -> list:
    buf = (sv_server_result * cap)()
    nout = ctypes.c_size_t()
    _check(_lib.sv_server_poll(srv.handle, buf, cap, ctypes.byref(nout), wait_ms))
    return [_result_dict(buf[i]) for i in range(nout.value)]


def sv_server_get_stats(srv: Server) -> dict:
    st = sv_server_stats()
    _check(_lib.sv_server_get_stats(srv.handle, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in sv_server_stats._fields_}


def sv_server_destroy(srv: Server) -> None:
    srv.destroy()
