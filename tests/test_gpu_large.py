"""The 30-, 32- and 33-qubit random grid circuits at their stated depth (24 cycles of
sqrtX/sqrtY/sqrtW + fSim(pi/2, pi/6), 1014-1188 gates), compared element by element.

* 30 qubits: the complex64 state (k = 5, tensor cores) and the complex128 state (a
  width-5 schedule, which complex128 runs fused again at width 4 on its tensor-core
  kernel) against the oracle's complex128 state of the unfused circuit (16 GiB on the
  host, a few minutes on the host cores).
* 32 qubits, complex128 (64 GiB) and 33 qubits, complex64 (64 GiB): the oracle does not
  fit, so the tensor-core path is compared with the CUDA-core path (FP64 / FP32 FMA, a
  different kernel and a different arithmetic) on the same fused schedule, both on the
  GPU.  The mirror invariant at these sizes is in test_gpu_parity.py.

Tolerances as everywhere: complex128 1e-12 max-abs amplitude error; complex64 1e-5
max-abs and 1 - fidelity <= 1e-6.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}
CHUNK = 1 << 24


def _torch():
    import torch
    return torch


def _compare_host(psi, ref):
    """(max-abs error, 1 - fidelity) of psi against ref, in chunks (no full-size
    temporaries)."""
    err, ip, na, nb = 0.0, 0j, 0.0, 0.0
    for i in range(0, ref.size, CHUNK):
        a = psi[i:i + CHUNK].astype(np.complex128)
        b = ref[i:i + CHUNK]
        err = max(err, float(np.max(np.abs(a - b))))
        ip += np.vdot(b, a)
        na += float(np.vdot(a, a).real)
        nb += float(np.vdot(b, b).real)
    return err, 1.0 - abs(ip) ** 2 / (na * nb)


def _compare_device(buf_a, buf_b, dtype):
    """The same on two device states (torch byte buffers), chunk by chunk on the GPU."""
    torch = _torch()
    cdt = torch.complex64 if dtype == 0 else torch.complex128
    a, b = buf_a.view(cdt), buf_b.view(cdt)
    err, ip, na, nb = 0.0, 0j, 0.0, 0.0
    step = 1 << 26
    for i in range(0, a.numel(), step):
        x = a[i:i + step].to(torch.complex128)
        y = b[i:i + step].to(torch.complex128)
        err = max(err, float((x - y).abs().max().item()))
        ip += complex(torch.vdot(y, x).item())
        na += float(torch.vdot(x, x).real.item())
        nb += float(torch.vdot(y, y).real.item())
        del x, y
    return err, 1.0 - abs(ip) ** 2 / (na * nb)


@pytest.fixture(scope="module")
def grid30_oracle():
    specs = W.grid_random(30, 24)
    assert len(specs) == 1014
    return specs, oracle.simulate(30, specs)


@pytest.mark.parametrize("dtype,k", [(0, 5), (1, 5)])
def test_grid_random_30q_against_oracle(gpu, grid30_oracle, dtype, k):
    sv = gpu
    torch = _torch()
    specs, ref = grid30_oracle
    c = sv.sv_fuse(sv.gates_from_specs(specs), 30, k)
    s = sv.sv_alloc(30, dtype, stream=torch.cuda.current_stream())
    rep = sv.sv_apply_circuit(s, c, adaptive=(dtype == 0))
    assert rep["promotions"] == 0 and rep["dtype_used"] == dtype
    assert rep["max_k_used"] == (5 if dtype == 0 else 4)
    psi = sv.sv_get_state(s)
    s.free()
    torch.cuda.empty_cache()
    err, infid = _compare_host(psi, ref)
    assert err <= TOL[dtype], f"max-abs error {err:.3e}"
    if dtype == 0:
        assert infid <= 1e-6, f"1 - F = {infid:.3e}"
    else:
        assert infid <= 1e-12, f"1 - F = {infid:.3e}"


@pytest.mark.parametrize("n,dtype,k", [(32, 1, 4), (33, 0, 5)])
def test_grid_random_full_size_tensor_vs_cuda_cores(gpu, n, dtype, k):
    sv = gpu
    torch = _torch()
    specs = W.grid_random(n, 24)
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, k)
    nbytes = (8 if dtype == 0 else 16) << n
    bufs = []
    for policy in (0, sv.SV_POLICY_NO_TENSOR_CORES):
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        s = sv.sv_alloc(n, dtype, dev_buf=buf, stream=torch.cuda.current_stream())
        sv.sv_set_policy(s, policy)
        rep = sv.sv_apply_circuit(s, c)
        assert rep["passes"] + rep["paired_passes"] == len(c)
        if policy == 0:
            assert rep["tc_passes"] >= 0.75 * rep["passes"]
        else:
            assert rep["tc_passes"] == 0
        sv.sv_sync(s)
        s.free()
        bufs.append(buf)
    err, infid = _compare_device(bufs[0], bufs[1], dtype)
    del bufs
    torch.cuda.empty_cache()
    assert err <= TOL[dtype], f"max-abs difference {err:.3e}"
    assert infid <= (1e-6 if dtype == 0 else 1e-12), f"1 - F = {infid:.3e}"
