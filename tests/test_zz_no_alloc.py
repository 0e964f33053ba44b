"""sv_expect_noalloc: the expectation entry point for callers that cannot allocate device
memory (a framework that owns the whole device-memory budget through its own pool, a
latency-critical loop where an allocation would synchronise the device).

It takes a caller-owned device state and a caller-owned device output and keeps its
block partials in a fixed array inside the library.  Checked against the oracle (the
state read back and the Pauli sum taken on the CPU) and against sv_expect, on two calls
in a row and on a second state through the same scratch array.  This file is collected
last on purpose.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}     # the reduction tolerances used by the other GPU tests


def _terms(n, rng):
    xs = [int(v) for v in rng.integers(0, 1 << n, 20)] + [0] * 40 + [5] * 3
    zs = [int(v) for v in rng.integers(0, 1 << n, len(xs))]
    cs = [float(v) for v in rng.normal(size=len(xs))]
    return xs, zs, cs


def _close(got, want, dtype):
    return abs(got - want) <= TOL[dtype] * max(1.0, abs(want))


@pytest.mark.parametrize("dtype", [0, 1])
def test_expect_noalloc_matches_oracle_and_sv_expect(gpu, dtype):
    sv = gpu
    import torch
    stream = torch.cuda.current_stream()
    n = 14
    rng = np.random.default_rng(300 + dtype)
    buf = torch.empty((8 if dtype == 0 else 16) << n, dtype=torch.uint8, device="cuda")
    s = sv.sv_alloc(n, dtype, dev_buf=buf, stream=stream)
    c = sv.sv_fuse(sv.gates_from_specs(W.brickwork(n, 8)), n, 3)
    sv.sv_set_basis(s, 77)
    sv.sv_apply_circuit(s, c)
    psi = sv.sv_get_state(s).astype(np.complex128)        # the state as stored
    xs, zs, cs = _terms(n, rng)
    want = oracle.expect(psi, xs, zs, cs)
    existing = sv.sv_expect(s, xs, zs, cs)                       # the allocating entry point
    assert _close(existing, want, dtype)
    out = torch.empty(1, dtype=torch.float64, device="cuda")     # owned by the caller
    for _ in range(2):                                           # two calls in a row
        out.fill_(float("nan"))
        sv.sv_expect_noalloc(buf, n, dtype, xs, zs, cs, out, stream=stream)
        stream.synchronize()
        got = float(out.item())
        assert _close(got, existing, dtype), (got, existing)
        assert _close(got, want, dtype), (got, want)
    # a different state and fewer terms through the same scratch array
    sv.sv_set_basis(s, 3)
    sv.sv_apply_circuit(s, c)
    psi2 = sv.sv_get_state(s).astype(np.complex128)
    want2 = oracle.expect(psi2, xs[:7], zs[:7], cs[:7])
    sv.sv_expect_noalloc(buf, n, dtype, xs[:7], zs[:7], cs[:7], out, stream=stream)
    stream.synchronize()
    assert _close(float(out.item()), want2, dtype)
    assert _close(float(out.item()), sv.sv_expect(s, xs[:7], zs[:7], cs[:7]), dtype)
    s.free()


def test_expect_noalloc_limits_and_pointers(gpu):
    sv = gpu
    import torch
    n = 8
    buf = torch.zeros(8 << n, dtype=torch.uint8, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    # 65 distinct X-parts need 65 term batches: beyond the fixed scratch array
    xs = list(range(1, 66))
    with pytest.raises(sv.SvError) as e:
        sv.sv_expect_noalloc(buf, n, 0, xs, [0] * 65, [1.0] * 65, out)
    assert e.value.status == 1 and "scratch" in str(e.value)
    with pytest.raises(sv.SvError):
        sv.sv_expect_noalloc(buf, n, 0, [1 << n], [0], [1.0], out)      # qubit >= n
    # host memory for the state or the output is refused before any launch
    host_state = np.zeros(1 << n, dtype=np.complex64)
    host_out = np.zeros(1, dtype=np.float64)
    with pytest.raises(sv.SvError) as e:
        sv.sv_expect_noalloc(host_state.ctypes.data, n, 0, [0], [1], [1.0], out)
    assert e.value.status == 1 and "device memory" in str(e.value)
    with pytest.raises(sv.SvError) as e:
        sv.sv_expect_noalloc(buf, n, 0, [0], [1], [1.0], host_out.ctypes.data)
    assert e.value.status == 1
    with pytest.raises(sv.SvError):                                    # misaligned output
        sv.sv_expect_noalloc(buf, n, 0, [0], [1], [1.0], int(buf.data_ptr()) + 4)
    sv.sv_expect_noalloc(buf, n, 0, [], [], [], out)                    # no terms -> 0
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
