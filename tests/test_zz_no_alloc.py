"""sv_expect_noalloc: the expectation entry point for callers that cannot allocate
device memory (code inside a global-mode CUDA stream capture, a framework that owns the
whole device-memory budget, a latency-critical loop that must not synchronise the device).

It takes a caller-owned device state and a caller-owned device output, keeps its block
partials in a fixed array inside the library, and must agree with sv_expect on the same
state, call after call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}     # the reduction tolerances used by the other GPU tests


def _terms(n, rng):
    xs = [int(v) for v in rng.integers(0, 1 << n, 20)] + [0] * 40 + [5] * 3
    zs = [int(v) for v in rng.integers(0, 1 << n, len(xs))]
    cs = [float(v) for v in rng.normal(size=len(xs))]
    return xs, zs, cs


@pytest.mark.parametrize("dtype", [0, 1])
def test_expect_noalloc_matches_sv_expect(gpu, dtype):
    sv = gpu
    import torch
    stream = torch.cuda.current_stream()
    n = 18
    rng = np.random.default_rng(300 + dtype)
    buf = torch.empty((8 if dtype == 0 else 16) << n, dtype=torch.uint8, device="cuda")
    s = sv.sv_alloc(n, dtype, dev_buf=buf, stream=stream)
    c = sv.sv_fuse(sv.gates_from_specs(W.brickwork(n, 8)), n, 3)
    sv.sv_set_basis(s, 77)
    sv.sv_apply_circuit(s, c)
    xs, zs, cs = _terms(n, rng)
    want = sv.sv_expect(s, xs, zs, cs)
    out = torch.empty(1, dtype=torch.float64, device="cuda")     # owned by the caller
    for _ in range(2):                                           # two calls in a row
        out.fill_(float("nan"))
        sv.sv_expect_noalloc(buf, n, dtype, xs, zs, cs, out, stream=stream)
        stream.synchronize()
        got = float(out.item())
        assert abs(got - want) <= TOL[dtype] * max(1.0, abs(want)), (got, want)
    # a different state through the same scratch array
    sv.sv_set_basis(s, 3)
    sv.sv_apply_circuit(s, c)
    want2 = sv.sv_expect(s, xs[:7], zs[:7], cs[:7])
    sv.sv_expect_noalloc(buf, n, dtype, xs[:7], zs[:7], cs[:7], out, stream=stream)
    stream.synchronize()
    assert abs(float(out.item()) - want2) <= TOL[dtype] * max(1.0, abs(want2))
    s.free()


def test_expect_noalloc_limits(gpu):
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
    sv.sv_expect_noalloc(buf, n, 0, [], [], [], out)                    # no terms -> 0
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
