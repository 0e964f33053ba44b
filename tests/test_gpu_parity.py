"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Tolerances (fixed by the target accuracy of the method): complex128 results within
1e-12 max-abs amplitude error; complex64 results within 1e-5 max-abs amplitude error
and 1 - fidelity <= 1e-6.  Integer results (top-k indices, fused schedules) bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import gates as OG
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}     # SV_C64, SV_C128


def _torch():
    import torch
    return torch


def run_gpu(sv, n, gl, dtype, max_k=0, x=0, adaptive=False):
    """Fuse (host), apply on cuda:0 through the C ABI, return the state as complex128."""
    c = sv.sv_fuse(gl, n, max_k)
    s = sv.sv_alloc(n, dtype, stream=_torch().cuda.current_stream())
    sv.sv_set_basis(s, x)
    rep = sv.sv_apply_circuit(s, c, adaptive=adaptive)
    psi = sv.sv_get_state(s).astype(np.complex128)
    s.free()
    return psi, rep


def check(psi, ref, dtype):
    err = float(np.max(np.abs(psi - ref)))
    assert err <= TOL[dtype], f"max-abs error {err:.3e}"
    if dtype == 0:
        f = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(psi, psi).real * np.vdot(ref, ref).real)
        assert 1 - f <= 1e-6, f"1 - F = {1 - f:.3e}"
    return err


def rand_state(n, rng):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_apply_random_gates_every_target_layout(gpu, dtype, k):
    sv = gpu
    rng = np.random.default_rng(10 * k + dtype)
    for n in sorted({k, 6, 11, 12, 13, 14, 16}):
        if n < k:
            continue
        layouts = [None, tuple(range(k)), tuple(range(n - k, n)),
                   tuple(reversed(range(n - k, n))), tuple(rng.choice(n, k, replace=False))]
        for tg in layouts:
            specs = W.random_unitary_gates(n, 4, k, rng, exact_k=True, targets=tg)
            psi0 = rand_state(n, rng)
            ref = oracle.run(psi0.copy(), OG.gate_list(specs))
            s = sv.sv_alloc(n, dtype, stream=_torch().cuda.current_stream())
            sv.sv_set_state(s, psi0.astype(np.complex64 if dtype == 0 else np.complex128))
            for tgt, u in sv.gates_from_specs(specs):
                sv.sv_apply_gate(s, tgt, u)
            psi = sv.sv_get_state(s).astype(np.complex128)
            s.free()
            check(psi, ref, dtype)


@pytest.mark.parametrize("dtype", [0, 1])
def test_closed_forms(gpu, dtype):
    sv = gpu
    bell, _ = run_gpu(sv, 2, sv.gates_from_specs(W.bell()), dtype, 2)
    want = np.zeros(4, complex)
    want[0] = want[3] = 1 / math.sqrt(2)
    check(bell, want, dtype)
    n = 20
    for k in (0, 2, 5):
        g, _ = run_gpu(sv, n, sv.gates_from_specs(W.ghz(n)), dtype, k)
        want = np.zeros(1 << n, complex)
        want[0] = want[-1] = 1 / math.sqrt(2)
        check(g, want, dtype)
    n = 16
    x = 40503
    y = np.arange(1 << n)
    want = np.exp(2j * np.pi * x * y / (1 << n)) / math.sqrt(1 << n)
    for k in (0, 2, 3, 4, 5):
        q, _ = run_gpu(sv, n, sv.gates_from_specs(W.qft(n)), dtype, k, x=x)
        check(q, want, dtype)


def test_brickwork_12q_c128_unfused(gpu):
    """12 qubits, 20 layers of U3 + CZ brickwork, complex128, per-gate application:
    full state, probabilities and <Z0 Z1>."""
    sv = gpu
    n = 12
    specs = W.brickwork(n, 20)
    assert len(specs) == 350
    ref = oracle.simulate(n, specs)
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, 0)
    assert len(c) == 350
    s = sv.sv_alloc(n, 1, stream=_torch().cuda.current_stream())
    sv.sv_apply_circuit(s, c)
    psi = sv.sv_get_state(s)
    check(psi, ref, 1)
    p = sv.sv_probs(s)
    assert p.dtype == np.float64
    assert np.max(np.abs(p - oracle.probs(ref))) < 1e-12
    assert abs(sv.sv_expect(s, [0], [0b11], [1.0]) - oracle.expect_pauli(ref, 0, 0b11).real) < 1e-12
    assert abs(sv.sv_norm(s) - oracle.norm(ref)) < 1e-12


@pytest.fixture(scope="module")
def qft_brickwork_24q():
    x, specs = W.qft_brickwork(24, 40)
    return x, specs, oracle.simulate(24, specs, x=x)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_qft_brickwork_24q_fused(gpu, qft_brickwork_24q, dtype, k):
    """24 qubits: QFT on a seeded basis state + 40 U3/CNOT-ladder layers, fused at
    k = 2..5, complex64 and complex128 against the oracle."""
    sv = gpu
    x, specs, ref = qft_brickwork_24q
    psi, rep = run_gpu(sv, 24, sv.gates_from_specs(specs), dtype, k, x=x)
    check(psi, ref, dtype)
    assert rep["passes"] < len(specs)
    # complex128 runs a width-5 schedule fused again at width 4 (tensor-core passes)
    assert rep["max_k_used"] == (min(k, 4) if dtype == 1 else k)


@pytest.mark.parametrize("dtype,k", [(0, 5), (1, 4)])
def test_qft_brickwork_24q_mirror(gpu, dtype, k):
    sv = gpu
    x, specs = W.qft_brickwork(24, 40)
    psi, _ = run_gpu(sv, 24, sv.gates_from_specs(W.mirror(specs)), dtype, k, x=x)
    assert abs(abs(psi[x]) ** 2 - 1) <= (1e-5 if dtype == 0 else 1e-12)


@pytest.mark.parametrize("n,dtype,k,cycles", [(30, 0, 4, 24), (30, 0, 5, 24), (33, 0, 5, 24),
                                              (30, 1, 4, 24), (30, 1, 5, 24), (32, 1, 4, 24)])
def test_grid_random_mirror_large(gpu, n, dtype, k, cycles):
    """30/32/33 qubits at the stated depth and widths: the mirror circuit C C^dagger |0> =
    |0> (Eq. 10 applied to C followed by its inverse).  The forward states themselves are
    compared element by element in test_gpu_large.py."""
    sv = gpu
    torch = _torch()
    specs = W.grid_random(n, cycles)
    c = sv.sv_fuse(sv.gates_from_specs(W.mirror(specs)), n, k)
    s = sv.sv_alloc(n, dtype, stream=torch.cuda.current_stream())
    sv.sv_apply_circuit(s, c)
    idx, p = sv.sv_topk(s, 2)
    tol = 1e-5 if dtype == 0 else 1e-12
    assert idx[0] == 0 and abs(p[0] - 1) <= tol
    assert abs(sv.sv_norm(s) - 1) <= tol
    s.free()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [0, 1])
def test_reductions_random_state(gpu, dtype):
    sv = gpu
    rng = np.random.default_rng(77 + dtype)
    for n in (1, 3, 6, 13, 17):
        psi0 = rand_state(n, rng)
        s = sv.sv_alloc(n, dtype, stream=_torch().cuda.current_stream())
        psi_in = psi0.astype(np.complex64 if dtype == 0 else np.complex128)
        sv.sv_set_state(s, psi_in)
        psi = psi_in.astype(np.complex128)                   # the input as stored
        tol = 1e-6 if dtype == 0 else 1e-13
        assert abs(sv.sv_norm(s) - oracle.norm(psi)) < tol
        p = sv.sv_probs(s)
        p_same = oracle.probs_in_precision(psi_in)
        assert np.array_equal(p, p_same)                     # same IEEE operations
        assert np.max(np.abs(p - oracle.probs(psi))) < tol
        xs = [int(v) for v in rng.integers(0, 1 << n, 12)] + [0, 0]
        zs = [int(v) for v in rng.integers(0, 1 << n, 14)]
        cs = [float(v) for v in rng.normal(size=14)]
        got = sv.sv_expect(s, xs, zs, cs)
        assert abs(got - oracle.expect(psi, xs, zs, cs)) < 10 * tol
        for x, z in zip(xs[:4], zs[:4]):
            assert abs(sv.sv_expect(s, [x], [z], [1.0]) - oracle.expect_pauli(psi, x, z).real) < tol
        idx, pv = sv.sv_topk(s, 64)
        want_i, want_p = oracle.topk(p_same.astype(np.float64), 64)
        assert np.array_equal(idx, want_i)                   # same precision decision
        assert np.array_equal(pv, want_p)
        s.free()


def test_topk_ties_and_uniform(gpu):
    sv = gpu
    n = 14
    c = sv.sv_fuse(sv.gates_from_specs([W.GateSpec("h", (q,)) for q in range(n)]), n, 3)
    for dtype in (0, 1):
        s = sv.sv_alloc(n, dtype)
        sv.sv_apply_circuit(s, c)
        idx, p = sv.sv_topk(s, 64)
        # all 2^14 probabilities are equal up to rounding: any 64 outcomes are a valid
        # answer, listed by (p desc, index asc)
        exact = np.full(1 << n, 2.0 ** -n)
        assert oracle.topk_valid(idx, exact, 64, 1e-6 * 2.0 ** -n)
        assert all(p[j] > p[j + 1] or (p[j] == p[j + 1] and idx[j] < idx[j + 1]) for j in range(63))
        s.free()
    # exact ties: |0> + |1> + ... planted with equal amplitudes, set from the host
    for dtype in (0, 1):
        m = 10
        amp = np.zeros(1 << m, dtype=np.complex64 if dtype == 0 else np.complex128)
        amp[[5, 900, 17, 3, 600]] = 0.5 ** 0.5 / 2 ** 0.5   # 0.5 each -> equal probabilities
        s = sv.sv_alloc(m, dtype)
        sv.sv_set_state(s, amp)
        idx, _ = sv.sv_topk(s, 64)
        want, _ = oracle.topk(oracle.probs_in_precision(amp).astype(np.float64), 64)
        assert np.array_equal(idx, want) and list(idx[:5]) == [3, 5, 17, 600, 900]
        s.free()


def test_zz_chain_on_ghz(gpu):
    sv = gpu
    n = 18
    psi, _ = run_gpu(sv, n, sv.gates_from_specs(W.ghz(n)), 1, 3)
    s = sv.sv_alloc(n, 1)
    sv.sv_set_state(s, psi)
    xs, zs, cs = W.zz_chain(n)
    assert abs(sv.sv_expect(s, xs, zs, cs) - (n - 1)) < 1e-12
    assert abs(sv.sv_expect(s, [(1 << n) - 1], [0], [1.0]) - 1) < 1e-12
    s.free()


def test_adaptive_promotion_replays_in_c128(gpu):
    """A slightly non-unitary gate makes the complex64 norm drift past 1e-6; the
    controller replays the circuit in complex128 and reports the promotion."""
    sv = gpu
    n = 14
    specs = W.brickwork(n, 6)
    gl = sv.gates_from_specs(specs)
    leak = np.diag([1.0 + 1e-4, 1.0]).astype(np.complex128)
    gl = gl[:40] + [((3,), leak)] + gl[40:]
    ogl = OG.gate_list(specs)
    ref = oracle.run(oracle.basis(n, 9), ogl[:40] + [((3,), leak)] + ogl[40:])
    psi, rep = run_gpu(sv, n, gl, 0, 3, x=9, adaptive=True)
    assert rep["promotions"] == 1 and rep["dtype_used"] == 1
    check(psi, ref, 1)
    # back to complex64 on the same state object
    c = sv.sv_fuse(sv.gates_from_specs(specs), n, 3)
    s = sv.sv_alloc(n, 0)
    sv.sv_apply_circuit(s, sv.sv_fuse(gl, n, 3), adaptive=True)
    assert sv.sv_info(s)[1] == 1
    sv.sv_set_dtype(s, 0)
    assert sv.sv_info(s)[1] == 0 and sv.sv_topk(s, 1)[0][0] == 0
    sv.sv_set_basis(s, 9)
    sv.sv_apply_circuit(s, c)
    check(sv.sv_get_state(s).astype(np.complex128), oracle.simulate(n, specs, x=9), 0)
    s.free()
    # unitary circuit: no promotion, stays complex64; a basis start has norm exactly 1
    psi2, rep2 = run_gpu(sv, n, sv.gates_from_specs(specs), 0, 3, x=9, adaptive=True)
    assert rep2["promotions"] == 0 and rep2["dtype_used"] == 0 and rep2["drift"] < 1e-6
    assert rep2["norm_before"] == 1.0
    check(psi2, oracle.simulate(n, specs, x=9), 0)


def test_adaptive_promotion_from_arbitrary_state_and_caller_buffer(gpu):
    sv = gpu
    torch = _torch()
    n = 12
    rng = np.random.default_rng(5)
    psi0 = rand_state(n, rng).astype(np.complex64)
    leak = ((0,), np.diag([1.001, 1.0]).astype(np.complex128))
    gl = sv.gates_from_specs(W.brickwork(n, 4)) + [leak]
    ref = oracle.run(psi0.astype(np.complex128), OG.gate_list(W.brickwork(n, 4)) + [leak])
    buf = torch.empty(16 << n, dtype=torch.uint8, device="cuda")   # room for complex128
    s = sv.sv_alloc(n, 0, dev_buf=buf, stream=torch.cuda.current_stream())
    sv.sv_set_state(s, psi0)
    c = sv.sv_fuse(gl, n, 2)
    rep = sv.sv_apply_circuit(s, c, adaptive=True, drift_check_every=3)
    assert rep["promotions"] == 1 and sv.sv_info(s)[1] == 1
    check(sv.sv_get_state(s), ref, 1)
    s.free()
    small = torch.empty(8 << n, dtype=torch.uint8, device="cuda")     # complex64 only
    s = sv.sv_alloc(n, 0, dev_buf=small, stream=torch.cuda.current_stream())
    with pytest.raises(sv.SvError) as e:
        sv.sv_apply_circuit(s, c, adaptive=True)
    assert e.value.status == 5
    s.free()


def test_edge_cases(gpu):
    sv = gpu
    torch = _torch()
    # n = 1, and n = k = 5 (the whole state is one group)
    for n, k in ((1, 1), (5, 5), (3, 3)):
        rng = np.random.default_rng(n)
        specs = W.random_unitary_gates(n, 3, k, rng, exact_k=True)
        ref = oracle.simulate(n, specs, x=1)
        for dtype in (0, 1):
            psi, _ = run_gpu(sv, n, sv.gates_from_specs(specs), dtype, 0, x=1)
            check(psi, ref, dtype)
    # empty circuit leaves the state alone
    c = sv.sv_fuse([], 8, 3)
    assert len(c) == 0
    s = sv.sv_alloc(8, 0)
    sv.sv_set_basis(s, 200)
    sv.sv_apply_circuit(s, c)
    assert sv.sv_topk(s, 1)[0][0] == 200
    # argument errors on a live state
    with pytest.raises(sv.SvError):
        sv.sv_set_basis(s, 256)
    with pytest.raises(sv.SvError):
        sv.sv_apply_gate(s, (8,), np.eye(2))
    with pytest.raises(sv.SvError):
        sv.sv_topk(s, 65)
    with pytest.raises(sv.SvError):
        sv.sv_expect(s, [1 << 9], [0], [1.0])
    with pytest.raises(sv.SvError):
        sv.sv_apply_circuit(s, sv.sv_fuse([], 9, 3))
    s.free()
    with pytest.raises(sv.SvError):
        sv.sv_alloc(10, 0, dev_buf=torch.empty(100, dtype=torch.uint8, device="cuda"))


def test_largest_state_one_gate(gpu):
    """34 qubits in complex64 (128 GiB): one 2-qubit gate on the two top bits."""
    sv = gpu
    torch = _torch()
    n = 34
    s = sv.sv_alloc(n, 0, stream=torch.cuda.current_stream())
    sv.sv_set_basis(s, (1 << n) - 1)
    h = np.kron(OG.H, OG.H)
    sv.sv_apply_gate(s, (32, 33), h)
    idx, p = sv.sv_topk(s, 4)
    assert sorted(int(i) for i in idx) == [(1 << 32) - 1 + (j << 32) for j in range(4)]
    assert np.allclose(p, 0.25, atol=1e-6)
    s.free()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [0, 1])
def test_probs_to_host_30q(gpu, dtype):
    """Probabilities of a 2^30-amplitude state copied to host memory (4 or 8 GiB)."""
    sv = gpu
    torch = _torch()
    n = 30
    x = (1 << 29) + 12345
    s = sv.sv_alloc(n, dtype, stream=torch.cuda.current_stream())
    sv.sv_set_basis(s, x)
    sv.sv_apply_gate(s, (0,), OG.H)
    p = sv.sv_probs(s)
    assert p.size == 1 << n
    nz = np.flatnonzero(p)
    assert list(nz) == [x - 1, x] and np.allclose(p[nz], 0.5, atol=1e-7)
    del p
    s.free()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [0, 1])
def test_expectation_term_groups(gpu, dtype):
    """Groups of 1..5 terms sharing an X-part (the complex64 fast kernels take 1..4 terms
    per launch, diagonal or not; 5 and more use the general kernel), against the oracle,
    on a state whose amplitudes span several binades, at sizes with a ragged grid tail."""
    sv = gpu
    rng = np.random.default_rng(911 + dtype)
    for n in (5, 11, 18):
        psi0 = rand_state(n, rng) * np.exp2(rng.integers(-6, 1, 1 << n))
        psi0 /= np.linalg.norm(psi0)
        s = sv.sv_alloc(n, dtype, stream=_torch().cuda.current_stream())
        psi_in = psi0.astype(np.complex64 if dtype == 0 else np.complex128)
        sv.sv_set_state(s, psi_in)
        psi = psi_in.astype(np.complex128)
        tol = 2e-6 if dtype == 0 else 1e-13
        for nt in (1, 2, 3, 4, 5, 7):
            for x in (0, int(rng.integers(1, 1 << n))):
                zs = [int(v) for v in rng.integers(0, 1 << n, nt)]
                cs = [float(v) for v in rng.normal(size=nt)]
                got = sv.sv_expect(s, [x] * nt, zs, cs)
                want = oracle.expect(psi, [x] * nt, zs, cs)
                assert abs(got - want) < tol * (1 + sum(abs(c) for c in cs)), (n, nt, x, got, want)
        s.free()


@pytest.mark.parametrize("dtype", [0, 1])
def test_probs_into_pinned_host_memory(gpu, dtype):
    """Page-locked host output (written by the kernel over the CPU-GPU link) equals the
    pageable-memory path bit for bit and the oracle's probabilities in the same precision."""
    sv = gpu
    torch = _torch()
    rng = np.random.default_rng(951 + dtype)
    for n in (9, 22):
        psi0 = rand_state(n, rng).astype(np.complex64 if dtype == 0 else np.complex128)
        s = sv.sv_alloc(n, dtype, stream=torch.cuda.current_stream())
        sv.sv_set_state(s, psi0)
        pageable = sv.sv_probs(s)
        pinned = torch.empty(1 << n, dtype=torch.float32 if dtype == 0 else torch.float64).pin_memory()
        pinned.fill_(-1.0)
        sv.sv_probs(s, pinned.numpy())
        assert np.array_equal(pinned.numpy(), pageable)
        assert np.array_equal(pageable, oracle.probs_in_precision(psi0))
        # staged through a device buffer and a copy-engine transfer: the same bits
        sv.sv_set_policy(s, sv.SV_POLICY_STAGED_PROBS)
        for _ in range(2):
            pinned.fill_(-1.0)
            sv.sv_probs(s, pinned.numpy())
            assert np.array_equal(pinned.numpy(), pageable)
        s.free()


def test_c128_width5_circuit_runs_on_the_tensor_cores(gpu):
    """A circuit fused at width 5, applied to a complex128 state: the state runs the input
    gates fused at width 4, every pass on the complex128 tensor-core kernel, and matches
    the oracle at 1e-12; an adaptive complex64 run that drifts replays the same way."""
    sv = gpu
    n = 20
    specs = W.grid_random(n, 8)
    gl = sv.gates_from_specs(specs)
    ref = oracle.simulate(n, specs, x=5)
    c5 = sv.sv_fuse(gl, n, 5)
    c4 = sv.sv_fuse(gl, n, 4)
    s = sv.sv_alloc(n, 1, stream=_torch().cuda.current_stream())
    sv.sv_set_basis(s, 5)
    rep = sv.sv_apply_circuit(s, c5)
    assert rep["max_k_used"] == 4 and rep["passes"] == len(c4)
    assert rep["tc_passes"] == rep["passes"]
    check(sv.sv_get_state(s), ref, 1)
    s.free()
    # promotion: a leaky gate makes the complex64 norm drift; the replay is complex128 at k = 4
    leak = ((2,), np.diag([1.0 + 1e-4, 1.0]).astype(np.complex128))
    ogl = OG.gate_list(specs)
    half = len(gl) // 2
    ref2 = oracle.run(oracle.basis(n, 5), ogl[:half] + [leak] + ogl[half:])
    cl = sv.sv_fuse(gl[:half] + [leak] + gl[half:], n, 5)
    psi, rep2 = run_gpu(sv, n, gl[:half] + [leak] + gl[half:], 0, 5, x=5, adaptive=True)
    assert rep2["promotions"] == 1 and rep2["dtype_used"] == 1 and rep2["max_k_used"] == 4
    check(psi, ref2, 1)
    assert len(cl) < rep2["passes"]


def test_promotion_allocation_failure_leaves_a_checked_state(gpu):
    """Out of memory during a promotion (forced through the library's allocation test
    hook): the call fails with SV_ERR_OOM, later calls on the state return SV_ERR_STATE
    instead of launching on a missing buffer, sv_set_dtype recovers it; with only the first
    allocation failing, the promotion releases the complex64 buffer first and succeeds."""
    sv = gpu
    n = 16
    specs = W.brickwork(n, 4)
    leak = ((0,), np.diag([1.0 + 1e-3, 1.0]).astype(np.complex128))
    gl = sv.gates_from_specs(specs) + [leak]
    ref = oracle.run(oracle.basis(n, 0), OG.gate_list(specs) + [leak])
    c = sv.sv_fuse(gl, n, 4)
    s = sv.sv_alloc(n, 0, stream=_torch().cuda.current_stream())
    try:
        sv.sv_debug_fail_allocs(2)
        with pytest.raises(sv.SvError) as e:
            sv.sv_apply_circuit(s, c, adaptive=True)
        assert e.value.status == 2
        sv.sv_debug_fail_allocs(0)
        for call in (lambda: sv.sv_norm(s), lambda: sv.sv_topk(s, 4), lambda: sv.sv_probs(s),
                     lambda: sv.sv_apply_circuit(s, c), lambda: sv.sv_set_basis(s, 1),
                     lambda: sv.sv_get_state(s), lambda: sv.sv_sample(s, 1, 4)):
            with pytest.raises(sv.SvError) as e:
                call()
            assert e.value.status == 5
        sv.sv_set_dtype(s, 0)
        assert abs(sv.sv_norm(s) - 1.0) < 1e-7 and sv.sv_info(s)[1] == 0
        sv.sv_debug_fail_allocs(1)
        rep = sv.sv_apply_circuit(s, c, adaptive=True)
        assert rep["promotions"] == 1 and sv.sv_info(s)[1] == 1
        check(sv.sv_get_state(s), ref, 1)
    finally:
        sv.sv_debug_fail_allocs(0)
    s.free()
