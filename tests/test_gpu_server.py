"""Continuous-batching server: admission by HBM budget, overlap, and results that do
not depend on the other requests in flight."""
import time

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _requests(seed=0, count=12):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(8, 19))
        d = int(rng.integers(3, 12))
        dt = 0 if rng.uniform() < 0.7 else 1
        out.append((n, dt, W.brickwork(n, d, seed=int(rng.integers(0, 2**31)))))
    return out


def _drain(sv, srv, expected, timeout_s=120):
    got = {}
    t0 = time.time()
    while len(got) < expected:
        for r in sv.sv_server_poll(srv, 256, 50):
            got[r["id"]] = r
        assert time.time() - t0 < timeout_s, "server did not finish"
    return got


def test_results_alone_equal_results_in_the_mix(gpu):
    sv = gpu
    reqs = _requests()
    arrays = [sv.GateArray(sv.gates_from_specs(g)) for _, _, g in reqs]
    srv = sv.sv_server_create(max_slots=8, max_k=4)
    alone = []
    for (n, dt, _), ga in zip(reqs, arrays):
        rid = sv.sv_server_submit(srv, n, dt, ga)
        alone.append(_drain(sv, srv, 1)[rid])
    ids = [sv.sv_server_submit(srv, n, dt, ga) for (n, dt, _), ga in zip(reqs, arrays)]
    mix = _drain(sv, srv, len(ids))
    srv.destroy()
    for (n, dt, g), a, rid in zip(reqs, alone, ids):
        m = mix[rid]
        assert a["status"] == 0 and m["status"] == 0
        assert np.array_equal(a["idx"], m["idx"]) and np.array_equal(a["p"], m["p"])
        assert a["t_submit"] <= a["t_admit"] <= a["t_done"]
        # and the answer is right: a valid top-64 of the oracle's distribution
        p_ref = oracle.probs(oracle.simulate(n, g))
        tol = 1e-5 if dt == 0 else 1e-12
        assert oracle.topk_valid(m["idx"], p_ref, 64, tol)
        assert np.max(np.abs(m["p"] - p_ref[m["idx"].astype(np.int64)])) < tol


def test_admission_respects_the_budget_and_rejects_what_never_fits(gpu):
    sv = gpu
    state18 = (8 << 18) + 16 * 16 * 8 + 4 * 1024 * 1024 + 64 * 1024   # about one 18q c64 request
    budget = 2 * state18 + (1 << 20)
    srv = sv.sv_server_create(budget_bytes=budget, max_slots=8, max_k=2)
    ga = sv.GateArray(sv.gates_from_specs(W.brickwork(18, 20)))
    ids = [sv.sv_server_submit(srv, 18, 0, ga) for _ in range(6)]
    big = sv.sv_server_submit(srv, 24, 0, sv.GateArray(sv.gates_from_specs(W.brickwork(24, 2))))
    peak = 0
    got = {}
    t0 = time.time()
    while len(got) < len(ids) + 1:
        st = sv.sv_server_get_stats(srv)
        assert st["in_use_bytes"] <= budget
        peak = max(peak, st["active"])
        for r in sv.sv_server_poll(srv, 64, 5):
            got[r["id"]] = r
        assert time.time() - t0 < 120
    srv.destroy()
    assert peak <= 2
    assert got[big]["status"] == 2                        # SV_ERR_OOM: can never fit
    assert all(got[i]["status"] == 0 for i in ids)
    ref = got[ids[0]]
    assert all(np.array_equal(got[i]["idx"], ref["idx"]) for i in ids)


def test_admission_prefers_short_requests(gpu):
    """One slot, a long request in it: a large request and then ten small ones queue
    behind it; the small ones (least estimated work) are admitted before the large one,
    which still completes (aging)."""
    sv = gpu
    srv = sv.sv_server_create(max_slots=1, max_k=4)
    blocker = sv.GateArray(sv.gates_from_specs(W.brickwork(26, 30, seed=1)))
    big = sv.GateArray(sv.gates_from_specs(W.brickwork(24, 40, seed=2)))
    small = [sv.GateArray(sv.gates_from_specs(W.brickwork(12, 6, seed=10 + i))) for i in range(10)]
    b0 = sv.sv_server_submit(srv, 26, 1, blocker)
    time.sleep(0.05)
    b1 = sv.sv_server_submit(srv, 24, 1, big)
    ids = [sv.sv_server_submit(srv, 12, 0, ga) for ga in small]
    got = _drain(sv, srv, 12)
    srv.destroy()
    assert all(r["status"] == 0 for r in got.values())
    assert got[b0]["t_admit"] < got[b1]["t_admit"]
    assert max(got[i]["t_admit"] for i in ids) < got[b1]["t_admit"]


def test_large_complex128_requests_under_a_budget_of_a_few_states(gpu):
    """28-30-qubit complex128 requests (4-16 GiB each) against a 40 GiB budget: the bytes
    in use never exceed the budget, requests queue while it is full, and every result is
    the one the same request gives alone."""
    sv = gpu
    budget = 40 << 30
    reqs = [(30, 1, 1), (30, 1, 2), (29, 1, 3), (28, 1, 4), (30, 1, 5), (29, 0, 6)]
    arrays = [sv.GateArray(sv.gates_from_specs(W.brickwork(n, 5, seed=s))) for n, _, s in reqs]
    srv = sv.sv_server_create(budget_bytes=budget, max_slots=8, max_k=4)
    alone = []
    for (n, dt, _), ga in zip(reqs, arrays):
        rid = sv.sv_server_submit(srv, n, dt, ga)
        alone.append(_drain(sv, srv, 1, timeout_s=300)[rid])
    ids = [sv.sv_server_submit(srv, n, dt, ga) for (n, dt, _), ga in zip(reqs, arrays)]
    got, peak, t0 = {}, 0, time.time()
    while len(got) < len(ids):
        st = sv.sv_server_get_stats(srv)
        assert st["in_use_bytes"] <= budget
        peak = max(peak, st["in_use_bytes"])
        for r in sv.sv_server_poll(srv, 64, 5):
            got[r["id"]] = r
        assert time.time() - t0 < 300
    srv.destroy()
    assert peak > (16 << 30)                             # several large states at once
    for a, rid in zip(alone, ids):
        m = got[rid]
        assert a["status"] == 0 and m["status"] == 0
        assert np.array_equal(a["idx"], m["idx"]) and np.array_equal(a["p"], m["p"])
    # two 30-qubit complex128 states (16 GiB each) fit the budget, three do not: the
    # last of the three is admitted only after one of the others has finished
    big = sorted((got[rid] for rid, (n, dt, _) in zip(ids, reqs) if n == 30 and dt == 1),
                 key=lambda r: r["t_admit"])
    assert big[2]["t_admit"] >= min(big[0]["t_done"], big[1]["t_done"])
