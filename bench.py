#!/usr/bin/env python
"""Benchmark: fused-gate state-vector simulation of a 30-qubit random grid circuit.

Workload (default): 30 qubits on a 5 x 6 grid, 24 cycles of {sqrtX, sqrtY, sqrtW} on
every qubit + fSim(pi/2, pi/6) on one of four edge classes (720 + 294 = 1014 gates),
seeded; complex64 state (8 GiB, larger than L2), DAG fusion at k = 5, adaptive
c64 -> c128 promotion on norm drift > 1e-6.  One step is the whole hot path:
  sv_fuse (host DAG fusion) -> sv_set_basis -> sv_apply_circuit (every fused pass, then
  the FP64 norm; a basis start's norm is exactly 1) -> sv_topk(64) -> sv_expect(<Z0 Z1>).
The default run then adds the unfused complex128 comparison and the other configurations
of the metric (28/33-qubit complex64, 30/32-qubit complex128, batched, sharded and served
summaries) as extra keys of the same line.
Metric: circuits/s (whole job), with the fused-gate HBM GB/s of the apply kernels.

--impl reference times the CPU oracle (complex128, unfused, OpenMP over the host cores)
on bounded samples of the same workload, scaled to circuits/s.
Under torchrun each rank runs an independent replica (no collective on the data path).
"""
import argparse
import concurrent.futures
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = ("fused-gate HBM GB/s & circuits/s at 28–33q vs unfused c128; "
          "served p50/p99 latency")
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic of one tensor-core pass from the ncu captures summarised under profiles/
# (27-qubit launches scaled by 2^3 to the 30-qubit bench), the kernel that dominates each
# precision's launch list, and the sources the numbers are valid for (traffic is reported
# as null once those sources hash differently).
KERNELS = {
    "c64": {"files": ("apply_tc.cu", "tc.cuh", "ptx.cuh", "plan.h"),
            "sha256_prefix": "de4565ba003a3a0c", "n": 30,
            "bytes_per_launch": (1.073838e9 + 1.012321e9) * 8,
            "kernel": "fused-gate passes: apply_tc<5,0,2,0,1> 97.5% of GPU time "
                      "(profiles/fused_pass_grid30q_k5_launches.md)",
            "traffic_source": "apply_tc<5,0,2,0,1> ncu capture at 27q scaled to 30q "
                              "(profiles/apply_tc5_c64_27q_ncu.md)"},
    "c128": {"files": ("apply_tc64.cu", "fixed_point.h", "tc.cuh", "ptx.cuh", "plan.h"),
             "sha256_prefix": "fe2ac4ee6436bc13", "n": 30,
             "bytes_per_launch": (2.147647e9 + 2.085257e9) * 8,
             "kernel": "fused-gate passes: apply_tc64<*> 98.1% of GPU time "
                       "(profiles/fused_pass_grid30q_c128_k4_launches.md); bound by the "
                       "integer ALU pipe, not HBM (profiles/apply_tc64_c128_27q_ncu.md)",
             "traffic_source": "apply_tc64<0,2,0> ncu capture at 27q scaled to 30q "
                               "(profiles/apply_tc64_c128_27q_ncu.md)"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--cycles", type=int, default=24)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--e2e-states", type=int, default=4,
                    help="states in flight in the end-to-end loop (one host thread and stream each)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare-unfused", action="store_true",
                    help="skip timing the unfused complex128 per-gate form of the circuit")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra lines of the default run (28-33 qubit configurations, "
                         "complex128, batched and served summaries)")
    ap.add_argument("--two-gate-passes", action="store_true",
                    help="apply pairs of dense gates that fit one tile in one pass "
                         "(SV_POLICY_TWO_GATE_PASSES; off by default)")
    ap.add_argument("--cpu-sample-s", type=float, default=12.0)
    ap.add_argument("--mode", default="single",
                    choices=["single", "batched", "serve", "sample", "noise", "qft", "shard", "pairs"],
                    help="single: the 30-qubit hot path (default line); batched: 512 HEA "
                         "circuits of 16-22 qubits; serve: Poisson request stream; sample: "
                         "measurement shots from the 30-qubit circuit's output state; "
                         "qft: QFT of a basis state with structure-aware passes against "
                         "the same schedule forced dense; shard: one state over the "
                         "ranks (global-qubit sharding, NCCL exchanges), --n qubits per GPU; "
                         "pairs: two-gate passes per tile layout against one-gate passes")
    ap.add_argument("--emulate-ranks", type=int, default=0,
                    help="shard: run this many ranks as threads on one GPU (exchanges are "
                         "device copies) instead of one process per GPU")
    ap.add_argument("--shots", type=int, default=1 << 20, help="sample: shots per step")
    ap.add_argument("--circuit", default="qft", choices=["qft", "phase_heavy", "qaoa"],
                    help="qft mode: the circuit family (QFT; random diagonal-heavy; QAOA layers)")
    ap.add_argument("--p-depol", type=float, default=0.01, help="noise: depolarizing p")
    ap.add_argument("--noise-n", type=int, default=15, help="noise: qubits of the density matrix")
    ap.add_argument("--count", type=int, default=512, help="batched: number of circuits")
    ap.add_argument("--batch-k", type=int, default=0,
                    help="batched: fixed fusion width with whole-batch chunks (0: autotune)")
    ap.add_argument("--rates", default="10,30,100,300,1000,2000", help="serve: req/s list")
    ap.add_argument("--duration", type=float, default=4.0, help="serve: seconds per rate")
    ap.add_argument("--requests", type=int, default=500,
                    help="serve: requests per rate (arrivals over requests / rate seconds)")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, world, device):
    """The job's time is its slowest rank's: all-reduce MAX of the per-rank milliseconds."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, ms):
    """Whole-job units per second: every rank ran `steps` units in at most `ms`."""
    return world * steps / (ms / 1000.0)


def kernel_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2604_03816_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def hbm_peak():
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
        finally:
            os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(specs, n, budget_s, gates_total):
    """The oracle (complex128, unfused, OpenMP) on a bounded sample: as many of the
    workload's gates as fit in about budget_s seconds at full width."""
    import oracle
    from oracle import gates as OG
    gl = OG.gate_list(specs)
    psi = oracle.basis(n, 0)
    t0 = time.perf_counter()
    done = 0
    while done < len(gl) and (done < 2 or time.perf_counter() - t0 < budget_s):
        oracle.apply_gate(psi, *gl[done])
        done += 1
    dt = time.perf_counter() - t0
    del psi
    per_gate = dt / done
    return {"value": 1.0 / (per_gate * gates_total), "unit": "circuits/s",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {done} of {gates_total} gates of the {n}-qubit workload, "
                      f"complex128 unfused, {dt:.1f} s, scaled to one circuit"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    from oracle import gates as OG
    specs = W.grid_random(args.n, args.cycles)
    gl = OG.gate_list(specs)
    nfused = len(oracle.fuse(gl, args.n, args.k))     # the same schedule length (Algorithm 2)
    psi = oracle.basis(args.n, 0)
    per_step = max(1, int(os.environ.get("REF_GATES_PER_STEP", "3")))
    times = []
    pos = 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            oracle.apply_gate(psi, *gl[pos % len(gl)])
            pos += 1
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = args.steps * per_step / total / len(gl)
    cores = oracle.num_threads()
    out = {"metric": METRIC, "value": value, "unit": "circuits/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": config_dict(args, len(specs), nfused),
           "cpu_baseline": {"value": value, "unit": "circuits/s", "cores": cores,
                            "kind": "oracle",
                            "sample": f"{per_step} gates per step of the {args.n}-qubit "
                                      f"workload (complex128, unfused), scaled to circuits"},
           "e2e": {"value": value, "unit": "circuits/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_sample(args):
    """Measurement sampling (sv_sample) from the output state of the 30-qubit grid circuit:
    one step = one sv_sample call of --shots shots to host memory (integer block sums over
    the whole state, prefix scans, the shots)."""
    import torch
    from paper_2604_03816_gb300 import sv
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    dt = sv.SV_C64 if args.dtype == "c64" else sv.SV_C128
    specs = W.grid_random(args.n, args.cycles)
    state = sv.sv_alloc(args.n, dt, stream=stream)
    with torch.cuda.stream(stream):
        sv.sv_apply_circuit(state, sv.sv_fuse(sv.gates_from_specs(specs), args.n, args.k))
        for w in range(args.warmup):
            sv.sv_sample(state, w, args.shots)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(None) as clk:
            e0.record(stream)
            for i in range(args.steps):
                shots = sv.sv_sample(state, 1000 + i, args.shots)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
    state.free()
    sbytes = (8 if dt == sv.SV_C64 else 16) << args.n
    peak, peak_kind = hbm_peak()
    out = {"metric": "measurement shots/s (sv_sample, 30q grid circuit output state)",
           "value": args.shots / (ms / 1000.0), "unit": "shots/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u64 sums", "data": "synthetic",
           "config": {"workload": f"grid_random {args.n}q depth {args.cycles}, {args.dtype}, "
                                  f"{args.shots} shots per call to host memory",
                      "state_bytes": sbytes, "seed": W.seed_for(3, args.n),
                      "l2": "state larger than L2 (inputs > 129 MB), no flush needed"},
           "roofline": {"bound": "hbm", "achieved": sbytes / (ms / 1000.0) / 1e9, "peak": peak,
                        "unit": "GB/s", "frac": sbytes / (ms / 1000.0) / 1e9 / peak,
                        "traffic": None, "peak_kind": peak_kind,
                        "kernel": "whole call (one read of the state for the integer block "
                                  "sums, then prefix scans and shots)"},
           "cpu_baseline": None, "e2e": None, "gpu_launches": 4 * args.steps,
           "clocks": clk.summary(), "last_shots_head": [int(v) for v in shots[:4]]}
    print(json.dumps(out), flush=True)


def run_noise(args):
    """Noisy simulation (Section 9.5): the grid circuit on --noise-n qubits with single-qubit
    depolarizing noise after every gate, as a density matrix (a vector of 2 x n qubits).
    One step = sv_fuse_density + sv_set_basis + sv_apply_circuit + sv_density_probs to
    host; F_cl and TVD against the noiseless distribution are reported."""
    import torch
    from paper_2604_03816_gb300 import sv
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    dt = sv.SV_C64 if args.dtype == "c64" else sv.SV_C128
    n = args.noise_n
    specs = W.grid_random(n, args.cycles)
    gates = sv.gates_from_specs(specs)
    state = sv.sv_alloc(2 * n, dt, stream=stream)
    k = min(args.k, 4)
    with torch.cuda.stream(stream):
        def step(timing=False):
            c = sv.sv_fuse_density(gates, n, args.p_depol, k)
            sv.sv_set_basis(state, 0)
            rep = sv.sv_apply_circuit(state, c, timing=timing)
            return rep, sv.sv_density_probs(state), len(c)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = []
        with ClockSampler(None) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                rep, pr, nfused = step(timing=True)
                reps.append(rep)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        ideal_state = sv.sv_alloc(n, sv.SV_C128, stream=stream)
        sv.sv_apply_circuit(ideal_state, sv.sv_fuse(gates, n, 4))
        ideal = sv.sv_probs(ideal_state).astype(np.float64)
        ideal_state.free()
    state.free()
    apply_ms = sum(r["apply_ms"] for r in reps)
    abytes = sum(r["bytes"] for r in reps)
    achieved = abytes / (apply_ms / 1000.0) / 1e9
    peak, peak_kind = hbm_peak()
    pr = pr.astype(np.float64)
    out = {"metric": "noisy circuits/s (density matrix, depolarizing after every gate)",
           "value": 1000.0 / ms, "unit": "circuits/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if dt == sv.SV_C64 else "f64", "data": "synthetic",
           "config": {"workload": f"grid_random {n}q depth {args.cycles} with depolarizing "
                                  f"p={args.p_depol} after every gate, density matrix as a "
                                  f"{2 * n}-qubit {args.dtype} vector, fused k={k}",
                      "gates": len(specs), "fused_gates": nfused, "seed": W.seed_for(3, n),
                      "state_bytes": (8 if dt == sv.SV_C64 else 16) << (2 * n),
                      "l2": "state larger than L2, no flush needed"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                        "kernel": "fused-gate passes on the density vector"},
           "result": {"trace": float(pr.sum()),
                      "F_cl_vs_noiseless": float(np.sum(np.sqrt(np.clip(pr, 0, None) * ideal)) ** 2),
                      "TVD_vs_noiseless": float(0.5 * np.sum(np.abs(pr - ideal)))},
           "cpu_baseline": None, "e2e": None,
           "gpu_launches": (reps[-1]["passes"] + 2) * args.steps, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_qft(args):
    """Structure-aware passes and commutation-aware fusion on circuits with diagonal and
    controlled gates: QFT of a seeded basis state (the QFT family of Tables 4 and 7;
    default), a random diagonal-heavy circuit, or QAOA layers.  One step = sv_fuse_ex +
    sv_set_basis + sv_apply_circuit + sv_norm.  Three variants are timed: the paper's
    fusion with every pass dense (SV_POLICY_DENSE_ONLY), the same schedule with the
    structure-aware passes, and commutation-aware fusion (SV_FUSE_COMMUTE) with the
    structure-aware passes; the line's value is the best of the last two."""
    import torch
    from paper_2604_03816_gb300 import sv
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    dt = sv.SV_C64 if args.dtype == "c64" else sv.SV_C128
    n = args.n
    # complex128 gates of width 5 have no tensor-core pass: fuse complex128 at k <= 4
    k = args.k if dt == sv.SV_C64 else min(args.k, 4)
    x = int(np.random.default_rng(W.seed_for(6, n)).integers(0, 1 << n))
    if args.circuit == "qft":
        specs, what = W.qft(n), "QFT (H + controlled phases + final swaps) of a seeded basis state"
    elif args.circuit == "phase_heavy":
        specs, what = W.phase_heavy(n, 16 * n), f"random diagonal-heavy circuit ({16 * n} gates) on a seeded basis state"
    else:
        specs, what = W.qaoa(n, 3, 3 * n), f"QAOA, 3 layers of {3 * n} ZZ phases + RX, on a seeded basis state"
    gates = sv.gates_from_specs(specs)
    state = sv.sv_alloc(n, dt, stream=stream)
    res = {}
    variants = (("dense", sv.SV_POLICY_DENSE_ONLY, 0), ("structure", 0, 0),
                ("structure+commute", 0, sv.SV_FUSE_COMMUTE))
    with torch.cuda.stream(stream):
        for name, policy, flags in variants:
            sv.sv_set_policy(state, policy)

            def step(timing=False):
                c = sv.sv_fuse_ex(gates, n, k, flags)
                sv.sv_set_basis(state, x)
                rep = sv.sv_apply_circuit(state, c, timing=timing)
                return rep, sv.sv_norm(state), len(c)
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = []
            with ClockSampler(None) as clk:
                e0.record(stream)
                for _ in range(args.steps):
                    rep, norm, nfused = step(timing=(policy == 0))
                    reps.append(rep)
                e1.record(stream)
                torch.cuda.synchronize()
            res[name] = (e0.elapsed_time(e1) / args.steps, reps, norm, nfused, clk.summary())
    state.free()
    best = min(("structure", "structure+commute"), key=lambda v: res[v][0])
    ms, reps, norm, nfused, clocks = res[best]
    dense_ms = res["dense"][0]
    apply_ms = sum(r["apply_ms"] for r in reps)
    abytes = sum(r["bytes"] for r in reps)
    dense_bytes = res["dense"][1][-1]["passes"] * 2 * ((8 if dt == sv.SV_C64 else 16) << n)
    achieved = abytes / (apply_ms / 1000.0) / 1e9
    peak, peak_kind = hbm_peak()
    out = {"metric": f"{args.circuit} circuits/s (structure-aware passes)", "value": 1000.0 / ms,
           "unit": "circuits/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if dt == sv.SV_C64 else "f64", "data": "synthetic",
           "config": {"workload": f"{what}, {n}q, {args.dtype}, DAG fusion k={k}, {best}",
                      "gates": len(specs), "fused_gates": nfused, "x": x,
                      "state_bytes": (8 if dt == sv.SV_C64 else 16) << n,
                      "l2": "state larger than L2, no flush needed"},
           "variants_ms_per_step": {v: res[v][0] for v in res},
           "variants_fused_gates": {v: res[v][3] for v in res},
           "speedup_vs_dense": dense_ms / ms,
           "algorithmic_bytes_per_step": abytes / len(reps),
           "dense_bytes_per_step": dense_bytes, "norm": norm,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                        "kernel": "all passes of the schedule; achieved = bytes of the amplitudes "
                                  "the passes touch / their CUDA-event time"},
           "cpu_baseline": None, "e2e": None,
           "gpu_launches": reps[-1]["passes"] + 3, "clocks": clocks}
    print(json.dumps(out), flush=True)


def serve_rates(sv, rates, n_requests, budget_gib=150, slots=16, max_k=5):
    """Poisson arrivals of seeded brickwork circuits (width U{10..30}, depth U{10..60}, 70%
    complex64 / 30% complex128, top-64 outcomes) at each offered rate, n_requests arrivals
    per rate (an arrival window of n_requests / rate seconds), through one server per rate
    under the HBM budget.  Latency = the server's clock from submission to the result.
    Above the server's capacity the queue grows over the window, so p50/p99 there describe
    a burst of n_requests, not a steady state; the achieved circuits/s is the capacity."""
    per_rate = []
    for rate in rates:
        reqs = W.serving_stream(rate, 1e9, max_requests=n_requests)
        arrays = [sv.GateArray(sv.gates_from_specs(r.gates)) for r in reqs]
        srv = sv.sv_server_create(budget_bytes=budget_gib << 30, max_slots=slots, max_k=max_k)
        t0 = time.perf_counter()
        ids = {}
        got = {}
        for r, ga in zip(reqs, arrays):
            while time.perf_counter() - t0 < r.arrival_s:
                for x in sv.sv_server_poll(srv, 256, 0):
                    got[x["id"]] = x
                time.sleep(0.0002)
            ids[sv.sv_server_submit(srv, r.width, 0 if r.dtype == "c64" else 1, ga)] = r
        while len(got) < len(ids):
            for x in sv.sv_server_poll(srv, 256, 20):
                got[x["id"]] = x
        srv.destroy()
        lat = np.array([got[i]["t_done"] - got[i]["t_submit"] for i in ids])
        first = min(got[i]["t_submit"] for i in ids)
        last = max(got[i]["t_done"] for i in ids)
        ok = sum(1 for i in ids if got[i]["status"] == 0)
        per_rate.append({"rate_hz": rate, "requests": len(ids), "ok": ok,
                         "arrival_window_s": reqs[-1].arrival_s,
                         "p50_ms": 1000 * float(np.percentile(lat, 50)),
                         "p99_ms": 1000 * float(np.percentile(lat, 99)),
                         "samples": int(lat.size),
                         "circuits_per_s": len(ids) / (last - first),
                         "c128_share": sum(1 for r in reqs if r.dtype == "c128") / len(reqs)})
    return per_rate


def run_serve(args):
    """The serving workload at every rate of --rates, --requests arrivals each."""
    import torch
    from paper_2604_03816_gb300 import sv
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    with ClockSampler(None) as clk:
        per_rate = serve_rates(sv, [float(r) for r in args.rates.split(",")], args.requests)
    best = max(per_rate, key=lambda d: d["circuits_per_s"])
    out = {"metric": "served circuits/s with p50/p99 latency (Poisson arrivals, 10-30 qubits, "
                     "70% c64 / 30% c128, top-64)",
           "value": best["circuits_per_s"], "unit": "circuits/s", "n_gpus": world,
           "steps": len(per_rate), "warmup": 0, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "mixed f32/f64", "data": "synthetic",
           "config": {"workload": "serving_stream", "budget_gib": 150, "max_slots": 16,
                      "max_k": "5 (complex128 requests of 11+ qubits fused at 4)",
                      "requests_per_rate": args.requests},
           "per_rate": per_rate, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def config_dict(args, ngates, nfused):
    return {"workload": f"grid_random {args.n}q depth {args.cycles} "
                        f"({'sqrtX/sqrtY/sqrtW + fSim(pi/2,pi/6)'}), {args.dtype}, "
                        f"DAG fusion k={args.k}, adaptive c64->c128 at drift 1e-6",
            "n_qubits": args.n, "gates": ngates, "fused_gates": nfused, "max_k": args.k,
            "state_dtype": args.dtype, "state_bytes": (8 if args.dtype == "c64" else 16) << args.n,
            "l2": "state larger than L2 (inputs > 129 MB), no flush needed",
            "host_fusion": "one sv_fuse per step, of the next circuit, on a host thread "
                           "overlapping the current circuit's GPU work",
            "two_gate_passes": bool(getattr(args, "two_gate_passes", False)),
            "seed": W.seed_for(3, args.n)}


def run_batched(args, steps=None, warmup=None):
    """512 hardware-efficient-ansatz circuits (widths U{16,18,20,22}, 6 layers of
    RY RZ + CNOT ladder, complex64), <sum Z_i Z_{i+1}> per circuit.  Per width: one batch,
    fusion width and chunking from the autotuner (tuned once, before timing).  One step =
    fusion of every circuit (sv_fuse for one, sv_fuse_like for the rest; the widest
    width's for the next step overlaps this step's GPU work) + sv_batch_apply per width
    (CUDA-graph replay) + sv_batch_expect per width."""
    import torch
    from paper_2604_03816_gb300 import sv
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    fam = W.hea_batch(args.count)
    widths = sorted({w for w, _ in fam})
    groups = {w: [g for ww, g in fam if ww == w] for w in widths}
    gates = {w: [sv.gates_from_specs(g) for g in groups[w]] for w in widths}
    arrays = {w: [sv.GateArray(g) for g in gates[w]] for w in widths}   # the input circuits
    batches, tune = {}, {}
    import concurrent.futures as cf
    pool = cf.ThreadPoolExecutor(max_workers=max(1, min(16, (os.cpu_count() or 4))))
    with torch.cuda.stream(stream):
        for w in widths:
            batches[w] = sv.sv_batch_alloc(w, sv.SV_C64, len(groups[w]), stream=stream)
            if args.batch_k:
                tune[w] = {"best_k": args.batch_k, "l2_bytes": (8 << w) * len(groups[w]), "ms": {}}
            else:
                tune[w] = sv.sv_batch_tune(batches[w], gates[w][0], 1, 5)

        def fuse_width(w):
            # Algorithm 2 once per width; the other circuits of the family replay its
            # decisions (same qubits, other angles), on host threads (the C calls release
            # the GIL)
            pattern = sv.sv_fuse(arrays[w][0], w, tune[w]["best_k"])
            return [pattern] + list(pool.map(lambda ga: sv.sv_fuse_like(pattern, ga), arrays[w][1:]))

        order = sorted(widths, reverse=True)
        fuser = cf.ThreadPoolExecutor(max_workers=1)
        ahead = [fuser.submit(fuse_width, order[0])]

        def step():
            fuse_s = 0.0
            out = {}
            # widest first: its passes (most of the GPU time) overlap the host work
            # (fusion, matrix tables) of the narrower ones; the widest width of the next
            # step is fused while this step's expectation values are computed
            for w in order:
                t0 = time.perf_counter()
                circs = ahead[0].result() if w == order[0] else fuse_width(w)
                fuse_s += time.perf_counter() - t0
                sv.sv_batch_set_basis(batches[w], 0)
                sv.sv_batch_apply(batches[w], circs, l2_bytes=tune[w]["l2_bytes"],
                                  tile_bits=tune[w].get("tile_bits", 0))
            ahead[0] = fuser.submit(fuse_width, order[0])
            for w in widths:
                xs, zs, cs = W.zz_chain(w)
                out[w] = sv.sv_batch_expect(batches[w], xs, zs, cs)
            return fuse_s, out

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fuse_total = 0.0
        with ClockSampler(None) as clk:
            e0.record(stream)
            for _ in range(steps):
                fs, out = step()
                fuse_total += fs
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ahead[0].result()
        fuser.shutdown(wait=True)
        # the same circuits one by one through sv_apply_circuit (unbatched), for context
        s1 = sv.sv_alloc(max(widths), sv.SV_C64, stream=stream)
        sample = [(w, gates[w][i]) for w in widths for i in range(4)]
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        states = {w: sv.sv_alloc(w, sv.SV_C64, stream=stream) for w in widths}
        f0.record(stream)
        for w, g in sample:
            c = sv.sv_fuse(g, w, tune[w]["best_k"])
            sv.sv_set_basis(states[w], 0)
            sv.sv_apply_circuit(states[w], c)
            xs, zs, cs = W.zz_chain(w)
            sv.sv_expect(states[w], xs, zs, cs)
        f1.record(stream)
        torch.cuda.synchronize()
        unb = len(sample) / (f0.elapsed_time(f1) / 1000.0)
        s1.free()
    value = args.count * steps / (ms / 1000.0)
    out = {"metric": "batched circuits/s (HEA, 16-22 qubits, complex64, <sum ZZ> per circuit)",
           "value": value, "unit": "circuits/s", "n_gpus": world, "steps": steps,
           "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"{args.count} hea circuits, widths {widths}, 6 layers, c64",
                      "per_width": {str(w): {"circuits": len(groups[w]),
                                             "best_k": tune[w]["best_k"],
                                             "l2_chunk_bytes": tune[w]["l2_bytes"],
                                             "tile_bits": tune[w].get("tile_bits", 0),
                                             "tune_ms": tune[w]["ms"]} for w in widths}},
           "host_fusion_s_per_step": fuse_total / steps,
           "unbatched_circuits_per_s": unb,
           "speedup_vs_unbatched": value / unb, "clocks": clk.summary()}
    for b in batches.values():
        b.free()
    for st in states.values():
        st.free()
    return out


def time_config(sv, torch, n, dtype, k, circuits, warmup, cycles=24):
    """One grid_random configuration on its own stream: `circuits` timed circuits after
    `warmup` untimed ones, each sv_fuse (host) + sv_set_basis + sv_apply_circuit (adaptive
    for complex64) + sv_topk(64).  The state is larger than L2 (no flush needed)."""
    stream = torch.cuda.Stream()
    specs = W.grid_random(n, cycles)
    gates = sv.GateArray(sv.gates_from_specs(specs))
    st = sv.sv_alloc(n, dtype, stream=stream)

    def one(timing):
        c = sv.sv_fuse(gates, n, k)
        if sv.sv_info(st)[1] != dtype:
            sv.sv_set_dtype(st, dtype)
        sv.sv_set_basis(st, 0)
        rep = sv.sv_apply_circuit(st, c, adaptive=(dtype == sv.SV_C64), timing=timing)
        sv.sv_topk(st, 64)
        return rep, len(c)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            one(False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(None) as clk:
            e0.record(stream)
            runs = [one(True) for _ in range(circuits)]
            e1.record(stream)
            torch.cuda.synchronize()
    st.free()
    ms = e0.elapsed_time(e1) / circuits
    reps = [r for r, _ in runs]
    apply_ms = sum(r["apply_ms"] for r in reps)
    abytes = sum(r["bytes"] for r in reps)
    achieved = abytes / (apply_ms / 1000.0) / 1e9
    peak, peak_kind = hbm_peak()
    return {"workload": f"grid_random {n}q depth {cycles}", "n_qubits": n,
            "dtype": "c64" if dtype == sv.SV_C64 else "c128", "max_k": k,
            "max_k_used": reps[-1]["max_k_used"], "gates": len(specs),
            "fused_gates": runs[-1][1], "passes_per_circuit": reps[-1]["passes"],
            "paired_passes_per_circuit": reps[-1]["paired_passes"],
            "tensor_core_passes": reps[-1]["tc_passes"], "circuits": circuits,
            "ms_per_circuit": ms, "circuits_per_s": 1000.0 / ms,
            "apply_ms_per_circuit": apply_ms / circuits,
            "fused_gate_hbm_gbs": achieved, "roofline_frac": achieved / peak,
            "peak_gbs": peak, "peak_kind": peak_kind,
            "promotions": sum(r["promotions"] for r in reps),
            "state_bytes": (8 if dtype == sv.SV_C64 else 16) << n, "clocks": clk.summary()}


def run_shard(args, emulate=None, steps=None, warmup=None, quiet=False):
    """One state over all ranks (global-qubit sharding): --n qubits per GPU, so n + g qubits
    on 2^g ranks (weak scaling: the amplitudes per GPU are fixed).  One step = sv_fuse
    (host) + the plan + every segment's passes and every exchange + the FP64 norm (one sum
    over the ranks) + top-64.  Under torchrun every rank is one GPU and the exchanges are
    NCCL send/recv; with --emulate-ranks R the R ranks are threads on one GPU and an
    exchange is a device copy (a check of the path, not of NVLink)."""
    import torch
    from paper_2604_03816_gb300 import sv
    from paper_2604_03816_gb300.shard import (GpuShard, ShardedState, ThreadComm, ThreadHub,
                                              TorchComm)
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dt = sv.SV_C64 if args.dtype == "c64" else sv.SV_C128
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    if emulate is None:
        emulate = args.emulate_ranks
    emulate = emulate if world == 1 else 0
    ranks = emulate if emulate else world
    g = ranks.bit_length() - 1
    if (1 << g) != ranks:
        raise SystemExit("shard: the number of ranks must be a power of two")
    n_total = args.n if emulate else args.n + g
    specs = W.grid_random(n_total, args.cycles)
    gates = sv.GateArray(sv.gates_from_specs(specs))

    def run_rank(r, comm, result):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            shard = GpuShard(n_total - g, dt, stream=stream)
            st = ShardedState(n_total, dt, comm, shard)

            def step():
                c = sv.sv_fuse(gates, n_total, args.k)
                st.set_basis(0)
                rep = st.apply_circuit(c)
                return rep, st.norm(), st.topk(64)
            for _ in range(warmup):
                step()
            torch.cuda.synchronize()
            comm.sum(0.0)                                   # all ranks start together
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bytes0 = st.exchanged_bytes
            for _ in range(steps):
                rep, norm, top = step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            result[r] = {"ms": comm.allgather(ms), "rep": rep, "norm": norm,
                         "exchanged_bytes_per_step": (st.exchanged_bytes - bytes0) / steps}
            shard.free()

    result = {}
    with ClockSampler(None) as clk:
        if emulate:
            import threading
            hub = ThreadHub(ranks)
            errs = []

            def worker(r):
                try:
                    torch.cuda.set_device(local)
                    run_rank(r, ThreadComm(hub, r), result)
                except BaseException as e:     # noqa: BLE001
                    errs.append(e)
                    hub.barrier.abort()
            th = [threading.Thread(target=worker, args=(r,)) for r in range(ranks)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            if errs:
                raise errs[0]
            me = result[0]
        else:
            import torch.distributed as dist
            if world > 1:
                dist.init_process_group("nccl")
                run_rank(rank, TorchComm(), result)
                me = result[rank]
            else:
                class _One:
                    rank, world = 0, 1

                    def sum(self, v):
                        return v

                    def allgather(self, o):
                        return [o]
                run_rank(0, _One(), result)
                me = result[0]
    ms = max(me["ms"])
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return None
    value = steps / (ms / 1000.0)
    out = {"metric": "sharded circuits/s (one state over the ranks, global-qubit sharding)",
           "value": value, "unit": "circuits/s", "n_gpus": world, "steps": steps,
           "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if dt == sv.SV_C64 else "f64", "data": "synthetic",
           "config": {"workload": f"grid_random {n_total}q depth {args.cycles}, {args.dtype}, "
                                  f"fusion k={args.k}, {ranks} ranks x 2^{n_total - g} amplitudes"
                                  + (" (threads on one GPU, exchanges as device copies)" if emulate
                                     else " (one GPU each, NCCL exchanges)"),
                      "ranks": ranks, "local_qubits": n_total - g},
           "passes_per_step": me["rep"]["passes"], "exchanges_per_step": me["rep"]["exchanges"],
           "swap_passes_per_step": me["rep"]["swap_passes"],
           "exchanged_bytes_per_step_per_rank": me["exchanged_bytes_per_step"],
           "norm": me["norm"], "clocks": clk.summary()}
    if not quiet:
        print(json.dumps(out), flush=True)
    return out


def run_extras(args, sv, torch):
    """The rest of the headline metric, measured in the default run after the 30-qubit
    line: the grid circuits at 28 and 33 qubits (complex64) and at 30 and 32 qubits
    (complex128, the width-5 schedule too), short batched, sharded and served summaries."""
    out = {}
    cfgs = [(28, sv.SV_C64, 5, 8, 2), (33, sv.SV_C64, 5, 3, 1), (30, sv.SV_C128, 4, 3, 1),
            (30, sv.SV_C128, 5, 2, 1), (32, sv.SV_C128, 4, 2, 1)]
    out["configs"] = [time_config(sv, torch, n, dt, k, nc, nw) for n, dt, k, nc, nw in cfgs]
    torch.cuda.empty_cache()
    b = run_batched(args, steps=3, warmup=2)
    out["batched"] = {kk: b[kk] for kk in ("metric", "value", "unit", "ms_per_step", "steps",
                                           "warmup", "speedup_vs_unbatched",
                                           "unbatched_circuits_per_s", "clocks")}
    out["batched"]["per_width"] = b["config"]["per_width"]
    torch.cuda.empty_cache()
    with ClockSampler(None) as clk:
        per_rate = serve_rates(sv, [10.0, 100.0], 100)
    shard = {}
    for ranks in (2, 4):
        r = run_shard(args, emulate=ranks, steps=2, warmup=1, quiet=True)
        shard[str(ranks)] = {kk: r[kk] for kk in ("value", "unit", "ms_per_step", "passes_per_step",
                                                  "exchanges_per_step", "swap_passes_per_step",
                                                  "exchanged_bytes_per_step_per_rank", "norm",
                                                  "clocks")}
    out["sharded"] = {"workload": f"grid_random {args.n}q depth {args.cycles}, {args.dtype}, k={args.k}, "
                                  "one state over R ranks run as threads on this GPU (exchanges as "
                                  "device copies; bench.py --mode shard under torchrun uses NCCL "
                                  "between GPUs)", "per_ranks": shard}
    torch.cuda.empty_cache()
    out["serving"] = {"workload": "serving_stream: Poisson arrivals, width U{10..30}, depth "
                                  "U{10..60}, 70% c64 / 30% c128, top-64, 150 GiB budget, 16 slots, "
                                  "fusion k = 5 (complex128 at 4); 100 arrivals per rate "
                                  "(bench.py --mode serve runs 500 per rate)",
                      "per_rate": per_rate, "clocks": clk.summary()}
    return out


# Tile layouts of two-gate passes (SV_POLICY_TWO_GATE_PASSES), as pairs of target sets:
# a contiguous tile, targets among the bank bits, and segments of 1 KiB, 512 B and 256 B.
PAIR_LAYOUTS = [
    ("contiguous L=12", (5, 6, 7, 8, 9), (7, 8, 9, 10, 11)),
    ("bank targets L=12", (0, 1, 2, 6, 7), (2, 3, 4, 9, 10)),
    ("1 KiB segments L=7", (16, 17, 22, 23), (4, 5, 11, 17)),
    ("1 KiB segments, bank targets L=7", (3, 4, 5, 11, 17), (9, 10, 11, 16, 17)),
    ("512 B segments L=6", (5, 11, 17, 23, 27), (4, 5, 10, 11, 16)),
    ("256 B segments L=5", (21, 22, 26, 27), (19, 20, 21, 25, 26)),
]


def run_pairs(args):
    """Two-gate passes per tile layout: 16 random unitaries alternating between the two
    target sets of a layout, applied with SV_POLICY_TWO_GATE_PASSES (8 passes) and one gate
    per pass (16 passes); the best of three timed runs (CUDA events on the state's
    stream, after a warm-up).  The state (--n qubits, complex64) exceeds L2."""
    import torch
    from paper_2604_03816_gb300 import sv
    torch.cuda.set_device(0)
    n = args.n
    rng = np.random.default_rng(W.seed_for(9, n))
    stream = torch.cuda.Stream()
    rows = []
    with torch.cuda.stream(stream):
        s = sv.sv_alloc(n, sv.SV_C64, stream=stream)
        with ClockSampler(None) as clk:
            for name, t0, t1 in PAIR_LAYOUTS:
                specs = [W.GateSpec("unitary", t, (), False, W.haar_unitary(1 << len(t), rng))
                         for t in (t0, t1) * 8]
                c = sv.sv_fuse(sv.gates_from_specs(specs), n, 0)
                row = {"layout": name, "targets": [list(t0), list(t1)]}
                for pol, key in ((sv.SV_POLICY_TWO_GATE_PASSES, "two_gate"), (0, "one_gate")):
                    sv.sv_set_policy(s, pol)
                    sv.sv_set_basis(s, 3)
                    sv.sv_apply_circuit(s, c)
                    best, rep = 1e30, None
                    for _ in range(3):
                        rep = sv.sv_apply_circuit(s, c, timing=True)
                        best = min(best, rep["apply_ms"])
                    row[key + "_ms_per_pass"] = best / rep["passes"]
                    row[key + "_passes"] = rep["passes"]
                row["two_gate_over_two_one_gate"] = row["two_gate_ms_per_pass"] / (2 * row["one_gate_ms_per_pass"])
                rows.append(row)
        s.free()
    print(json.dumps({"metric": "two-gate pass time per tile layout", "n_qubits": n, "dtype": "c64",
                      "unit": "ms per pass", "layouts": rows, "clocks": clk.summary()}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.mode == "batched":
        print(json.dumps(run_batched(args)), flush=True)
        return
    if args.mode == "serve":
        run_serve(args)
        return
    if args.mode == "sample":
        run_sample(args)
        return
    if args.mode == "noise":
        run_noise(args)
        return
    if args.mode == "qft":
        run_qft(args)
        return
    if args.mode == "shard":
        run_shard(args)
        return
    if args.mode == "pairs":
        run_pairs(args)
        return
    rank, world, local = dist_info()
    import torch
    from paper_2604_03816_gb300 import sv
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    dt = sv.SV_C64 if args.dtype == "c64" else sv.SV_C128
    specs = W.grid_random(args.n, args.cycles)
    gates = sv.gates_from_specs(specs)          # gate construction: once, host
    ga = sv.GateArray(gates)
    state = sv.sv_alloc(args.n, dt, stream=stream)
    base_policy = sv.SV_POLICY_TWO_GATE_PASSES if args.two_gate_passes else 0
    sv.sv_set_policy(state, base_policy)
    launches_per_step = [0]
    # Each step fuses one circuit on the host (Algorithm 2) and runs it on the GPU; the
    # fusion of the next circuit runs on a host thread while the GPU works on the current
    # one (ctypes releases the GIL), as a pipelined simulator would.
    fuser = concurrent.futures.ThreadPoolExecutor(max_workers=1)
    next_c = [fuser.submit(sv.sv_fuse, gates, args.n, args.k)]

    def step(timing=False):
        c = next_c[0].result()
        next_c[0] = fuser.submit(sv.sv_fuse, gates, args.n, args.k)
        if sv.sv_info(state)[1] != dt:           # a promotion widened the state last time
            sv.sv_set_dtype(state, dt)
        sv.sv_set_basis(state, 0)
        rep = sv.sv_apply_circuit(state, c, adaptive=True, timing=timing)
        idx, p = sv.sv_topk(state, 64)
        zz = sv.sv_expect(state, [0], [3], [1.0])
        # kernels: passes + the norm after the run (2; a basis start needs none before it,
        # a promotion adds one) + set_basis (1) + top-k (2) + expect (2)
        launches_per_step[0] = rep["passes"] + 2 * (1 + rep["promotions"]) + 1 + 2 + 2
        return rep, len(c), (idx, p, zz)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            rep, nfused, _ = step()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        uuid = None
        try:
            uuid = str(torch.cuda.get_device_properties(local).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            pass
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = []
        with ClockSampler(uuid) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                reps.append(step(timing=True)[0])
            e1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        clocks = clk.summary()

        # dominant kernel: the apply passes, timed with CUDA events on the state's stream
        apply_ms = sum(r["apply_ms"] for r in reps)
        apply_bytes = sum(r["bytes"] for r in reps)
        passes = sum(r["passes"] for r in reps)
        achieved = apply_bytes / (apply_ms / 1000.0) / 1e9
        peak, peak_kind = hbm_peak()
        kinfo = KERNELS[args.dtype]
        sha = kernel_sha(kinfo["files"])
        traffic = None
        if sha.startswith(kinfo["sha256_prefix"]) and args.n == kinfo["n"] and args.k >= 4:
            traffic = kinfo["bytes_per_launch"]

        if sv.sv_info(state)[1] != dt:          # a promotion widened the state: start over
            sv.sv_set_dtype(state, dt)
        # end to end through the C ABI with host buffers: every step copies the initial
        # state in from pinned host memory, fuses its circuit, applies it and writes all 2^n
        # probabilities out to pinned host memory.  --e2e-states states with their own
        # streams are driven by as many host threads (pipelining, as a simulator serving a
        # stream of circuits would run), so one circuit's link transfers overlap another's
        # passes; the timed region is bracketed by CUDA events joined across the streams.
        e2e = None
        if args.e2e_steps > 0:
            npdt = np.complex64 if dt == sv.SV_C64 else np.complex128
            h_in = torch.zeros(1 << args.n, dtype=torch.complex64 if dt == sv.SV_C64
                               else torch.complex128).pin_memory()
            h_in[0] = 1.0
            S = max(1, args.e2e_states)
            h_outs = [torch.empty(1 << args.n, dtype=torch.float32 if dt == sv.SV_C64
                                  else torch.float64).pin_memory() for _ in range(S)]
            h_in_np = h_in.numpy()
            assert h_in_np.dtype == npdt
            streams = [stream] + [torch.cuda.Stream() for _ in range(S - 1)]
            states = [state] + [sv.sv_alloc(args.n, dt, stream=streams[w]) for w in range(1, S)]
            # probabilities leave through a device buffer and the copy engine, so that one
            # state's transfer does not hold the SMs while another's passes run
            for st_, ho in zip(states, h_outs):
                sv.sv_set_policy(st_, sv.SV_POLICY_STAGED_PROBS | base_policy)
                sv.sv_probs(st_, ho.numpy())      # allocates the staging buffer, untimed
            torch.cuda.synchronize()

            import threading
            input_in = [threading.Event() for _ in range(S)]

            def worker(w, nsteps):
                st, out = states[w], h_outs[w].numpy()
                # state w starts once state w-1's first input is in: started together, the
                # states would move in lockstep (all uploading, then all computing at a
                # fraction of the speed) and no transfer would overlap a pass
                if w > 0:
                    input_in[w - 1].wait()
                with torch.cuda.stream(streams[w]):
                    for _ in range(nsteps):
                        if sv.sv_info(st)[1] != dt:
                            sv.sv_set_dtype(st, dt)
                        sv.sv_set_state(st, h_in_np)
                        input_in[w].set()
                        c = sv.sv_fuse(gates, args.n, args.k)
                        sv.sv_apply_circuit(st, c, adaptive=True)
                        sv.sv_probs(st, out)
                input_in[w].set()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(streams[0])
            for w in range(1, S):
                streams[w].wait_event(f0)
            share = [args.e2e_steps // S + (1 if w < args.e2e_steps % S else 0) for w in range(S)]
            with concurrent.futures.ThreadPoolExecutor(max_workers=S) as pool:
                for fut in [pool.submit(worker, w, share[w]) for w in range(S)]:
                    fut.result()
            for w in range(1, S):
                done = torch.cuda.Event()
                done.record(streams[w])
                streams[0].wait_event(done)
            f1.record(streams[0])
            torch.cuda.synchronize()
            e2e_ms = f0.elapsed_time(f1)
            e2e = {"value": world * args.e2e_steps / (e2e_ms / 1000.0), "unit": "circuits/s",
                   "h2d_bytes_per_step": int(h_in_np.nbytes),
                   "d2h_bytes_per_step": int(h_outs[0].numpy().nbytes),
                   "steps": args.e2e_steps, "states_in_flight": S,
                   "includes": "sv_set_state(host pinned) + sv_fuse + sv_apply_circuit + "
                               "sv_probs(host pinned, staged through the copy engine) per step; "
                               f"{S} states in flight on {S} streams (host threads), transfers "
                               "of one overlapping the others' passes"}
            for w in range(1, S):
                states[w].free()
            del h_in, h_outs

        unfused = None
        if not args.no_compare_unfused and world == 1:
            s128 = sv.sv_alloc(args.n, sv.SV_C128, stream=stream)
            cu = sv.sv_fuse(gates, args.n, 0)
            r = sv.sv_apply_circuit(s128, cu, timing=True)
            unfused = {"circuits_per_s": 1000.0 / r["apply_ms"], "passes": r["passes"],
                       "apply_ms": r["apply_ms"],
                       "effective_gbs": r["bytes"] / (r["apply_ms"] / 1000.0) / 1e9}
            s128.free()

    fuser.shutdown(wait=True)
    state.free()
    extras = None
    if world == 1 and not args.no_extras:
        extras = run_extras(args, sv, torch)
    if rank != 0:
        return
    value = job_throughput(world, args.steps, ms)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(specs, args.n, args.cpu_sample_s, len(specs))
    out = {"metric": METRIC, "value": value, "unit": "circuits/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if dt == sv.SV_C64 else "f64", "data": "synthetic",
           "config": config_dict(args, len(specs), nfused),
           "fused_gate_hbm_gbs": achieved,
           "passes_per_circuit": reps[-1]["passes"],
           "paired_passes_per_circuit": reps[-1]["paired_passes"],
           "promotions": sum(r["promotions"] for r in reps),
           "max_drift": max(r["drift"] for r in reps),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": traffic,
                        "kernel": kinfo["kernel"],
                        "traffic_source": kinfo["traffic_source"],
                        "peak_kind": peak_kind,
                        "algorithmic_bytes_per_launch": apply_bytes / passes,
                        "avg_launch_ms": apply_ms / passes},
           "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step[0] * args.steps,
           "clocks": clocks}
    if unfused:
        out["unfused_c128"] = unfused
        out["speedup_vs_unfused_c128"] = value / unfused["circuits_per_s"]
    if extras:
        out.update(extras)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
