"""Benchmark of the consensus sweep on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload all|knn|lfr|sbm|batch|serve] [--n N] [--k K]
                    [--no-cpu-baseline] [--no-extras]

One step = one whole consensus job on resident inputs: reset to the singleton
start (contingency table rebuilt) and synchronous sweeps until no proposal or
20 sweeps.  The metric is (directed edges x input partitions) evaluated per
second: nnz * k per sweep that ran, summed over the step, divided by the step
time (CUDA events on the job's stream).  Prints one JSON line on rank 0.

--workload all (the default): the headline is the largest single-job
workload that fits one GPU, the kNN-15 graph of a 200-component Gaussian
mixture in 50-D (n = 2,000,000, k = 50); the same line carries, under "lfr",
"batch" and "serve", bounded runs of the LFR-style job (n = 1,000,000,
k = 20), of the batched mix and of the served mix (rank 0, one GPU only).

Multi-GPU: a single job does not shard, so N processes run N independent
replicas of the job (weak scaling, no collective on the data path).

--impl reference times the CPU oracle (the method written out plainly in C,
OpenMP over vertices) on the headline workload; each step is its proposal
pass from the singleton start for one block of n/8 vertices (blocks in turn).

--workload batch: the batched form.  4,096 jobs (n log-uniform in
[200, 200000], half SBM and half LFR-style, k uniform in [5, 64]) drawn from a
pool of distinct generated jobs, planned into batches by lane bin and device
budget (cc_plan_batches), each batch one context (cc_batch_create) run to
convergence; metric jobs/s end to end (host inputs in, labels out), next to
the same jobs one at a time through cc_create.  Every job's labels are
compared between the two, and a sample with the oracle.

--workload serve: the served form.  Requests with Poisson arrivals at
multiples of the server's saturated rate, jobs LFR-style (n log-uniform in
[1000, 2000000], mean degree 10-30, k in [8, 32]) drawn from a pool; served
by cc_server (continuous batching) and by a one-job-at-a-time loop on the
same arrivals; p50/p99 latency and jobs/s for each.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sweep (edges x partitions)/s and % HBM roofline; batched jobs/s, p50/p99 latency"
UNIT = "edge-partitions/s"

# DRAM bytes (read + write) of the proposal kernels (k_own, k_edges,
# k_collect) over one step, from ncu captures of those kernels on a smaller
# case of the same workload, scaled by nnz to the full size; reported as
# roofline.traffic while the kernels are the ones captured (empty when they
# changed since).
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the roofline's peak is the measured copy rate)

PROPOSAL_TRAFFIC = {"knn_n2000000_k50": 47.90e9, "lfr_n1000000_k20": 3.648e9}
PROPOSAL_TRAFFIC_SOURCE = {
    "knn_n2000000_k50": "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_own, k_edges, k_collect over one "
                        "run at n=500000 (11.706 GB), scaled by nnz (x4.0921)",
    "lfr_n1000000_k20": "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_own, k_edges, k_collect over one "
                        "run at n=500000 (1.824 GB), scaled by nnz (x2.0002)"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default: enough for about 2 s of timed work, at least 10)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["all", "lfr", "sbm", "knn", "batch", "serve"], default="all")
    p.add_argument("--jobs", type=int, default=None, help="jobs of the batched / served mix (4096 / 20000)")
    p.add_argument("--pool", type=int, default=None, help="distinct generated jobs the mix draws from")
    p.add_argument("--requests", type=int, default=None,
                   help="served form: requests per arrival rate (1000 alone, 400 inside --workload all)")
    p.add_argument("--rates", type=str, default="0.5,0.9,1.5",
                   help="served form: arrival rates as multiples of the server's saturated jobs/s")
    p.add_argument("--budget-frac", type=float, default=0.85, help="share of free device memory for batches")
    p.add_argument("--n", type=int, default=None)
    p.add_argument("--k", type=int, default=None)
    p.add_argument("--max-sweeps", type=int, default=20)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-seconds", type=float, default=20.0,
                   help="bound of the oracle's timed sample (sweeps are added while under it)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="warm-up and timed steps only (for profilers): no e2e, active set, metrics, "
                        "algorithmic bytes, oracle or extra workloads")
    p.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2, 4, 8, 16, 32],
                   help="lanes per scored item (0 automatic; identical results)")
    p.add_argument("--no-regions", action="store_true",
                   help="plain graph nodes instead of conditional regions (for ncu; identical results)")
    p.add_argument("--sweep-mode", type=int, default=0, choices=[0, 1, 2],
                   help="0 automatic, 1 staged deltas, 2 rebuild (identical results)")
    return p.parse_args()


def make_workload(name, args, device="cpu"):
    from workloads import make_config

    kw = {}
    if args.n:
        kw["n"] = args.n
    if args.k:
        kw["k"] = args.k
    if name == "knn":
        kw["device"] = device
    return make_config(name, **kw)


def describe(c):
    p = c["params"]
    if c["name"].startswith("lfr"):
        return (f"LFR-style power-law graph n={p['n']}, mean degree {p['avg_deg']}, max degree {p['max_deg']}, "
                f"degree exponent {p['gamma']}, community sizes exponent {p['beta']} in [{p['cmin']},{p['cmax']}], "
                f"mu={p['mu']}; k={p['k']} partitions by merge/split/neighbour-relabel, rho~U{list(p['rho'])}")
    if c["name"].startswith("sbm"):
        return (f"planted-partition SBM n={p['n']} in {p['communities']} communities, p_in={p['p_in']}, "
                f"p_out={p['p_out']}; k={p['k']} perturbed partitions")
    return (f"symmetrised kNN-{p['knn']} graph of a {p['comps']}-component Gaussian mixture in {p['dim']}-D, "
            f"n={p['n']}; k={p['k']} partitions at resolutions log-uniform in [50, 2000] plus 10% neighbour relabel")


class Clocks:
    """nvidia-smi samples (every 50 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 50):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)  # the first sample precedes the timed work
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "period_ms": self.period_ms}


class ByteModel:
    """Bytes the proposal step must move for one sweep from state C, per the
    unit costs of the method: CSR offsets and columns, C of each neighbour,
    the vertex's own label row and cluster, the size of each distinct
    candidate, and per distinct candidate (own cluster included) either the
    member's label row (singleton, 4k bytes) or k contingency probes of 12
    bytes (8-byte key + 4-byte count).  Counted with torch on the device
    (untimed instrumentation)."""

    def __init__(self, torch, row_off, col, k, device):
        self.torch = torch
        self.n = len(row_off) - 1
        self.k = k
        self.nnz = len(col)
        deg = torch.from_numpy(np.diff(row_off)).to(device)
        self.src = torch.repeat_interleave(torch.arange(self.n, device=device), deg)
        self.col = torch.from_numpy(np.ascontiguousarray(col)).to(device).long()
        self.device = device

    def __call__(self, C_np):
        t = self.torch
        n, k, nnz = self.n, self.k, self.nnz
        C = t.from_numpy(np.ascontiguousarray(C_np)).to(self.device).long()
        cu = C[self.col]
        m = (cu != C[self.src]) & (self.col != self.src)
        pairs = t.unique(self.src[m] * n + cu[m])
        cand = pairs % n
        size = t.bincount(C, minlength=n)
        q = int(pairs.numel())
        single = int((size[cand] == 1).sum())
        own_multi = int((size[C] > 1).sum())
        b = 8 * (n + 1) + 4 * nnz + 4 * nnz + 4 * k * n + 8 * n
        b += 4 * q + single * 4 * k + (q - single) * 12 * k + own_multi * 12 * k
        return int(b), q

    def close(self):
        del self.src, self.col


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle

    name = "knn" if args.workload == "all" else args.workload
    c = make_workload(name, args, device="cuda" if name == "knn" else "cpu")
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    k, n = lab.shape
    nnz = len(col)
    cores = os.cpu_count() or 1
    steps = args.steps or 10
    # one step: the oracle's proposal pass (every vertex's best move, Eq.
    # objective4, against the singleton start) for one block of n / 8
    # vertices, blocks taken in turn, so that a run of K + W steps stays
    # within minutes on the host cores
    blocks = 8
    bounds = [n * b // blocks for b in range(blocks + 1)]
    C0 = oracle.singletons(n)

    def step(s):
        b = s % blocks
        oracle.sync_propose_range(ro, col, lab, C0, bounds[b], bounds[b + 1])
        return float(ro[bounds[b + 1]] - ro[bounds[b]]) * k

    for s in range(args.warmup):
        step(s)
    units = 0.0
    t0 = time.perf_counter()
    for s in range(steps):
        units += step(s)
    dt = time.perf_counter() - t0
    value = units / dt
    sample = (f"proposal pass (best graph-restricted move of every vertex against the singleton start) of one "
              f"block of n/{blocks} vertices per step, blocks in turn; units = the block's CSR entries x k")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
           "data": "synthetic", "config": {"workload": c["name"], "description": describe(c), "n": n,
                                            "nnz": nnz, "k": k},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline(c, job, budget_s):
    """The oracle, as it stands, on the same job (all host cores, OpenMP):
    synchronous sweeps from the singleton start, one at a time, while the
    time taken stays under budget_s (the whole run if it converges first);
    then the GPU's run over the same sweeps is compared with it."""
    import oracle

    ro, col, lab = c["row_off"], c["col"], c["labels"]
    k, n = lab.shape
    C = oracle.singletons(n)
    F = None
    stats = []
    t_total = 0.0
    while len(stats) < 20:
        t0 = time.perf_counter()
        r = oracle.sync_step(ro, col, lab, C, F)
        t_total += time.perf_counter() - t0
        stats.append(r.stats)
        C, F = r.C, r.stats["F"]
        if r.stats["proposals"] == 0 or t_total > budget_s:
            break
    whole = stats[-1]["proposals"] == 0 or len(stats) == 20
    job.reset()
    got = [job.sweep() for _ in range(len(stats))]
    same = got == stats and np.array_equal(job.cluster_ids(), C)
    what = "whole run" if whole else f"first {len(stats)} sweeps"
    return {"value": len(col) * k * len(stats) / t_total, "unit": UNIT, "cores": os.cpu_count() or 1,
            "kind": "oracle", "seconds": round(t_total, 2),
            "sample": f"{what} of the job: {len(stats)} synchronous sweeps from the singleton start, "
                      f"each from the previous one's state",
            "parity": (f"bit-exact ({what}: every sweep record and the raw cluster ids)" if same else "MISMATCH")}, C


def single_thread_sample(c, target_s=1.0):
    """The oracle's proposal pass (every vertex's best move against the
    singleton start) on one host thread, over the first vertices of the job:
    the block doubles from n/256 until it takes target_s or covers n/8."""
    import oracle

    ro, col, lab = c["row_off"], c["col"], c["labels"]
    k, n = lab.shape
    C0 = oracle.singletons(n)
    nb = max(1, n // 256)
    while True:
        t0 = time.perf_counter()
        oracle.sync_propose_range(ro, col, lab, C0, 0, nb, threads=1)
        dt = time.perf_counter() - t0
        if dt >= target_s or nb >= max(1, n // 8):
            break
        nb = min(2 * nb, max(1, n // 8))
    units = float(ro[nb] - ro[0]) * k
    return {"value": units / dt, "unit": UNIT, "cores": 1, "seconds": round(dt, 3),
            "sample": f"proposal pass of vertices [0, {nb}) against the singleton start on one thread; "
                      f"units = their CSR entries x k"}


def over_ranks(dist, seconds, units, device):
    """Whole-job figures of N replicas: the slowest rank's time and the units
    of all ranks (each rank runs its own copy of the job; nothing else is
    exchanged)."""
    import torch

    t = torch.tensor([seconds, units], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
    except OSError:
        p = {}
    return float(p.get("hbm_gbs", 6800.0)), ("measured" if "hbm_gbs" in p else "fallback")


def single_job(args, c, local, dist, rank, world, extras=True):
    """The single-job workload c: warm-up, K timed steps, then (extras) the
    algorithmic bytes, e2e through the C ABI, the active set, the distances
    and the oracle baseline.  Returns the JSON fields of its line."""
    import torch
    import paper_2408_11331_gb300 as ccg

    ro, col, lab = c["row_off"], c["col"], c["labels"]
    k, n = lab.shape
    nnz = len(col)
    stream = torch.cuda.Stream()

    opts = ccg.cc_default_options()
    opts.sweep_mode = args.sweep_mode
    opts.lanes = args.lanes
    opts.no_regions = 1 if args.no_regions else 0
    job = ccg.Consensus(ro, col, lab, opts)
    job.set_stream(stream.cuda_stream)
    warm_ms = []
    for _ in range(max(args.warmup, 3)):
        job.reset()
        job.run_until_converged(args.max_sweeps)
        warm_ms.append(float(np.sum(job.last_run_timing()[0])))
    steps = args.steps or max(10, math.ceil(2000.0 / max(min(warm_ms), 1e-3)))
    launches0 = job.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sweeps_total = 0
    prop_ms = []
    sweep_ms = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(steps):
            job.reset()
            s = job.run_until_converged(args.max_sweeps)
            sweeps_total += s
            a, b = job.last_run_timing()
            sweep_ms.append(a)
            prop_ms.append(b)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = job.launch_count() - launches0
    units = float(nnz) * k * sweeps_total
    if dist:
        ms, units = over_ranks(dist, ms, units, "cuda")
    value = units / (ms / 1e3)
    sw = sweeps_total / steps
    per_step_prop = [float(np.sum(p)) for p in prop_ms]
    prop_total_ms = float(np.mean(per_step_prop))
    n_sw = len(prop_ms[-1])
    peak, peak_src = peaks()
    out = {
        "value": value, "unit": UNIT, "steps": steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / steps,
        "config": {"workload": c["name"], "description": describe(c), "n": n, "nnz": nnz, "k": k,
                   "sweeps_per_step": sw, "max_sweeps": args.max_sweeps,
                   "step": "reset to singletons + synchronous sweeps until no proposal",
                   "l2": "inputs larger than L2 (CSR + labels + contingency hash > 129 MB), no flush",
                   "parallelism": f"replicas x{world}",
                   "timed_s": round(ms / 1e3, 3),
                   "sweep_ms": [round(float(x), 4) for x in sweep_ms[-1]],
                   "propose_ms": [round(float(x), 4) for x in prop_ms[-1]]},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if not extras:
        job.close()
        return out

    # untimed instrumentation: the start state of every sweep, for the
    # algorithmic bytes of each proposal launch
    model = ByteModel(torch, ro, col, k, f"cuda:{local}")
    job.reset()
    balg, qs = [], []
    for _ in range(args.max_sweeps):
        b, q = model(job.cluster_ids())
        info = job.sweep()
        balg.append(b)
        qs.append(q)
        if info["proposals"] == 0:
            break
    model.close()
    out["config"]["distinct_candidates_per_sweep"] = qs[:n_sw]
    achieved = float(np.sum(balg[:n_sw])) / (prop_total_ms / 1e3) / 1e9
    traffic = PROPOSAL_TRAFFIC.get(c["name"])
    out["roofline"] = {
        "kernel": "proposal step (k_own + k_edges + k_collect, one launch each per sweep)",
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
        "traffic": traffic,
        "achieved_kind": "algorithmic: unit-cost bytes of the method per step / proposal-kernel time",
        "dram_achieved": (traffic / (prop_total_ms / 1e3) / 1e9) if traffic else None,
        "dram_frac": (traffic / (prop_total_ms / 1e3) / 1e9 / peak) if traffic else None,
        "traffic_source": PROPOSAL_TRAFFIC_SOURCE.get(c["name"]),
        "peak_source": peak_src,
        "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
        "algorithmic_bytes_per_step": int(np.sum(balg[:n_sw])),
        "propose_ms_per_step": prop_total_ms}

    # end to end through the C ABI with host buffers (pinned), copies inside
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    ro_h, col_h, lab_h = pin(ro), pin(col), pin(lab)
    out_h = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    e2e_sweeps = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        j2 = ccg.Consensus(ro_h, col_h, lab_h, opts)
        e2e_sweeps += j2.run_until_converged(args.max_sweeps)
        ccg._native.cc_consensus_labels(j2._ctx, n, out_h)
        j2.close()
    e2e_s = time.perf_counter() - t0
    e2e_units = float(nnz) * k * e2e_sweeps
    if dist:
        e2e_s, e2e_units = over_ranks(dist, e2e_s, e2e_units, "cuda")
    out["e2e"] = {"value": e2e_units / e2e_s, "unit": UNIT,
                  "h2d_bytes_per_step": int(ro.nbytes + col.nbytes + lab.nbytes),
                  "d2h_bytes_per_step": int(4 * n + 8 * 64),
                  "steps": args.e2e_steps, "ms_per_step": 1e3 * e2e_s / args.e2e_steps,
                  "what": "cc_create from pinned host arrays, run to convergence, labels to the host, destroy"}

    # the same job with the active set (cc_options.active_set): sweeps after
    # the first re-score only vertices near clusters that changed, so fewer
    # edges are evaluated; reported beside the headline, not in it
    opts_a = ccg.cc_default_options()
    opts_a.sweep_mode = args.sweep_mode
    opts_a.lanes = args.lanes
    opts_a.active_set = 1
    opts_a.no_regions = opts.no_regions
    with ccg.Consensus(ro, col, lab, opts_a) as ja:
        ja.set_stream(stream.cuda_stream)
        for _ in range(3):
            ja.reset()
            ja.run_until_converged(args.max_sweeps)
        torch.cuda.synchronize()
        ev2 = torch.cuda.Event(enable_timing=True)
        ev3 = torch.cuda.Event(enable_timing=True)
        reps = min(steps, 10)
        ev2.record(stream)
        for _ in range(reps):
            ja.reset()
            ja.run_until_converged(args.max_sweeps)
        ev3.record(stream)
        torch.cuda.synchronize()
        ms_a = ev2.elapsed_time(ev3) / reps
        hist_a = ja.history()
        sw_a = [round(float(x), 4) for x in ja.last_run_timing()[0]]
    job.reset()
    job.run_until_converged(args.max_sweeps)
    out["active_set"] = {"ms_per_step": ms_a, "speedup": (ms / steps) / ms_a, "sweep_ms": sw_a,
                         "same_result": hist_a == job.history(),
                         "note": "cc_options.active_set = 1: after a run's first sweep, a vertex whose cluster and "
                                 "previous target did not change scores only its candidates whose cluster changed; "
                                 "fewer edges evaluated, identical results"}

    # the two variants of the method (options that change the results; their
    # parity with the oracle is tested at smaller sizes), one timed run each
    # beside the synchronous run's F and sweeps
    F_sync = int(job.objective())
    variants = {"synchronous": {"F": F_sync, "sweeps": len(job.history()), "ms_per_run": ms / steps}}
    for name in ("colour_batched", "empty_moves"):
        ov = ccg.cc_default_options()
        setattr(ov, name, 1)
        ov.no_regions = opts.no_regions
        with ccg.Consensus(ro, col, lab, ov) as jv:
            jv.set_stream(stream.cuda_stream)
            jv.run_until_converged(args.max_sweeps)
            jv.reset()
            torch.cuda.synchronize()
            ev4 = torch.cuda.Event(enable_timing=True)
            ev5 = torch.cuda.Event(enable_timing=True)
            ev4.record(stream)
            jv.run_until_converged(args.max_sweeps)
            ev5.record(stream)
            torch.cuda.synchronize()
            Fv = int(jv.objective())
            variants[name] = {"F": Fv, "sweeps": len(jv.history()), "ms_per_run": ev4.elapsed_time(ev5),
                              "F_over_synchronous": Fv / F_sync if F_sync else None}
    variants["note"] = ("colour_batched: colour classes of a greedy colouring run in turn, each class's moves "
                        "applied before the next proposes; empty_moves: a vertex may also move into a new "
                        "cluster of its own")
    out["variants"] = variants

    # partition distances of the consensus to each input partition (Methods,
    # Evaluation metrics), timed on the host around a synchronous call
    job.metrics()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    met = job.metrics()
    metrics = {"ms": 1e3 * (time.perf_counter() - t0),
               "what": "Mirkin, split-join, Rand distance and VI to each of the k partitions "
                       "(table rebuild + 3 reduction kernels, host-timed, synchronous)",
               "mean_rand_distance": float(np.mean(met["rand_distance"])), "mean_vi": float(np.mean(met["vi"]))}

    # grouping homogeneous partitions: the k x k distances between the input
    # partitions (each partition made the consensus in turn, then restored)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pdist = job.partition_distances()
    grouping = {"ms": 1e3 * (time.perf_counter() - t0),
                "what": f"{k} x {k} split-join / Mirkin / Rand / VI distances between the input partitions",
                "split_join_median": float(np.median(pdist["split_join"][np.triu_indices(k, 1)]))}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        cpu, _ = cpu_baseline(c, job, args.cpu_seconds)
        cpu["single_thread"] = single_thread_sample(c)
        job.reset()
        job.run_until_converged(args.max_sweeps)
        C_gpu = job.cluster_ids()
        t0 = time.perf_counter()
        om = oracle.metrics(lab, C_gpu)
        metrics["oracle_ms"] = 1e3 * (time.perf_counter() - t0)
        t0 = time.perf_counter()
        row0 = oracle.metrics(lab, lab[0])
        grouping["oracle_ms_row0"] = 1e3 * (time.perf_counter() - t0)
        grouping["oracle_ms_estimate"] = grouping["oracle_ms_row0"] * k
        grouping["parity_row0"] = "exact" if np.array_equal(row0["split_join"], pdist["split_join"][0]) and \
            np.array_equal(row0["mirkin"], pdist["mirkin"][0]) else "MISMATCH"
        metrics["parity"] = ("exact Mirkin and split-join, VI within %.1e" % float(np.max(np.abs(om["vi"] - met["vi"])))
                             if np.array_equal(om["mirkin"], met["mirkin"]) and np.array_equal(om["split_join"],
                                                                                                 met["split_join"])
                             else "MISMATCH")
    out["metrics"] = metrics
    out["grouping"] = grouping
    out["cpu_baseline"] = cpu
    job.close()
    return out


def autotune_record(ccg):
    """Lane counts the library's autotuner chose per lane bin (k 1..10,
    11..20, 21..40, 41..80, 81..160, above; 0: not tuned)."""
    import ctypes

    rec = (ctypes.c_int32 * 6)()
    ccg._native._check(ccg._native.lib.cc_autotune_record(6, rec), None)
    return {b: int(rec[i]) for i, b in enumerate(["1-10", "11-20", "21-40", "41-80", "81-160", "161-"]) if rec[i]}


def mix_pool(args, kind):
    """Specs of the batched / served mix, the pool job each spec draws, and the pool."""
    from workloads.configs import batch_job_specs, serve_job_specs
    from workloads.pool import generate, quantile_pool

    if kind == "batch":
        specs = batch_job_specs(args.jobs or 4096)
        rep, member = quantile_pool([s[0] for s in specs], args.pool or 256)
        gen = [(specs[r][0], specs[r][1], specs[r][2], None, specs[r][3]) for r in rep]
    else:
        specs = serve_job_specs(args.jobs or 20000)
        rep, member = quantile_pool([s[0] for s in specs], args.pool or 48)
        gen = [(specs[r][0], "lfr", specs[r][1], specs[r][2], specs[r][3]) for r in rep]
    t0 = time.perf_counter()
    pool = generate(gen)
    return specs, member, pool, time.perf_counter() - t0


def mix_config(kind, specs, member, pool, gen_s):
    ns = np.array([len(pool[m][0]) - 1 for m in member])
    return {"workload": f"{kind}_mix_{len(specs)}", "jobs": len(specs), "pool_distinct_jobs": len(pool),
            "sum_n": int(ns.sum()), "median_n": float(np.median(ns)),
            "draw": "specs sorted by n, cut into equal-count groups; each group's middle spec generated once",
            "generation_s": round(gen_s, 1)}


def run_batch(args, world, local, specs, member, pool, gen_s):
    import torch

    torch.cuda.set_device(local)
    import paper_2408_11331_gb300 as ccg

    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    pool = [tuple(pin(a) for a in job) for job in pool]
    J = len(specs)
    jobs = [pool[m] for m in member]
    sizes = [(len(ro) - 1, len(col), lab.shape[0]) for ro, col, lab in jobs]
    opts = ccg.cc_default_options()
    opts.active_set = 1  # jobs/s: re-score only the active set (identical results)
    opts.autotune = 1    # lanes per item timed per lane bin on its first context (identical results)
    budget = int(torch.cuda.mem_get_info()[0] * args.budget_frac)
    batch_of, nb = ccg._native.cc_plan_batches(sizes, budget, 0, opts)
    waves = [[] for _ in range(nb)]
    for j, b in enumerate(batch_of):
        waves[b].append(j)
    units = 0.0

    def batched(record=None):
        nonlocal units
        dev_ms = 0.0
        for w in waves:
            with ccg.ConsensusBatch([jobs[j] for j in w], opts) as b:
                b.run_until_converged(args.max_sweeps)
                lab = b.consensus_labels()
                dev_ms += float(np.sum(b.last_run_timing()[0]))
                if record is not None:
                    for i, j in enumerate(w):
                        record[j] = lab[b.offsets[i]:b.offsets[i + 1]]
                        units += float(sizes[j][1]) * sizes[j][2] * b.sweeps(i)
        return dev_ms

    def plain(record=None):
        for j in range(J):
            with ccg.Consensus(*jobs[j], opts) as c:
                c.run_until_converged(args.max_sweeps)
                lab = c.consensus_labels()
                if record is not None:
                    record[j] = lab

    # warm-up: the first batch (code paths, pool of the CUDA allocator)
    small = waves[0][:64]
    for _ in range(max(args.warmup, 3)):
        with ccg.ConsensusBatch([jobs[j] for j in small], opts) as b:
            b.run_until_converged(args.max_sweeps)
            b.consensus_labels()
        with ccg.Consensus(*jobs[small[0]], opts) as c:
            c.run_until_converged(args.max_sweeps)
    steps = 1
    got = {}
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        dev_ms = batched(got)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
    ref = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain(ref)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    same = all(np.array_equal(got[j], ref[j]) for j in range(J))
    # the oracle on the smallest distinct jobs of the pool
    import oracle

    # the distinct pool jobs from the smallest up: at least 8, then more while
    # under 15 s of oracle time
    by_size = sorted(range(len(pool)), key=lambda i: len(pool[i][0]))
    first = {int(m): j for j, m in reversed(list(enumerate(member)))}
    ok_oracle = True
    checked = 0
    t_or = time.perf_counter()
    for i in by_size:
        if checked >= 8 and time.perf_counter() - t_or > 15.0:
            break
        ro, col, lab = pool[i]
        r = oracle.sync_run(ro, col, lab, args.max_sweeps)
        ok_oracle &= bool(np.array_equal(got[first[i]], oracle.renumber(r.C)))
        checked += 1
    largest_checked = len(pool[by_size[checked - 1]][0]) - 1
    cfg = mix_config("batch", specs, member, pool, gen_s)
    cfg.update({"batches": nb, "jobs_per_batch": [len(w) for w in waves], "budget_bytes": budget,
                "planner": "cc_plan_batches: lane bins of k, then batches within the device budget",
                "options": "active_set = 1, autotune = 1 in both arms",
                "autotune_lanes_by_bin": autotune_record(ccg),
                "l2": "inputs larger than L2, no flush"})
    return {"metric": "batched jobs/s", "value": J / tb, "unit": "jobs/s", "n_gpus": world, "steps": steps,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * tb, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": cfg,
            "e2e": {"value": J / tb, "unit": "jobs/s", "h2d_bytes_per_step": int(sum(
                a.nbytes for ro, col, lab in jobs for a in (ro, col, lab))), "d2h_bytes_per_step": int(4 * sum(
                    s_[0] for s_ in sizes))},
            "device_ms_per_step": dev_ms,
            "edge_partitions_per_s": units / tb,
            "plain_loop": {"value": J / tp, "unit": "jobs/s", "ms": 1e3 * tp,
                           "how": "each job alone: cc_create, run, labels, destroy"},
            "speedup_vs_plain_loop": tp / tb,
            "parity": ("bit-exact per job vs one-at-a-time" if same else "MISMATCH") +
                      (f"; oracle bit-exact on the {checked} smallest distinct pool jobs (n up to "
                       f"{largest_checked})" if ok_oracle else "; oracle sample MISMATCH"),
            "clocks": clk.summary()}


def run_serve(args, world, local, specs, member, pool, gen_s, requests):
    import torch

    torch.cuda.set_device(local)
    import paper_2408_11331_gb300 as ccg
    from workloads.configs import poisson_arrivals

    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    pool = [tuple(pin(a) for a in job) for job in pool]
    R = min(requests, len(member))
    req = [int(m) for m in member[:R]]
    opts = ccg.cc_default_options()
    opts.active_set = 1  # jobs/s: re-score only the active set (identical results)
    opts.autotune = 1    # lanes per item timed per lane bin on its first context (identical results)

    def solo(i):
        with ccg.Consensus(*pool[i], opts) as c:
            c.run_until_converged(args.max_sweeps)
            return c.consensus_labels()

    # reference labels of every pool job, and warm-up
    ref = {}
    for i in sorted(set(req)):
        ref[i] = solo(i)
    # service rate of the one-job-at-a-time loop
    probe = req[: min(R, 200)]
    t0 = time.perf_counter()
    for i in probe:
        solo(i)
    mu = len(probe) / (time.perf_counter() - t0)

    def serve_server(arr):
        lat = np.zeros(R)
        with ccg.Server(max_active=8, max_batch_jobs=256, options=opts) as srv:
            tick = {}
            nxt = 0
            bad = 0
            t0 = time.perf_counter()
            left = R
            while left:
                now = time.perf_counter() - t0
                while nxt < R and arr[nxt] <= now:
                    tick[srv.submit(*pool[req[nxt]])] = nxt
                    nxt += 1
                done, _ = srv.progress(wait=nxt >= R)
                now = time.perf_counter() - t0
                for t in done:
                    r = tick[t]
                    lat[r] = now - arr[r]
                    res = srv.result(t, pop=True)
                    bad += int(res["status"] != 0 or not np.array_equal(res["labels"], ref[req[r]]))
                    left -= 1
            span = time.perf_counter() - t0
            st = srv.stats()
        return lat, span, bad, st

    def serve_plain(arr):
        lat = np.zeros(R)
        t0 = time.perf_counter()
        for r in range(R):
            now = time.perf_counter() - t0
            if arr[r] > now:
                time.sleep(arr[r] - now)
            solo(req[r])
            lat[r] = time.perf_counter() - t0 - arr[r]
        return lat, time.perf_counter() - t0

    results = []
    with Clocks(local) as clk:
        # saturated throughput of the server: every request waiting at t = 0
        _, sat_span, sat_bad, _ = serve_server(np.zeros(R))
        sat = R / sat_span
        rates = [float(x) * sat for x in args.rates.split(",")]
        for q, rate in enumerate(rates):
            arr = poisson_arrivals(R, rate, 0x5EED + 4 + q)
            lat, span, bad, st = serve_server(arr)
            plat, pspan = serve_plain(arr)
            results.append({
                "rate_jobs_per_s": rate, "rate_vs_saturated": rate / sat,
                "served": {"jobs_per_s": R / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                           "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mismatches": bad,
                           "contexts": st["batches"], "max_in_flight": st["max_in_flight"],
                           "loaded_into_running_contexts": st["admitted_running"],
                           "peak_bytes": st["peak_bytes"]},
                "plain": {"jobs_per_s": R / pspan, "p50_ms": 1e3 * float(np.percentile(plat, 50)),
                          "p99_ms": 1e3 * float(np.percentile(plat, 99))}})
    top = results[-1]
    cfg = mix_config("serve", specs, member[:R], pool, gen_s)
    cfg.update({"requests_per_rate": R, "arrivals": "Poisson, seeds 0x5EED + 4 + rate index",
                "plain_service_rate_jobs_per_s": mu, "server_saturated_jobs_per_s": sat,
                "rates": "0.5, 0.9, 1.5 x the server's saturated jobs/s (all requests waiting at t = 0)",
                "server": "cc_server max_active 8, max_batch_jobs 256; jobs released as they stop, waiting jobs "
                          "loaded into finished places of running contexts",
                "options": "active_set = 1, autotune = 1 in both arms",
                "autotune_lanes_by_bin": autotune_record(ccg)})
    return {"metric": "served jobs/s, p50/p99 latency", "value": top["served"]["jobs_per_s"], "unit": "jobs/s",
            "n_gpus": world, "steps": len(rates), "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": cfg, "rates": results,
            "parity": "bit-exact per request vs the job alone" if sat_bad == 0 and all(
                r["served"]["mismatches"] == 0 for r in results) else "MISMATCH",
            "clocks": clk.summary()}


def run_mix_reference(args, rank, kind, specs, member, pool, gen_s):
    """The oracle on the mix's jobs in order, for a bounded time (about 20 s)."""
    if rank != 0:
        return
    import oracle

    t0 = time.perf_counter()
    done = 0
    for m in member:
        ro, col, lab = pool[m]
        oracle.sync_run(ro, col, lab, args.max_sweeps)
        done += 1
        if time.perf_counter() - t0 > 20.0:
            break
    dt = time.perf_counter() - t0
    cfg = mix_config(kind, specs, member, pool, gen_s)
    unit = "jobs/s"
    out = {"impl": "reference", "metric": "batched jobs/s" if kind == "batch" else "served jobs/s, p50/p99 latency",
           "value": done / dt, "unit": unit, "n_gpus": args.gpus, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * dt,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
           "config": cfg,
           "cpu_baseline": {"value": done / dt, "unit": unit, "cores": os.cpu_count() or 1, "kind": "oracle",
                            "sample": f"first {done} jobs of the mix in order, whole runs ({dt:.1f} s)"},
           "e2e": {"value": done / dt, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def compact(part):
    """The summary of an extra single-job workload kept in the headline line."""
    keep = ("value", "unit", "ms_per_step", "steps", "roofline", "e2e", "cpu_baseline", "active_set", "variants",
            "clocks", "gpu_launches")
    d = {key: part.get(key) for key in keep}
    d["workload"] = part["config"]["workload"]
    d["description"] = part["config"]["description"]
    d["config"] = {key: part["config"][key] for key in ("n", "nnz", "k", "sweeps_per_step", "sweep_ms",
                                                          "propose_ms") if key in part["config"]}
    return d


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload in ("batch", "serve"):
        if rank != 0:
            return
        specs, member, pool, gen_s = mix_pool(args, args.workload)
        if args.impl == "reference":
            return run_mix_reference(args, rank, args.workload, specs, member, pool, gen_s)
        if args.workload == "batch":
            out = run_batch(args, world, local, specs, member, pool, gen_s)
        else:
            out = run_serve(args, world, local, specs, member, pool, gen_s, args.requests or 1000)
        print(json.dumps(out), flush=True)
        return
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2408_11331_gb300  # noqa: F401  (fails loudly without libcc.so)

    name = "knn" if args.workload == "all" else args.workload
    extras = not args.no_extras
    c = make_workload(name, args, device=f"cuda:{local}")
    head = single_job(args, c, local, dist, rank, world, extras=extras)
    del c
    line = {"metric": METRIC, "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic"}
    line.update(head)
    if args.workload == "all" and extras and world == 1 and rank == 0:
        c = make_workload("lfr", argparse.Namespace(n=None, k=None))
        line["lfr"] = compact(single_job(args, c, local, None, rank, world))
        del c
        specs, member, pool, gen_s = mix_pool(args, "batch")
        line["batch"] = run_batch(args, world, local, specs, member, pool, gen_s)
        del pool
        specs, member, pool, gen_s = mix_pool(args, "serve")
        line["serve"] = run_serve(args, world, local, specs, member, pool, gen_s, args.requests or 400)
        del pool
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
