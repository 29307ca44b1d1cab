"""Benchmark of the consensus sweep on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload lfr|sbm|knn] [--n N] [--k K] [--no-cpu-baseline]

One step = one whole consensus job on resident inputs: reset to the singleton
start (contingency table rebuilt) and synchronous sweeps until no proposal or
20 sweeps.  The metric is (directed edges x input partitions) evaluated per
second: nnz * k per sweep that ran, summed over the step, divided by the step
time (CUDA events on the job's stream).  Prints one JSON line on rank 0.

Multi-GPU: a single job does not shard, so N processes run N independent
replicas of the job (weak scaling, no collective on the data path).

--impl reference times the CPU oracle (the method written out plainly in C,
OpenMP over vertices) on the same workload; each step is its first sweep.
"""
from __future__ import annotations

import argparse
import json
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


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["lfr", "sbm", "knn"], default="lfr")
    p.add_argument("--n", type=int, default=None)
    p.add_argument("--k", type=int, default=None)
    p.add_argument("--max-sweeps", type=int, default=20)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--sweep-mode", type=int, default=0, choices=[0, 1, 2],
                   help="0 automatic, 1 staged deltas, 2 rebuild (identical results)")
    return p.parse_args()


def workload(args, device="cpu"):
    from workloads import make_config

    kw = {}
    if args.n:
        kw["n"] = args.n
    if args.k:
        kw["k"] = args.k
    if args.workload == "knn":
        kw["device"] = device
    return make_config(args.workload, **kw)


def describe(c):
    p = c["params"]
    if c["name"].startswith("lfr"):
        return (f"LFR-style power-law graph n={p['n']}, mean degree {p['avg_deg']}, max degree {p['max_deg']}, "
                f"degree exponent {p['gamma']}, community sizes exponent {p['beta']} in [{p['cmin']},{p['cmax']}], "
                f"mu={p['mu']}; k={p['k']} partitions by merge/split/neighbour-relabel, rho~U{list(p['rho'])}")
    if c["name"].startswith("sbm"):
        return (f"planted-partition SBM n={p['n']} in {p['communities']} communities, p_in={p['p_in']}, "
                f"p_out={p['p_out']}; k={p['k']} perturbed partitions")
    return f"kNN-{p['knn']} graph of a {p['comps']}-component Gaussian mixture in {p['dim']}-D, n={p['n']}; k={p['k']}"


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
                "samples": len(sm)}


def algorithmic_bytes(row_off, col, labels, C):
    """Bytes the proposal step must move for one sweep from state C, per the
    unit costs of the method: CSR offsets and columns, C of each neighbour, the
    vertex's own label row and cluster, the size of each distinct candidate,
    and per distinct candidate (own cluster included) either the member's label
    row (singleton, 4k bytes) or k contingency probes of 12 bytes (8-byte key +
    4-byte count)."""
    n = len(C)
    k = labels.shape[0]
    nnz = len(col)
    deg = np.diff(row_off)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    cu = C[col].astype(np.int64)
    m = (cu != C[src]) & (col != src)
    pairs = np.unique(src[m] * n + cu[m])
    cand = pairs % n
    size = np.bincount(C, minlength=n)
    q = len(pairs)
    single = int((size[cand] == 1).sum())
    own_multi = int((size[C] > 1).sum())
    b = 8 * (n + 1) + 4 * nnz + 4 * nnz + 4 * k * n + 8 * n
    b += 4 * q + single * 4 * k + (q - single) * 12 * k + own_multi * 12 * k
    return int(b), q


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle

    c = workload(args)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    k, n = lab.shape
    nnz = len(col)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.sync_step(ro, col, lab, oracle.singletons(n))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sync_step(ro, col, lab, oracle.singletons(n))
    dt = time.perf_counter() - t0
    value = nnz * k * args.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
           "data": "synthetic", "config": {"workload": c["name"], "description": describe(c), "n": n,
                                            "nnz": nnz, "k": k},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "first synchronous sweep from the singleton start over the whole graph"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline(c):
    """The oracle, as it stands, on the same job: the full run to convergence
    (all host cores via OpenMP)."""
    import oracle

    ro, col, lab = c["row_off"], c["col"], c["labels"]
    k, n = lab.shape
    t0 = time.perf_counter()
    r = oracle.sync_run(ro, col, lab, 20)
    dt = time.perf_counter() - t0
    return {"value": len(col) * k * r.sweeps / dt, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"whole job: {r.sweeps} synchronous sweeps from the singleton start ({dt:.1f} s)"}, r


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2408_11331_gb300 as ccg

    c = workload(args, device=f"cuda:{local}")
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    k, n = lab.shape
    nnz = len(col)
    stream = torch.cuda.Stream()

    opts = ccg.cc_default_options()
    opts.sweep_mode = args.sweep_mode
    job = ccg.Consensus(ro, col, lab, opts)
    job.set_stream(stream.cuda_stream)
    for _ in range(max(args.warmup, 3)):
        job.reset()
        job.run_until_converged(args.max_sweeps)
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
        for _ in range(args.steps):
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
        t = torch.tensor([ms, units], dtype=torch.float64, device="cuda")
        mx = t.clone()
        dist.all_reduce(mx[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        ms, units = float(mx[0]), float(t[1])
    value = units / (ms / 1e3)

    # untimed instrumentation: the start state of every sweep, for the
    # algorithmic bytes of each proposal launch
    job.reset()
    balg = []
    qs = []
    C = job.cluster_ids()
    for _ in range(args.max_sweeps):
        b, q = algorithmic_bytes(ro, col, lab, C)
        info = job.sweep()
        balg.append(b)
        qs.append(q)
        C = job.cluster_ids()
        if info["proposals"] == 0:
            break
    per_step_prop = [float(np.sum(p)) for p in prop_ms]
    prop_total_ms = float(np.mean(per_step_prop))
    n_sw = len(prop_ms[-1])
    achieved = float(np.sum(balg[:n_sw])) / (prop_total_ms / 1e3) / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

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
        t = torch.tensor([e2e_s, e2e_units], dtype=torch.float64, device="cuda")
        mx = t.clone()
        dist.all_reduce(mx[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:], op=dist.ReduceOp.SUM)
        e2e_s, e2e_units = float(mx[0]), float(t[1])

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, ref = cpu_baseline(c)
        job.reset()
        job.run_until_converged(args.max_sweeps)
        if job.history() != ref.stats or not np.array_equal(job.cluster_ids(), ref.C):
            cpu["parity"] = "MISMATCH"
        else:
            cpu["parity"] = "bit-exact (labels, every sweep record)"

    if rank == 0:
        sw = sweeps_total / args.steps
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": c["name"], "description": describe(c), "n": n, "nnz": nnz, "k": k,
                       "sweeps_per_step": sw, "max_sweeps": args.max_sweeps,
                       "step": "reset to singletons + synchronous sweeps until no proposal",
                       "l2": "inputs larger than L2 (CSR + labels + contingency hash > 129 MB), no flush",
                       "parallelism": f"replicas x{world}",
                       "sweep_ms": [round(float(x), 4) for x in sweep_ms[-1]],
                       "propose_ms": [round(float(x), 4) for x in prop_ms[-1]],
                       "distinct_candidates_per_sweep": qs[:n_sw]},
            "e2e": {"value": e2e_units / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(ro.nbytes + col.nbytes + lab.nbytes),
                    "d2h_bytes_per_step": int(4 * n + 8 * 64),
                    "steps": args.e2e_steps, "ms_per_step": 1e3 * e2e_s / args.e2e_steps},
            "roofline": {"kernel": "k_propose", "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "peak_source": peak_src,
                         "algorithmic_bytes_per_step": int(np.sum(balg[:n_sw])),
                         "propose_ms_per_step": prop_total_ms},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    job.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
