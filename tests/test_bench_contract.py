"""bench.py's reference arm runs on the host cores (the oracle), so its JSON
line can be checked here: one line, with every key of the bench contract."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    return json.loads(lines[0])


def _check_common(d):
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_single_job_line():
    d = _run("--workload", "sbm", "--steps", "2", "--warmup", "1")
    _check_common(d)
    assert d["unit"] == "edge-partitions/s" and d["steps"] == 2


@pytest.mark.slow
def test_reference_batch_line():
    d = _run("--workload", "batch", "--jobs", "8", "--pool", "2")
    _check_common(d)
    assert d["unit"] == "jobs/s" and d["config"]["jobs"] == 8


def _bench_module():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def test_single_thread_sample():
    """The single-thread oracle sample beside the all-core baseline."""
    sys.path.insert(0, ROOT)
    from workloads import make_config

    bench = _bench_module()
    c = make_config("sbm")
    s = bench.single_thread_sample(c, target_s=0.01)
    assert s["cores"] == 1 and s["value"] > 0 and s["unit"] == bench.UNIT
    assert "one thread" in s["sample"]


def test_byte_model_counts_candidates():
    """The roofline's algorithmic bytes: distinct (vertex, other cluster)
    pairs over the CSR and the per-candidate unit costs, checked against a
    plain enumeration on a small graph (torch on the CPU)."""
    import numpy as np
    import torch

    sys.path.insert(0, ROOT)
    from workloads import make_config

    bench = _bench_module()
    c = make_config("sbm", n=300, communities=5, k=6, seed=3)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    k, n = lab.shape
    rng = np.random.default_rng(0)
    C = rng.integers(0, 40, n).astype(np.int32)
    C[:40] = np.arange(40)  # every id a vertex of its cluster
    model = bench.ByteModel(torch, ro, col, k, "cpu")
    b, q = model(C)
    pairs = set()
    for v in range(n):
        for e in range(ro[v], ro[v + 1]):
            u = int(col[e])
            if u != v and C[u] != C[v]:
                pairs.add((v, int(C[u])))
    size = np.bincount(C, minlength=n)
    single = sum(1 for _, x in pairs if size[x] == 1)
    own_multi = int((size[C] > 1).sum())
    nnz = len(col)
    want = 8 * (n + 1) + 8 * nnz + 4 * k * n + 8 * n + 4 * len(pairs) + 4 * k * single \
        + 12 * k * (len(pairs) - single) + 12 * k * own_multi
    assert q == len(pairs) and b == want
