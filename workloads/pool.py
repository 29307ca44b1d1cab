"""Pools of distinct jobs for the batched and served mixes.

Generating every job of the mixes (4,096 batched jobs with sum n of about
1.2e8; 20,000 served jobs with sum n of about 5e9) on the host takes far
longer than serving them, so a run draws its jobs from a pool: the mix's
specs are sorted by n and cut into P groups of equal count, the middle spec
of each group is generated, and every job of the group uses it.  The n
distribution of the mix is kept to within a group; each drawn job is a
separate job of the batch or request stream (its own vertices, table rows
and results), only its input arrays are shared.

Generation runs in worker processes started with ``spawn`` (safe to call
before or after CUDA is initialised in the parent).
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

from .configs import make_job


def _make(spec):
    n, kind, k, deg, seed = spec
    d = make_job(np.random.default_rng(seed), n, kind, k, deg=deg)
    return d["row_off"], d["col"], d["labels"]


def generate(specs, procs: int | None = None):
    """specs: list of (n, kind, k, deg or None, seed) -> list of (row_off, col, labels)."""
    procs = procs or min(16, os.cpu_count() or 1)
    if procs <= 1 or len(specs) <= 1:
        return [_make(s) for s in specs]
    order = sorted(range(len(specs)), key=lambda i: -specs[i][0])  # largest first
    out = [None] * len(specs)
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        for i, r in zip(order, ex.map(_make, [specs[i] for i in order])):
            out[i] = r
    return out


def quantile_pool(ns, groups: int):
    """Indices of the representative spec of each group and, for every spec,
    the group it belongs to (groups of equal count by n)."""
    ns = np.asarray(ns)
    order = np.argsort(ns, kind="stable")
    groups = max(1, min(groups, len(ns)))
    cuts = np.linspace(0, len(ns), groups + 1).astype(np.int64)
    rep = np.empty(groups, dtype=np.int64)
    member = np.empty(len(ns), dtype=np.int64)
    for g in range(groups):
        idx = order[cuts[g]:cuts[g + 1]]
        rep[g] = idx[len(idx) // 2]
        member[idx] = g
    return rep, member
