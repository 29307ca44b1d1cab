"""Input partitions made from planted labels.

The paper builds its input partitions with Louvain runs and other community
detection algorithms (Results, "Input partitions"); those are not available
here.  The stand-in perturbs the planted partition in three steps, applied in
this order (the order and the snapshot relabel are a reading; the workload
description only names the three operations):

1. merge   for each community in id order, with probability ``p_merge`` it is
           united with a uniformly random other community (union-find; the
           united label is the smaller id);
2. split   for each original community, with probability ``p_split`` its
           members are shuffled and one half gets a fresh label;
3. relabel with probability rho ~ U[rho_lo, rho_hi] (drawn once per partition)
           a vertex takes the label, in the partition after step 2, of a
           uniformly random neighbour; isolated vertices keep theirs.
"""
from __future__ import annotations

import numpy as np


def _find(parent, x):
    while parent[x] != x:
        parent[x] = parent[parent[x]]
        x = parent[x]
    return x


def perturb(truth, row_off, col, rng, p_merge=0.2, p_split=0.2, rho=(0.05, 0.3)):
    truth = np.asarray(truth, dtype=np.int64)
    n = len(truth)
    K = int(truth.max()) + 1 if n else 0
    parent = list(range(K))
    for c in range(K):
        if K > 1 and rng.random() < p_merge:
            o = int(rng.integers(0, K - 1))
            o = o + 1 if o >= c else o
            ra, rb = _find(parent, c), _find(parent, o)
            if ra != rb:
                lo, hi = min(ra, rb), max(ra, rb)
                parent[hi] = lo
    root = np.asarray([_find(parent, c) for c in range(K)], dtype=np.int64)
    lab = root[truth] if K else truth.copy()

    order = np.argsort(truth, kind="stable")
    bounds = np.concatenate([[0], np.cumsum(np.bincount(truth, minlength=K))])
    fresh = K
    for c in range(K):
        if rng.random() < p_split:
            members = order[bounds[c]:bounds[c + 1]]
            if len(members) >= 2:
                members = members[rng.permutation(len(members))]
                lab[members[: len(members) // 2]] = fresh
                fresh += 1

    r = rng.uniform(rho[0], rho[1])
    deg = np.diff(row_off)
    pick = (rng.random(n) < r) & (deg > 0)
    idx = np.nonzero(pick)[0]
    j = row_off[idx] + np.floor(rng.random(len(idx)) * deg[idx]).astype(np.int64)
    out = lab.copy()
    out[idx] = lab[col[j]]
    return out.astype(np.int32)


def perturb_many(truth, row_off, col, k: int, rng, **kw):
    """k independent perturbations, stacked partition-major as int32[k, n]."""
    return np.stack([perturb(truth, row_off, col, rng, **kw) for _ in range(k)])
