"""Named workloads.  Each returns a dict with

* ``row_off`` int64[n+1], ``col`` int32[nnz]  the symmetric graph
* ``labels``  int32[k, n]                     the k input partitions, partition-major
* ``truth``   int32[n]                        the planted communities
* ``name``, ``seed``, ``params``

Seeds are 0x5EED + the workload's index (0 small SBM, 1 LFR-style, 2 kNN,
3 batched mix, 4 served mix); ``seed=`` overrides it.  Sizes can be scaled
down with keyword overrides for tests (``n=...``, ``k=...``).
"""
from __future__ import annotations

import math

import numpy as np

from .graphs import sbm, lfr_like, knn_mixture, log_uniform_int
from .partitions import perturb_many

SEED_BASE = 0x5EED

CONFIG_NAMES = {
    "sbm": 0,     # SBM n=1,000 in 10 communities, p_in=0.1, p_out=0.005, k=10
    "lfr": 1,     # LFR-style n=1,000,000, mean degree 20, k=20
    "knn": 2,     # kNN-15 of a 200-component mixture in 50-D, n=2,000,000, k=50
    "batch": 3,   # 4,096 independent jobs
    "serve": 4,   # Poisson arrivals of jobs
}


def make_sbm(n=1000, communities=10, p_in=0.1, p_out=0.005, k=10, rho=(0.05, 0.3), seed=None):
    seed = SEED_BASE + 0 if seed is None else seed
    rng = np.random.default_rng(seed)
    sizes = [n // communities + (1 if i < n % communities else 0) for i in range(communities)]
    row_off, col, truth = sbm(sizes, p_in, p_out, rng)
    labels = perturb_many(truth, row_off, col, k, rng, rho=rho)
    return dict(name=f"sbm_n{n}_k{k}", seed=seed, row_off=row_off, col=col, labels=labels,
                truth=truth, params=dict(n=n, communities=communities, p_in=p_in, p_out=p_out, k=k,
                                         rho=rho))


def make_lfr(n=1_000_000, avg_deg=20.0, max_deg=1000, gamma=2.5, beta=1.5, cmin=50, cmax=5000,
             mu=0.3, k=20, rho=(0.05, 0.4), seed=None):
    seed = SEED_BASE + 1 if seed is None else seed
    rng = np.random.default_rng(seed)
    row_off, col, truth = lfr_like(n, avg_deg, max_deg, gamma, beta, cmin, cmax, mu, rng)
    labels = perturb_many(truth, row_off, col, k, rng, rho=rho)
    return dict(name=f"lfr_n{n}_k{k}", seed=seed, row_off=row_off, col=col, labels=labels,
                truth=truth, params=dict(n=n, avg_deg=avg_deg, max_deg=max_deg, gamma=gamma,
                                         beta=beta, cmin=cmin, cmax=cmax, mu=mu, k=k, rho=rho))


def graded_partitions(truth, points, comps, row_off, col, k, rng, kmin=50, kmax=2000,
                      relabel=0.10):
    """k partitions at resolutions K ~ log-uniform[kmin, kmax] from mixture components.

    K <= comps: components are grouped at random into K non-empty groups.
    K >  comps: each component is cut into q = ceil(K / comps) parts by rank
    along a random projection, and K exactly is reached by giving q-1 parts to
    comps*q - K randomly chosen components.  Then each vertex, with
    probability ``relabel``, takes the label of a uniformly random neighbour.
    """
    n = len(truth)
    out = np.empty((k, n), dtype=np.int32)
    deg = np.diff(row_off)
    order = np.argsort(truth, kind="stable")
    bounds = np.concatenate([[0], np.cumsum(np.bincount(truth, minlength=comps))])
    for i in range(k):
        K = int(np.clip(log_uniform_int(rng, kmin, kmax), kmin, kmax))
        if K <= comps:
            perm = rng.permutation(comps)
            group = np.empty(comps, dtype=np.int64)
            group[perm[:K]] = np.arange(K)
            group[perm[K:]] = rng.integers(0, K, comps - K)
            lab = group[truth]
        else:
            q = math.ceil(K / comps)
            parts = np.full(comps, q, dtype=np.int64)
            fewer = rng.choice(comps, comps * q - K, replace=False)
            parts[fewer] -= 1
            first = np.concatenate([[0], np.cumsum(parts)])
            direction = rng.standard_normal(points.shape[1]).astype(np.float32)
            proj = points @ direction
            lab = np.empty(n, dtype=np.int64)
            for c in range(comps):
                mem = order[bounds[c]:bounds[c + 1]]
                if len(mem) == 0:
                    continue
                rank = np.empty(len(mem), dtype=np.int64)
                rank[np.argsort(proj[mem], kind="stable")] = np.arange(len(mem))
                lab[mem] = first[c] + (rank * parts[c]) // len(mem)
        pick = (rng.random(n) < relabel) & (deg > 0)
        idx = np.nonzero(pick)[0]
        j = row_off[idx] + np.floor(rng.random(len(idx)) * deg[idx]).astype(np.int64)
        new = lab.copy()
        new[idx] = lab[col[j]]
        out[i] = new
    return out


def make_knn(n=2_000_000, comps=200, dim=50, knn=15, k=50, seed=None, device="cpu"):
    seed = SEED_BASE + 2 if seed is None else seed
    rng = np.random.default_rng(seed)
    pts = []
    row_off, col, truth = knn_mixture(n, comps, dim, knn, rng, device=device, points_out=pts)
    labels = graded_partitions(truth, pts[0], comps, row_off, col, k, rng)
    return dict(name=f"knn_n{n}_k{k}", seed=seed, row_off=row_off, col=col, labels=labels,
                truth=truth, params=dict(n=n, comps=comps, dim=dim, knn=knn, k=k))


def make_job(rng, n, kind, k, mu=None, deg=None):
    """One job of the batched / served mixes (SBM or LFR-style)."""
    if kind == "sbm":
        sizes = []
        total = 0
        while total < n:
            s = int(min(rng.integers(20, 501), n - total))
            sizes.append(s)
            total += s
        d = float(rng.uniform(10, 30)) if deg is None else deg
        r = float(rng.uniform(20, 100))
        s_mean = float(np.mean(sizes))
        # expected degree d = p_in (s-1) + p_out (n-s), with p_in = r p_out
        p_out = d / (r * max(s_mean - 1, 1) + max(n - s_mean, 1))
        p_in = min(1.0, r * p_out)
        row_off, col, truth = sbm(sizes, p_in, p_out, rng)
    else:
        mu = float(rng.uniform(0.1, 0.5)) if mu is None else mu
        d = 20.0 if deg is None else deg
        row_off, col, truth = lfr_like(n, d, int(min(1000, max(n // 10, 2 * d))), 2.5, 1.5,
                                       min(50, n), min(5000, n), mu, rng)
    labels = perturb_many(truth, row_off, col, k, rng, rho=(0.05, 0.3))
    return dict(row_off=row_off, col=col, labels=labels, truth=truth, n=n, k=k, kind=kind)


def batch_job_specs(jobs=4096, nmin=200, nmax=200_000, seed=None):
    """(n, kind, k, seed) of each job in the batched mix: n log-uniform, half SBM
    and half LFR-style, k uniform in [5, 64]."""
    seed = SEED_BASE + 3 if seed is None else seed
    rng = np.random.default_rng(seed)
    ns = log_uniform_int(rng, nmin, nmax, jobs)
    kinds = np.where(np.arange(jobs) % 2 == 0, "sbm", "lfr")
    ks = rng.integers(5, 65, jobs)
    seeds = rng.integers(0, 2 ** 62, jobs)
    return [(int(ns[j]), str(kinds[j]), int(ks[j]), int(seeds[j])) for j in range(jobs)]


def serve_job_specs(jobs=20_000, nmin=1000, nmax=2_000_000, seed=None):
    """(n, k, mean degree, seed) of each job in the served mix (LFR-style)."""
    seed = SEED_BASE + 4 if seed is None else seed
    rng = np.random.default_rng(seed)
    ns = log_uniform_int(rng, nmin, nmax, jobs)
    ks = rng.integers(8, 33, jobs)
    degs = rng.uniform(10, 30, jobs)
    seeds = rng.integers(0, 2 ** 62, jobs)
    return [(int(ns[j]), int(ks[j]), float(degs[j]), int(seeds[j])) for j in range(jobs)]


def poisson_arrivals(count, rate, seed):
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))


def make_config(name: str, **kw):
    if name == "sbm":
        return make_sbm(**kw)
    if name == "lfr":
        return make_lfr(**kw)
    if name == "knn":
        return make_knn(**kw)
    raise ValueError(f"unknown workload {name!r}")
