"""Seeded graph generators.  Every function returns (row_off, col, truth):

* row_off  int64[n+1]  CSR row offsets of the symmetric adjacency
* col      int32[nnz]  sorted neighbour lists, no self-loops, no duplicates
* truth    int32[n]    the planted community of each vertex

The graphs stand in for the paper's LFR benchmark graphs and single-cell kNN
graphs (Results, "Graphs"); those datasets and networkx are not used here.
"""
from __future__ import annotations

import math

import numpy as np


def csr_from_edges(n: int, u, v):
    """Undirected edge list -> symmetric CSR (self-loops and repeats dropped)."""
    u = np.asarray(u, dtype=np.int64).ravel()
    v = np.asarray(v, dtype=np.int64).ravel()
    keep = u != v
    u, v = u[keep], v[keep]
    key = np.concatenate([u * n + v, v * n + u])
    key.sort()
    if len(key):
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    rows = key // n
    cols = (key - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    row_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_off[1:])
    return row_off, cols


def _pairs_in_block(rng, members, p):
    """Bernoulli(p) edges among the members of one community."""
    s = len(members)
    if s < 2 or p <= 0.0:
        return np.empty(0, np.int64), np.empty(0, np.int64)
    npairs = s * (s - 1) // 2
    if s <= 3000:
        iu, ju = np.triu_indices(s, 1)
        m = rng.random(npairs) < p
        return members[iu[m]], members[ju[m]]
    cnt = rng.binomial(npairs, p)
    a = rng.integers(0, s, cnt)
    b = rng.integers(0, s, cnt)
    return members[a], members[b]


def sbm(sizes, p_in: float, p_out: float, rng):
    """Planted-partition stochastic block model.

    Small graphs (n <= 5000) draw every vertex pair; larger ones draw the
    within-community pairs per community and the between-community edges as a
    binomial number of uniform vertex pairs, rejecting same-community pairs.
    """
    sizes = np.asarray(sizes, dtype=np.int64)
    n = int(sizes.sum())
    truth = np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)
    if n <= 5000:
        iu, ju = np.triu_indices(n, 1)
        same = truth[iu] == truth[ju]
        prob = np.where(same, p_in, p_out)
        m = rng.random(len(iu)) < prob
        row_off, col = csr_from_edges(n, iu[m], ju[m])
        return row_off, col, truth
    starts = np.concatenate([[0], np.cumsum(sizes)])
    us, vs = [], []
    for c in range(len(sizes)):
        members = np.arange(starts[c], starts[c + 1], dtype=np.int64)
        a, b = _pairs_in_block(rng, members, p_in)
        us.append(a)
        vs.append(b)
    n_between = n * (n - 1) // 2 - int((sizes * (sizes - 1) // 2).sum())
    cnt = rng.binomial(n_between, p_out) if p_out > 0 else 0
    a = rng.integers(0, n, cnt)
    b = rng.integers(0, n, cnt)
    keep = truth[a] != truth[b]
    us.append(a[keep])
    vs.append(b[keep])
    row_off, col = csr_from_edges(n, np.concatenate(us), np.concatenate(vs))
    return row_off, col, truth


def _power_law(rng, count, expo, lo, hi):
    """Continuous power law p(x) ~ x^-expo on [lo, hi] by inverse transform."""
    u = rng.random(count)
    a = 1.0 - expo
    return (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)


def _power_law_mean(expo, lo, hi):
    a = 1.0 - expo
    b = 2.0 - expo
    return (a / b) * (hi ** b - lo ** b) / (hi ** a - lo ** a)


def lfr_like(n: int, avg_deg: float, max_deg: int, gamma: float, beta: float,
             cmin: int, cmax: int, mu: float, rng):
    """LFR-style graph whose realised mean degree is ``avg_deg``: dropping
    repeated pairs, self-loops and external pairs inside one community loses
    a few percent of the stubs, so the graph is drawn once, its realised mean
    degree measured, and drawn again from the same generator state with the
    target raised by the lost share (see ``_lfr_draw`` for the model)."""
    state = rng.bit_generator.state
    row_off, col, truth = _lfr_draw(n, avg_deg, max_deg, gamma, beta, cmin, cmax, mu, rng)
    got = len(col) / max(n, 1)
    if got <= 0 or got >= avg_deg:
        return row_off, col, truth
    rng.bit_generator.state = state
    return _lfr_draw(n, min(avg_deg * avg_deg / got, 0.9 * max_deg), max_deg, gamma, beta, cmin, cmax, mu, rng)


def _lfr_draw(n: int, avg_deg: float, max_deg: int, gamma: float, beta: float,
              cmin: int, cmax: int, mu: float, rng):
    """LFR-style benchmark graph built with a configuration model.

    Degrees follow a power law with exponent ``gamma`` on [d_min, max_deg],
    d_min solved so that the mean is ``avg_deg``; community sizes follow a
    power law with exponent ``beta`` on [cmin, cmax].  A vertex of degree d has
    round((1-mu) d) stubs inside its community and the rest outside.  Vertices
    whose internal degree needs a large community are placed first.  Stubs are
    paired at random; self-loops, repeats and (for external stubs) pairs inside
    one community are dropped, so the realised degrees are slightly lower.
    """
    cmax = min(cmax, n)
    cmin = min(cmin, cmax)
    lo, hi = 1.0, float(max_deg)
    for _ in range(100):  # bisection on the lower degree cut-off
        mid = 0.5 * (lo + hi)
        if _power_law_mean(gamma, mid, max_deg) < avg_deg:
            lo = mid
        else:
            hi = mid
    dmin = 0.5 * (lo + hi)
    deg = np.clip(np.rint(_power_law(rng, n, gamma, dmin, max_deg)), 1, max_deg).astype(np.int64)

    sizes = []
    total = 0
    while total < n:
        s = int(round(_power_law(rng, 1, beta, cmin, cmax)[0]))
        s = min(s, n - total)
        if s < cmin and sizes:
            sizes[rng.integers(0, len(sizes))] += s
        else:
            sizes.append(s)
        total += s
    sizes = np.asarray(sizes, dtype=np.int64)
    ncomm = len(sizes)

    din = np.rint((1.0 - mu) * deg).astype(np.int64)
    din = np.minimum(din, int(sizes.max()) - 1)
    free = sizes.copy()
    truth = np.full(n, -1, dtype=np.int64)
    order_c = np.argsort(-sizes, kind="stable")
    sorted_sizes = sizes[order_c]
    big = np.nonzero(din >= cmin - 1)[0]
    big = big[np.argsort(-din[big], kind="stable")]
    for v in big:  # few vertices: place each in a community large enough
        limit = int(np.searchsorted(-sorted_sizes, -(din[v] + 1), side="right"))
        limit = max(limit, 1)
        for _ in range(64):
            c = order_c[rng.integers(0, limit)]
            if free[c] > 0:
                break
        else:
            cand = order_c[:limit][free[order_c[:limit]] > 0]
            c = cand[0] if len(cand) else int(np.argmax(free))
        truth[v] = c
        free[c] -= 1
    rest = np.nonzero(truth < 0)[0]
    slots = np.repeat(np.arange(ncomm, dtype=np.int64), free)
    slots = slots[rng.permutation(len(slots))]
    truth[rest[rng.permutation(len(rest))]] = slots[: len(rest)]
    din = np.minimum(din, sizes[truth] - 1)
    dout = deg - din

    # internal stubs, paired inside each community
    stub_v = np.repeat(np.arange(n, dtype=np.int64), din)
    stub_c = truth[stub_v]
    order = np.lexsort((rng.random(len(stub_v)), stub_c))
    stub_v, stub_c = stub_v[order], stub_c[order]
    cnt = np.bincount(stub_c, minlength=ncomm)
    start = np.concatenate([[0], np.cumsum(cnt)])
    pos = np.arange(len(stub_v)) - start[stub_c]
    usable = pos < (cnt[stub_c] // 2) * 2
    stub_v = stub_v[usable]
    u_in, v_in = stub_v[0::2], stub_v[1::2]

    # external stubs, paired across the whole graph
    ext = np.repeat(np.arange(n, dtype=np.int64), dout)
    ext = ext[rng.permutation(len(ext))]
    ext = ext[: (len(ext) // 2) * 2]
    u_out, v_out = ext[0::2], ext[1::2]
    keep = truth[u_out] != truth[v_out]
    u_out, v_out = u_out[keep], v_out[keep]

    row_off, col = csr_from_edges(n, np.concatenate([u_in, u_out]),
                                  np.concatenate([v_in, v_out]))
    return row_off, col, truth.astype(np.int32)


def knn_mixture(n: int, comps: int, dim: int, knn: int, rng, mean_scale: float = 3.0,
                device: str = "cpu", points_out: list | None = None):
    """Symmetrised exact kNN graph of a Gaussian mixture (single-cell shaped).

    Component weights ~ Dirichlet(1); component c has mean ~ N(0, mean_scale^2 I)
    and covariance s_c^2 I with s_c ~ U[0.5, 2].  The k nearest neighbours are
    found by brute-force squared distances in float32 tiles (torch, on
    ``device``); an edge u-v is kept if either end lists the other.
    ``truth`` is the mixture component.  If ``points_out`` is a list, the points
    (float32 [n, dim]) are appended to it.
    """
    import torch

    w = rng.dirichlet(np.ones(comps))
    truth = rng.choice(comps, size=n, p=w).astype(np.int32)
    means = rng.standard_normal((comps, dim)).astype(np.float32) * mean_scale
    scale = rng.uniform(0.5, 2.0, comps).astype(np.float32)
    x = rng.standard_normal((n, dim)).astype(np.float32)
    x = x * scale[truth][:, None] + means[truth]
    if points_out is not None:
        points_out.append(x)

    dev = torch.device(device)
    X = torch.from_numpy(x).to(dev)
    sq = (X * X).sum(1)
    tile = 2048 if device == "cpu" else 4096
    nbr = torch.empty((n, knn), dtype=torch.int64, device=dev)
    for s in range(0, n, tile):
        e = min(n, s + tile)
        # |x_r - x_u|^2 = |x_r|^2 + |x_u|^2 - 2 x_r.x_u; |x_r|^2 is the same for
        # every u of row r, so ranking |x_u|^2 - 2 x_r.x_u (one fused matmul)
        # gives the same neighbours
        d = torch.addmm(sq[None, :], X[s:e], X.T, beta=1.0, alpha=-2.0)
        d[torch.arange(e - s, device=dev), torch.arange(s, e, device=dev)] = float("inf")
        nbr[s:e] = torch.topk(d, knn, dim=1, largest=False).indices
        del d
    nb = nbr.cpu().numpy()
    del X, sq, nbr
    if dev.type == "cuda":
        torch.cuda.empty_cache()
    u = np.repeat(np.arange(n, dtype=np.int64), knn)
    row_off, col = csr_from_edges(n, u, nb.ravel())
    return row_off, col, truth


def log_uniform_int(rng, lo: float, hi: float, size=None):
    """Integers log-uniform on [lo, hi]."""
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size))).astype(np.int64)
