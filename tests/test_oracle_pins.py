"""Pins of the CPU oracle to things other than itself (no GPU).

Each test names what fixes the expected value: a hand-worked example in
tests/golden/, pair enumeration, a library routine, brute force over all set
partitions, an algebraic identity, or an invariance of the method.
"""
import json
import os

import numpy as np
import pytest

import oracle
from workloads import csr_from_edges, make_config

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _random_case(rng, n, k, nlab, nclu):
    labels = rng.integers(-5, nlab - 5, size=(k, n)).astype(np.int32)
    # consensus ids must be vertex ids; pick one representative per class
    cls = rng.integers(0, nclu, n)
    C = np.empty(n, np.int32)
    for c in np.unique(cls):
        mem = np.nonzero(cls == c)[0]
        C[mem] = rng.choice(mem)
    return labels, C


def _random_graph(rng, n, p):
    iu, ju = np.triu_indices(n, 1)
    m = rng.random(len(iu)) < p
    return csr_from_edges(n, iu[m], ju[m])


# ----------------------------------------------------------------- P1: F


def test_mirkin_hand_examples():
    """Appendix Eq. distance: hand-counted symmetric differences of pair sets."""
    for case in _golden("mirkin_examples.json")["cases"]:
        X = np.array(case["X"], np.int32)
        Y = np.array(case["Y"], np.int32)
        assert oracle.mirkin_pairs(X, Y) == case["ordered"]
        assert oracle.mirkin_pairs(Y, X) == case["ordered"]
        # F with one input partition and C = X is Mirkin(X, Y)
        Cx = np.array([np.nonzero(X == X[v])[0][0] for v in range(len(X))], np.int32)
        assert oracle.objective(Y[None, :], Cx) == case["ordered"]


def test_mirkin_against_rand_index():
    """Methods / Evaluation metrics: the rand distance is the normalised Mirkin
    distance, so Mirkin_ordered = (1 - RandIndex) n (n - 1)."""
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(1)
    for _ in range(20):
        n = int(rng.integers(2, 60))
        X = rng.integers(0, rng.integers(1, 8), n).astype(np.int32)
        Y = rng.integers(0, rng.integers(1, 8), n).astype(np.int32)
        expect = (1.0 - sk.rand_score(X, Y)) * n * (n - 1)
        assert oracle.mirkin_pairs(X, Y) == int(round(expect))


@pytest.mark.parametrize("seed", range(12))
def test_objective_equals_pair_count(seed):
    """P1: the contingency form of F equals sum_i Mirkin(C, P_i) by pair enumeration."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 70))
    k = int(rng.integers(1, 7))
    labels, C = _random_case(rng, n, k, int(rng.integers(1, 9)), int(rng.integers(1, 12)))
    expect = sum(oracle.mirkin_pairs(C, labels[i]) for i in range(k))
    assert oracle.objective(labels, C) == expect


def test_objective_singletons_closed_form():
    """P2: at singletons F0 = sum_i sum_j |P_ij|^2 - k n, and each Mirkin term is
    the number of ordered pairs co-clustered in P_i."""
    rng = np.random.default_rng(7)
    for _ in range(10):
        n = int(rng.integers(1, 80))
        k = int(rng.integers(1, 6))
        labels = rng.integers(0, 6, size=(k, n)).astype(np.int32)
        C = np.arange(n, dtype=np.int32)
        pairs = sum(int((labels[i][:, None] == labels[i][None, :]).sum()) - n for i in range(k))
        assert oracle.objective(labels, C) == pairs
        sq = sum(int((np.bincount(np.unique(labels[i], return_inverse=True)[1]) ** 2).sum()) for i in range(k))
        assert oracle.partition_sq(labels) == sq
        assert oracle.objective(labels, C) == sq - k * n


def test_objective_zero_iff_equal():
    """Mirkin is a metric: F = 0 when every P_i equals C, > 0 otherwise."""
    rng = np.random.default_rng(3)
    n = 40
    lab = rng.integers(0, 5, n).astype(np.int32)
    C = np.array([np.nonzero(lab == lab[v])[0][0] for v in range(n)], np.int32)
    labels = np.stack([lab, lab + 10, lab * 3])
    assert oracle.objective(labels, C) == 0
    C2 = C.copy()
    C2[0] = 1 if C2[0] != 1 else 2
    assert oracle.objective(labels, C2) > 0


# -------------------------------------------------------------- P3: gains


@pytest.mark.parametrize("seed", range(6))
def test_gain_forms_agree_with_objective_difference(seed):
    """P3: member-iteration dD = closed-form dD, and F(after) - F(before) = 2 dD
    for every vertex and every target cluster (Eq. objective3, u != v)."""
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 30))
    k = int(rng.integers(1, 6))
    labels, C = _random_case(rng, n, k, int(rng.integers(1, 5)), int(rng.integers(1, 8)))
    F = oracle.objective(labels, C)
    ids = np.unique(C)
    for v in range(n):
        for b in ids:
            if b == C[v]:
                continue
            gm = oracle.gain_member(labels, C, v, int(b))
            gc = oracle.gain_closed(labels, C, v, int(b))
            C2 = C.copy()
            C2[v] = b
            assert gm == gc
            assert oracle.objective(labels, C2) - F == 2 * gm


def _brute_proposals(row_off, col, labels, C):
    """Each vertex's best graph-restricted move, evaluated with the member form
    for every candidate (Eq. objective4, ties to the smaller id, dD < 0 only)."""
    n = len(C)
    target = np.full(n, -1, np.int32)
    gain = np.zeros(n, np.int64)
    for v in range(n):
        cands = sorted({int(C[u]) for u in col[row_off[v]:row_off[v + 1]] if u != v} - {int(C[v])})
        best = None
        for x in cands:
            g = oracle.gain_member(labels, C, v, x)
            if best is None or g < best[0]:
                best = (g, x)
        if best is not None and best[0] < 0:
            gain[v], target[v] = best
    return target, gain


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("mode", [0, 1])
def test_proposals_are_brute_force_argmin(seed, mode):
    """P4 (step check): every proposal is the argmin over the graph-restricted
    candidates, evaluated one by one with the member form."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 40))
    k = int(rng.integers(1, 6))
    labels, C = _random_case(rng, n, k, int(rng.integers(1, 4)), int(rng.integers(1, n)))
    row_off, col = _random_graph(rng, n, 0.25)
    t, g, cnt = oracle.sync_propose(row_off, col, labels, C, mode=mode)
    bt, bg = _brute_proposals(row_off, col, labels, C)
    np.testing.assert_array_equal(t, bt)
    np.testing.assert_array_equal(g, bg)
    assert cnt == int((bt >= 0).sum())


# ------------------------------------------------- the synchronous sweep rule


def _apply_rule(C, target, gain, labels, F):
    """The sweep rule written out from its definition (singleton guard, exact
    F of P1 by the pinned objective, matching by least (dD, v) per cluster)."""
    n = len(C)
    size = np.bincount(C, minlength=n)
    P = [v for v in range(n) if target[v] >= 0]
    if not P:
        return C.copy(), dict(proposals=0, p1=0, dF_p1=0, fallback=0, moves=0, F=F)
    P1 = [v for v in P if not (size[C[v]] == 1 and size[target[v]] == 1) or target[v] < C[v]]
    C1 = C.copy()
    for v in P1:
        C1[v] = target[v]
    dF = oracle.objective(labels, C1) - F if P1 else 0
    if P1 and dF < 0:
        return C1, dict(proposals=len(P), p1=len(P1), dF_p1=dF, fallback=0, moves=len(P1), F=F + dF)
    best = {}
    for v in P:
        for x in (int(C[v]), int(target[v])):
            key = (int(gain[v]), v)
            if x not in best or key < best[x]:
                best[x] = key
    M = [v for v in P if best[int(C[v])] == (int(gain[v]), v) == best[int(target[v])]]
    touched = [x for v in M for x in (int(C[v]), int(target[v]))]
    assert len(touched) == len(set(touched)), "matching must touch disjoint clusters"
    assert M, "matching of a non-empty proposal set is non-empty"
    C2 = C.copy()
    for v in M:
        C2[v] = target[v]
    F2 = oracle.objective(labels, C2)
    assert F2 - F == 2 * sum(int(gain[v]) for v in M), "disjoint moves add exactly"
    return C2, dict(proposals=len(P), p1=len(P1), dF_p1=dF, fallback=1, moves=len(M), F=F2)


def test_golden_path3():
    g = _golden("path3_sync.json")
    e = np.array(g["edges"])
    row_off, col = csr_from_edges(g["n"], e[:, 0], e[:, 1])
    labels = np.array(g["labels"], np.int32)
    C = oracle.singletons(g["n"])
    assert oracle.objective(labels, C) == g["F0"]
    F = g["F0"]
    for want in g["sweeps"]:
        r = oracle.sync_step(row_off, col, labels, C, F)
        for key in ("proposals", "p1", "dF_p1", "fallback", "moves", "F"):
            assert r.stats[key] == want[key], key
        np.testing.assert_array_equal(r.C, want["C"])
        C, F = r.C, r.stats["F"]
    run = oracle.sync_run(row_off, col, labels, 20)
    assert run.sweeps == len(g["sweeps"])
    assert run.F == g["sweeps"][-1]["F"]


def test_golden_swap_fallback():
    g = _golden("swap_fallback.json")
    e = np.array(g["edges"])
    row_off, col = csr_from_edges(g["n"], e[:, 0], e[:, 1])
    labels = np.array(g["labels"], np.int32)
    C0 = np.array(g["C0"], np.int32)
    assert oracle.objective(labels, C0) == g["F0"]
    r = oracle.sync_step(row_off, col, labels, C0)
    for key, val in g["sweep"].items():
        if key == "C":
            np.testing.assert_array_equal(r.C, val)
        else:
            assert r.stats[key] == val, key
    np.testing.assert_array_equal(r.gain, g["gains"])


@pytest.mark.parametrize("seed", range(8))
def test_sync_step_follows_rule(seed):
    """Each oracle sweep equals the rule applied to its (independently pinned)
    proposals, including fallback sweeps."""
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(6, 60))
    k = int(rng.integers(1, 6))
    labels, C = _random_case(rng, n, k, int(rng.integers(1, 4)), int(rng.integers(1, n)))
    if seed % 2 == 0:
        C = np.arange(n, dtype=np.int32)
    row_off, col = _random_graph(rng, n, 0.2)
    F = oracle.objective(labels, C)
    for _ in range(20):
        r = oracle.sync_step(row_off, col, labels, C, F)
        bt, bg = _brute_proposals(row_off, col, labels, C)
        np.testing.assert_array_equal(r.target, bt)
        np.testing.assert_array_equal(r.gain, bg)
        C_rule, st = _apply_rule(C, bt, bg, labels, F)
        np.testing.assert_array_equal(r.C, C_rule)
        assert r.stats == st
        assert r.stats["F"] == oracle.objective(labels, r.C)
        if st["proposals"] == 0:
            break
        assert r.stats["F"] < F  # P5: strictly lower whenever moves are committed
        C, F = r.C, r.stats["F"]


def test_fallback_sweeps_follow_rule():
    """The matching branch, on random starts where it is taken: the committed
    moves are exactly the proposals holding the least (dD, v) at both ends."""
    seen = 0
    partial = 0
    for seed in range(80):
        rng = np.random.default_rng(500 + seed)
        # groups that agree in (almost) every partition, each split in two
        # halves: both halves want to move into the other at the same time
        sizes = 2 * rng.integers(2, 5, int(rng.integers(2, 6)))
        n = int(sizes.sum())
        group = np.repeat(np.arange(len(sizes)), sizes)
        k = int(rng.integers(2, 5))
        labels = np.stack([group + 10 * i for i in range(k)]).astype(np.int32)
        noise = rng.random(labels.shape) < 0.1
        labels[noise] = rng.integers(0, 50, int(noise.sum()))
        C = np.empty(n, np.int32)
        start = 0
        for s in sizes:
            mem = np.arange(start, start + s)
            half = rng.permutation(mem)
            cut = int(s // 2 + rng.integers(-1, 2) * (seed % 3 == 0))
            C[half[:cut]] = half[0]
            C[half[cut:]] = half[cut]
            start += s
        iu, ju = np.triu_indices(n, 1)
        keep = (group[iu] == group[ju]) & (rng.random(len(iu)) < 0.8) | (rng.random(len(iu)) < 0.05)
        row_off, col = csr_from_edges(n, iu[keep], ju[keep])
        F = oracle.objective(labels, C)
        r = oracle.sync_step(row_off, col, labels, C, F)
        if not r.stats["fallback"]:
            continue
        seen += 1
        C_rule, st = _apply_rule(C, r.target, r.gain, labels, F)
        np.testing.assert_array_equal(r.C, C_rule)
        assert r.stats == st
        partial += st["moves"] < st["proposals"]
    assert seen >= 3 and partial >= 1


@pytest.mark.parametrize("seed", range(10))
def test_matching_definition(seed):
    """The fallback matching on random proposal sets full of chains and shared
    ends: kept moves touch pairwise-disjoint clusters, the least key overall is
    always kept, and a move is kept iff its key is the least at both its ends."""
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(5, 300))
    ids = rng.choice(n, max(2, n // int(rng.integers(2, 8))), replace=False).astype(np.int32)
    C = ids[rng.integers(0, len(ids), n)]
    target = np.full(n, -1, np.int32)
    gain = np.zeros(n, np.int64)
    for v in range(n):
        if rng.random() < 0.6:
            t = ids[rng.integers(0, len(ids))]
            if t != C[v]:
                target[v] = t
                gain[v] = -int(rng.integers(1, 6))  # many equal gains: ties by v
    moved = oracle.match(C, target, gain)
    P = np.nonzero(target >= 0)[0]
    if len(P) == 0:
        assert not moved.any()
        return
    ends = [x for v in np.nonzero(moved)[0] for x in (C[v], target[v])]
    assert len(ends) == len(set(ends))
    gmin = min((int(gain[v]), int(v)) for v in P)
    assert moved[gmin[1]]
    for v in P:
        keys_a = [(int(gain[w]), int(w)) for w in P if C[v] in (C[w], target[w])]
        keys_b = [(int(gain[w]), int(w)) for w in P if target[v] in (C[w], target[w])]
        mine = (int(gain[v]), int(v))
        assert moved[v] == (min(keys_a) == mine and min(keys_b) == mine)
    assert not moved[target < 0].any()


def test_self_loops_ignored():
    """A pair is two distinct vertices: self-loops in the CSR change nothing."""
    c = make_config("sbm", n=200, communities=4, k=4)
    ro, col = c["row_off"], c["col"]
    n = len(ro) - 1
    rows = np.repeat(np.arange(n), np.diff(ro))
    rows2 = np.concatenate([rows, np.arange(n)])
    cols2 = np.concatenate([col, np.arange(n, dtype=np.int32)])
    order = np.lexsort((cols2, rows2))
    ro2 = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows2, minlength=n), out=ro2[1:])
    col2 = cols2[order].astype(np.int32)
    a = oracle.sync_run(ro, col, c["labels"], 20)
    b = oracle.sync_run(ro2, col2, c["labels"], 20)
    np.testing.assert_array_equal(a.C, b.C)
    assert a.stats == b.stats
    rng = np.random.default_rng(4)
    labels, C = _random_case(rng, n, 4, 3, 40)
    t1, g1, _ = oracle.sync_propose(ro, col, labels, C)
    t2, g2, _ = oracle.sync_propose(ro2, col2, labels, C)
    np.testing.assert_array_equal(t1, t2)
    np.testing.assert_array_equal(g1, g2)


# -------------------------------------------------------------- P4: optimum


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_bounds_and_local_optimum(seed):
    """P4: F* (all set partitions, pair-counted) <= F(sync), F(seq); the brute
    optimum has the same F under the contingency form; converged states admit
    no graph-restricted move with dD < 0."""
    rng = np.random.default_rng(600 + seed)
    n = int(rng.integers(3, 10))
    k = int(rng.integers(1, 5))
    labels = rng.integers(0, 3, size=(k, n)).astype(np.int32)
    row_off, col = _random_graph(rng, n, 0.5)
    Fstar, Cstar = oracle.brute_force(labels)
    Crep = np.array([np.nonzero(Cstar == Cstar[v])[0][0] for v in range(n)], np.int32)
    assert oracle.objective(labels, Crep) == Fstar
    run = oracle.sync_run(row_off, col, labels, 50)
    Cs, Ft, _ = oracle.seq_run(row_off, col, labels, 50)
    assert run.F >= Fstar
    assert Ft[-1] >= Fstar if len(Ft) else oracle.objective(labels, Cs) >= Fstar
    for C in (run.C, Cs):
        t, _, cnt = oracle.sync_propose(row_off, col, labels, C)
        assert cnt == 0
        for v in range(n):
            for u in col[row_off[v]:row_off[v + 1]]:
                if C[u] != C[v]:
                    assert oracle.gain_member(labels, C, v, int(C[u])) >= 0


def test_brute_force_exhaustive_count():
    """Bell(n) partitions are visited: with k = 1 and all labels distinct the
    optimum is the all-singleton partition (F = 0); with all labels equal it is
    one cluster (F = 0); anything else would show a missed or repeated case."""
    for n in range(1, 10):
        F, C = oracle.brute_force(np.arange(n, dtype=np.int32)[None, :])
        assert F == 0 and len(set(C.tolist())) == n
        F, C = oracle.brute_force(np.zeros((1, n), np.int32))
        assert F == 0 and len(set(C.tolist())) == 1


# ------------------------------------------------------- P5-P7: properties


def test_sequential_trace():
    """Sequential greedy: every sweep lowers F, and F matches the objective."""
    c = make_config("sbm", n=300, communities=6, k=6)
    C, Ft, Mt = oracle.seq_run(c["row_off"], c["col"], c["labels"], 20)
    assert np.all(np.diff(Ft) <= 0)
    assert Ft[-1] == oracle.objective(c["labels"], C)
    assert Mt[-1] == 0 or len(Mt) == 20


def _seq_golden(g, labels):
    e = np.array(g["edges"])
    row_off, col = csr_from_edges(g["n"], e[:, 0], e[:, 1])
    return oracle.seq_run(row_off, col, np.array(labels, np.int32), 20)


def test_golden_sequential_visit_order():
    """Sequential greedy (Parallel algorithm section, one move at a time):
    the hand-worked trajectory in increasing vertex order.  A decreasing
    order ends in another partition, so a reversed visit order fails here."""
    g = _golden("seq_order_path5.json")
    assert oracle.objective(np.array(g["labels"], np.int32), oracle.singletons(g["n"])) == g["F0"]
    C, Ft, Mt = _seq_golden(g, g["labels"])
    np.testing.assert_array_equal(C, g["increasing"]["C"])
    assert Ft.tolist() == g["increasing"]["F_trace"]
    assert Mt.tolist() == g["increasing"]["moves_trace"]
    assert not np.array_equal(oracle.renumber(np.array(g["decreasing"]["C"])), oracle.renumber(C))
    # the mirrored instance: its increasing order is the original's decreasing one
    C, Ft, Mt = _seq_golden(g, g["mirrored_labels"])
    np.testing.assert_array_equal(C, g["mirrored_increasing"]["C"])
    assert Ft.tolist() == g["mirrored_increasing"]["F_trace"]
    mirrored_back = C[::-1]
    np.testing.assert_array_equal(oracle.renumber(mirrored_back),
                                  oracle.renumber(np.array(g["decreasing"]["C"])))


def test_golden_sequential_tie_rule():
    """Sequential greedy: a tie between candidate clusters goes to the
    smaller id (hand-worked on a 3-vertex star)."""
    g = _golden("seq_tie_star3.json")
    C, Ft, Mt = _seq_golden(g, g["labels"])
    np.testing.assert_array_equal(C, g["C"])
    assert Ft.tolist() == g["F_trace"] and Mt.tolist() == g["moves_trace"]
    assert not np.array_equal(C, g["tie_to_larger_C"]) and not np.array_equal(C, g["decreasing_C"])


def test_identical_copies_recover_partition():
    """P6: k identical copies of P whose clusters induce connected subgraphs ->
    both variants end at C = P with F = 0."""
    c = make_config("sbm", n=400, communities=8, p_in=0.3, p_out=0.01, k=1)
    truth = c["truth"].astype(np.int32)
    labels = np.stack([truth, truth + 100, truth * 7, truth])
    run = oracle.sync_run(c["row_off"], c["col"], labels, 200)
    assert run.F == 0
    np.testing.assert_array_equal(oracle.renumber(run.C), oracle.renumber(truth))
    Cs, Ft, _ = oracle.seq_run(c["row_off"], c["col"], labels, 200)
    assert Ft[-1] == 0
    np.testing.assert_array_equal(oracle.renumber(Cs), oracle.renumber(truth))


def test_invariances():
    """P7: permuting partitions and relabelling inside a partition change
    nothing; duplicating every partition doubles F and keeps the labels and
    the sweep count."""
    c = make_config("sbm", n=500, communities=5, k=6)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    base = oracle.sync_run(ro, col, lab, 20)
    perm = oracle.sync_run(ro, col, lab[::-1].copy(), 20)
    rng = np.random.default_rng(9)
    relab = lab.copy()
    m = rng.permutation(1000)
    relab[2] = m[lab[2]] - 77
    rel = oracle.sync_run(ro, col, relab, 20)
    dup = oracle.sync_run(ro, col, np.concatenate([lab, lab]), 20)
    for r in (perm, rel):
        np.testing.assert_array_equal(r.C, base.C)
        assert r.stats == base.stats
    np.testing.assert_array_equal(dup.C, base.C)
    assert dup.sweeps == base.sweeps
    assert [s["F"] for s in dup.stats] == [2 * s["F"] for s in base.stats]


def test_sync_monotone_on_workloads():
    """P5 on the small SBM and a small LFR-style graph: F after every sweep equals
    the objective recomputed from scratch and never increases."""
    for c in (make_config("sbm"), make_config("lfr", n=3000, k=8, cmin=20, cmax=300)):
        lab = c["labels"]
        C = oracle.singletons(lab.shape[1])
        F = oracle.objective(lab, C)
        for _ in range(20):
            r = oracle.sync_step(c["row_off"], c["col"], lab, C, F)
            assert r.stats["F"] == oracle.objective(lab, r.C)
            assert r.stats["F"] <= F
            if r.stats["proposals"] == 0:
                break
            C, F = r.C, r.stats["F"]


def test_gain_modes_same_trajectory():
    """The contingency lookups and the member iteration give the same run."""
    c = make_config("sbm", n=300, communities=6, k=5)
    a = oracle.sync_run(c["row_off"], c["col"], c["labels"], 20, mode=0)
    b = oracle.sync_run(c["row_off"], c["col"], c["labels"], 20, mode=1)
    np.testing.assert_array_equal(a.C, b.C)
    assert a.stats == b.stats


# ------------------------------------------- move-to-empty variant (option)


def _brute_proposals_empty(row_off, col, labels, C):
    """Best move of each vertex with the empty cluster of id v among the
    candidates when no vertex carries that id; every gain from the pinned
    objective: dD = (F(after) - F(before)) / 2."""
    n = len(C)
    F = oracle.objective(labels, C)
    size = np.bincount(C, minlength=n)
    target = np.full(n, -1, np.int32)
    gain = np.zeros(n, np.int64)
    for v in range(n):
        cands = {int(C[u]) for u in col[row_off[v]:row_off[v + 1]] if u != v} - {int(C[v])}
        if size[v] == 0:
            cands.add(v)
        best = None
        for x in sorted(cands):
            C2 = C.copy()
            C2[v] = x
            d2 = oracle.objective(labels, C2) - F
            assert d2 % 2 == 0
            if best is None or d2 // 2 < best[0]:
                best = (d2 // 2, x)
        if best is not None and best[0] < 0:
            gain[v], target[v] = best
    return target, gain


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("mode", [0, 1])
def test_empty_move_proposals_are_brute_force_argmin(seed, mode):
    """Move-to-empty variant: every proposal is the argmin over the neighbours'
    clusters and, when the id v is free, the empty cluster v (ties to the
    smaller id), each gain recomputed from the objective; both gain forms."""
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(5, 40))
    k = int(rng.integers(1, 6))
    labels, C = _random_case(rng, n, k, int(rng.integers(1, 4)), int(rng.integers(1, max(2, n // 3))))
    row_off, col = _random_graph(rng, n, 0.2)
    t, g, cnt = oracle.sync_propose(row_off, col, labels, C, mode=mode, empty=True)
    bt, bg = _brute_proposals_empty(row_off, col, labels, C)
    np.testing.assert_array_equal(t, bt)
    np.testing.assert_array_equal(g, bg)
    assert cnt == int((bt >= 0).sum())
    assert np.any(bt == np.arange(n)) or seed > 3  # the empty move is exercised


@pytest.mark.parametrize("seed", range(6))
def test_empty_move_gain_closed_form(seed):
    """The empty-target gain 2 (A_a - k) - k (|a| - 1) (closed form, a free
    id b) equals the member form and half the objective difference."""
    rng = np.random.default_rng(800 + seed)
    n = int(rng.integers(3, 30))
    k = int(rng.integers(1, 6))
    labels, C = _random_case(rng, n, k, int(rng.integers(1, 5)), int(rng.integers(1, max(2, n // 2))))
    F = oracle.objective(labels, C)
    size = np.bincount(C, minlength=n)
    for v in range(n):
        if size[v] != 0:
            continue
        gm = oracle.gain_member(labels, C, v, v)
        gc = oracle.gain_closed(labels, C, v, v)
        C2 = C.copy()
        C2[v] = v
        assert gm == gc and oracle.objective(labels, C2) - F == 2 * gm


@pytest.mark.parametrize("seed", range(6))
def test_empty_move_sweeps_follow_rule(seed):
    """With the variant, each sweep is the written rule (guards, matching)
    applied to the brute-force proposals, F falls strictly on every sweep that
    moves, and no vertex ever carries an id that another cluster holds."""
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(8, 36))
    k = int(rng.integers(2, 6))
    labels, C = _random_case(rng, n, k, int(rng.integers(2, 4)), int(rng.integers(1, 4)))
    row_off, col = _random_graph(rng, n, 0.2)
    F = oracle.objective(labels, C)
    for _ in range(8):
        bt, bg = _brute_proposals_empty(row_off, col, labels, C)
        want_C, want = _apply_rule(C, bt, bg, labels, F)
        r = oracle.sync_step(row_off, col, labels, C, F, empty=True)
        assert r.stats == want
        np.testing.assert_array_equal(r.C, want_C)
        if r.stats["moves"]:
            assert r.stats["F"] < F
        C, F = r.C, r.stats["F"]
        if r.stats["proposals"] == 0:
            break


def test_golden_empty_move():
    g = _golden("empty_move_path3.json")
    e = np.array(g["edges"])
    row_off, col = csr_from_edges(g["n"], e[:, 0], e[:, 1])
    labels = np.array(g["labels"], np.int32)
    C = np.array(g["C0"], np.int32)
    assert oracle.objective(labels, C) == g["F0"]
    # the base rule has no candidate here
    assert oracle.sync_step(row_off, col, labels, C).stats["proposals"] == 0
    F = g["F0"]
    for s, want in enumerate(g["sweeps"]):
        r = oracle.sync_step(row_off, col, labels, C, F, empty=True)
        for key in ("proposals", "p1", "dF_p1", "fallback", "moves", "F"):
            assert r.stats[key] == want[key], key
        np.testing.assert_array_equal(r.C, want["C"])
        if s == 0:
            assert r.gain[2] == want["gain_v2"] and r.target[2] == 2
        C, F = r.C, r.stats["F"]


def test_propose_range_is_a_slice():
    """The block-restricted proposal pass (used to time a bounded sample)
    gives exactly the full pass's proposals inside the block and none outside."""
    c = make_config("sbm", n=300, communities=5, k=4, seed=4)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    C = oracle.singletons(300)
    t, g, cnt = oracle.sync_propose(ro, col, lab, C)
    tr, gr, cr = oracle.sync_propose_range(ro, col, lab, C, 100, 220)
    np.testing.assert_array_equal(tr[100:220], t[100:220])
    np.testing.assert_array_equal(gr[100:220], g[100:220])
    assert np.all(tr[:100] == -1) and np.all(tr[220:] == -1)
    assert cr == int((t[100:220] >= 0).sum())


# ------------------------------------------- colour-batched greedy (variant)


def test_priority_is_splitmix64():
    """The colouring priority is the first output of splitmix64 seeded with
    v: its published sequence for seed 0 is 0xe220a8397b1dcdaf,
    0x6e789e6aa1b965f4, 0x06c45d188009454f (seeds 0, g, 2g with g its
    increment 0x9E3779B97F4A7C15)."""
    g = 0x9E3779B97F4A7C15
    assert oracle.priority(0) == 0xE220A8397B1DCDAF
    assert oracle.priority(g) == 0x6E789E6AA1B965F4
    assert oracle.priority(2 * g) == 0x06C45D188009454F


@pytest.mark.parametrize("seed", range(6))
def test_colouring_is_proper_and_greedy(seed):
    """Adjacent vertices get different colours, and each colour is the least
    one that no higher-priority neighbour holds (greedy in priority order)."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 300))
    row_off, col = _random_graph(rng, n, float(rng.uniform(0.01, 0.3)))
    cls, ncol = oracle.colour(row_off, col)
    pri = [oracle.priority(v) for v in range(n)]
    assert ncol == (int(cls.max()) + 1 if n else 0)
    for v in range(n):
        nb = [int(u) for u in col[row_off[v]:row_off[v + 1]] if u != v]
        assert all(cls[u] != cls[v] for u in nb)
        higher = {int(cls[u]) for u in nb if pri[u] > pri[v]}
        assert cls[v] == min(set(range(len(higher) + 1)) - higher)


@pytest.mark.parametrize("seed", range(6))
def test_colour_sweeps_follow_rule(seed):
    """Each colour class is the written rule (singleton guard, exact guard,
    matching) applied to the brute-force proposals of that class's vertices
    against the state the earlier classes left; a sweep's record sums the
    classes; F never rises; the run stops at a sweep without proposals."""
    rng = np.random.default_rng(1100 + seed)
    n = int(rng.integers(6, 30))
    k = int(rng.integers(1, 5))
    labels = rng.integers(0, int(rng.integers(2, 4)), size=(k, n)).astype(np.int32)
    row_off, col = _random_graph(rng, n, 0.3)
    cls, ncol = oracle.colour(row_off, col)
    run = oracle.colour_run(row_off, col, labels, 30)
    C = oracle.singletons(n)
    F = oracle.objective(labels, C)
    for rec in run.stats:
        tot = dict(proposals=0, p1=0, dF_p1=0, fallback=0, moves=0)
        for c in range(ncol):
            bt, bg = _brute_proposals(row_off, col, labels, C)
            bt = np.where(cls == c, bt, -1)
            bg = np.where(cls == c, bg, 0)
            C, st = _apply_rule(C, bt, bg, labels, F)
            assert st["F"] <= F
            F = st["F"]
            for key in tot:
                tot[key] += st[key]
        assert rec == dict(tot, F=F)
    np.testing.assert_array_equal(run.C, C)
    assert run.stats[-1]["proposals"] == 0 or run.sweeps == 30


@pytest.mark.parametrize("seed", range(5))
def test_colour_run_bounds(seed):
    """Against brute force over all set partitions (n <= 9): F(colour) >= F*,
    and the end state has no improving graph-restricted move."""
    rng = np.random.default_rng(1200 + seed)
    n = int(rng.integers(4, 10))
    k = int(rng.integers(1, 4))
    labels = rng.integers(0, 3, size=(k, n)).astype(np.int32)
    row_off, col = _random_graph(rng, n, 0.5)
    Fstar, _ = oracle.brute_force(labels)
    run = oracle.colour_run(row_off, col, labels, 50)
    assert run.F >= Fstar
    assert run.F == oracle.objective(labels, run.C)
    t, _, cnt = oracle.sync_propose(row_off, col, labels, run.C)
    assert cnt == 0


def test_colour_run_recovers_identical_copies():
    """k identical copies of P whose clusters are connected: the colour-batched
    run ends at C = P with F = 0, as the other variants do."""
    c = make_config("sbm", n=400, communities=8, p_in=0.3, p_out=0.01, k=1)
    truth = c["truth"].astype(np.int32)
    labels = np.stack([truth, truth + 100, truth * 7, truth])
    run = oracle.colour_run(c["row_off"], c["col"], labels, 200)
    assert run.F == 0
    np.testing.assert_array_equal(oracle.renumber(run.C), oracle.renumber(truth))
