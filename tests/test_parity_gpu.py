"""Parity of the CUDA sweep with the CPU oracle, through the C ABI.

Integer arithmetic on both sides, so the bar is bit-exact: the sweep count,
every per-sweep record (|P|, |P1|, dF of P1, fallback, moves, F), the raw
cluster ids after each sweep, the renumbered labels and the objective.
"""
import json
import os

import numpy as np
import pytest

import oracle
from workloads import csr_from_edges, make_config

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2408_11331_gb300 as m

    return m


def gpu_run(cc, row_off, col, labels, max_sweeps=20, **opt):
    o = cc.cc_default_options()
    for key, val in opt.items():
        setattr(o, key, val)
    with cc.Consensus(row_off, col, labels, o) as job:
        sweeps = job.run_until_converged(max_sweeps)
        return dict(sweeps=sweeps, hist=job.history(), C=job.cluster_ids(), F=job.objective(),
                    Frec=job.objective_recompute(), labels=job.consensus_labels())


def assert_same(g, ref):
    assert g["sweeps"] == ref.sweeps
    assert g["hist"] == ref.stats
    np.testing.assert_array_equal(g["C"], ref.C)
    assert g["F"] == ref.F == g["Frec"]
    np.testing.assert_array_equal(g["labels"], oracle.renumber(ref.C))


MODES = [0, 1, 2]  # automatic, always staged deltas, always rebuild


def options(cc, **kw):
    o = cc.cc_default_options()
    for key, val in kw.items():
        setattr(o, key, val)
    return o


@pytest.mark.parametrize("mode", MODES)
def test_sbm_full_run(cc, mode):
    c = make_config("sbm")
    ref = oracle.sync_run(c["row_off"], c["col"], c["labels"], 20)
    assert_same(gpu_run(cc, c["row_off"], c["col"], c["labels"], 20, sweep_mode=mode), ref)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,k,seed", [(20000, 8, 11), (5003, 37, 12), (3001, 1, 13), (12000, 64, 14)])
def test_lfr_stepwise(cc, n, k, seed, mode):
    """Sweep by sweep: several lane groups, ragged tails, k not a multiple of
    4, k above one warp, and k = 1; in every sweep mode."""
    c = make_config("lfr", n=n, k=k, cmin=20, cmax=min(1000, n), max_deg=min(1000, n // 4), seed=seed)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    C = oracle.singletons(n)
    F = oracle.objective(lab, C)
    with cc.Consensus(ro, col, lab, options(cc, sweep_mode=mode)) as job:
        assert job.objective() == F
        for _ in range(25):
            r = oracle.sync_step(ro, col, lab, C, F)
            info = job.sweep()
            assert info == r.stats
            np.testing.assert_array_equal(job.cluster_ids(), r.C)
            if r.stats["proposals"] == 0:
                break
            C, F = r.C, r.stats["F"]
        assert job.objective_recompute() == F


@pytest.mark.parametrize("mode", MODES)
def test_knn_small(cc, mode):
    c = make_config("knn", n=6000, comps=30, dim=20, k=12, seed=21)
    ref = oracle.sync_run(c["row_off"], c["col"], c["labels"], 30)
    assert_same(gpu_run(cc, c["row_off"], c["col"], c["labels"], 30, sweep_mode=mode), ref)


def _edges(n, pairs):
    e = np.array(pairs, dtype=np.int64).reshape(-1, 2)
    return csr_from_edges(n, e[:, 0], e[:, 1])


def _cases():
    rng = np.random.default_rng(5)
    out = {}
    # no edges at all: one sweep, no proposal
    out["empty"] = (np.zeros(51, np.int64), np.zeros(0, np.int32), rng.integers(0, 3, (4, 50)).astype(np.int32))
    out["single_vertex"] = (np.zeros(2, np.int64), np.zeros(0, np.int32), np.array([[5], [7]], np.int32))
    # star whose centre has 100 singleton neighbours (several 32-wide chunks)
    ro, col = _edges(101, [(0, i) for i in range(1, 101)])
    out["star"] = (ro, col, rng.integers(0, 2, (6, 101)).astype(np.int32))
    # degrees exactly 32 and 33 around two hubs
    pairs = [(0, i) for i in range(1, 33)] + [(40, i) for i in range(41, 74)]
    ro, col = _edges(80, pairs)
    out["deg32_33"] = (ro, col, rng.integers(0, 3, (5, 80)).astype(np.int32))
    # two cliques joined by one edge, identical labels -> the cliques
    pairs = [(i, j) for i in range(10) for j in range(i + 1, 10)] + \
            [(i, j) for i in range(10, 25) for j in range(i + 1, 25)] + [(9, 10)]
    ro, col = _edges(25, pairs)
    lab = np.array([[0] * 10 + [1] * 15] * 3, np.int32)
    out["two_cliques"] = (ro, col, lab)
    # path with all-equal labels
    ro, col = _edges(40, [(i, i + 1) for i in range(39)])
    out["path"] = (ro, col, np.full((2, 40), -7, np.int32))
    # extreme and negative label values
    c = make_config("sbm", n=300, communities=5, k=4, seed=3)
    lab = c["labels"].astype(np.int64) * 1_000_003 - 2 ** 31 + 5
    lab = np.clip(lab, -2 ** 31, 2 ** 31 - 1).astype(np.int32)
    out["extreme_labels"] = (c["row_off"], c["col"], lab)
    # self-loops and repeated entries in the CSR
    rows = np.repeat(np.arange(300), np.diff(c["row_off"]))
    rows2 = np.concatenate([rows, np.arange(300), rows[:500]])
    cols2 = np.concatenate([c["col"], np.arange(300, dtype=np.int32), c["col"][:500]])
    order = np.lexsort((cols2, rows2))
    ro2 = np.zeros(301, np.int64)
    np.cumsum(np.bincount(rows2, minlength=300), out=ro2[1:])
    out["loops_and_repeats"] = (ro2, cols2[order].astype(np.int32), c["labels"])
    # identical partitions: the planted partition is recovered exactly
    c = make_config("sbm", n=400, communities=8, p_in=0.3, p_out=0.01, k=1, seed=4)
    out["identical_copies"] = (c["row_off"], c["col"], np.stack([c["truth"]] * 5).astype(np.int32))
    return out


CASES = _cases()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", sorted(CASES))
def test_edge_cases(cc, name, mode):
    ro, col, lab = CASES[name]
    ref = oracle.sync_run(ro, col, lab, 60)
    g = gpu_run(cc, ro, col, lab, 60, sweep_mode=mode)
    assert_same(g, ref)
    if name == "identical_copies":
        assert g["F"] == 0
    if name in ("empty", "single_vertex"):
        assert g["sweeps"] == 1 and g["hist"][0]["proposals"] == 0


def test_warm_start_swap_fallback(cc):
    """The hand-worked swap: P1 only exchanges two clusters, the matching commits one move."""
    with open(os.path.join(GOLDEN, "swap_fallback.json")) as f:
        g = json.load(f)
    ro, col = _edges(g["n"], g["edges"])
    lab = np.array(g["labels"], np.int32)
    with cc.Consensus(ro, col, lab) as job:
        job.set_cluster_ids(np.array(g["C0"], np.int32))
        assert job.objective() == g["F0"]
        info = job.sweep()
        want = {k: v for k, v in g["sweep"].items() if k != "C"}
        assert info == want
        np.testing.assert_array_equal(job.cluster_ids(), g["sweep"]["C"])


@pytest.mark.parametrize("mode", MODES)
def test_warm_start_fallback_random(cc, mode):
    """Starts where each group is split in two halves that want to swap: the
    fallback branch, including partial matchings, against the oracle."""
    seen = 0
    for seed in range(60):
        rng = np.random.default_rng(900 + seed)
        sizes = 2 * rng.integers(2, 6, int(rng.integers(2, 8)))
        n = int(sizes.sum())
        group = np.repeat(np.arange(len(sizes)), sizes)
        k = int(rng.integers(2, 6))
        lab = np.stack([group + 10 * i for i in range(k)]).astype(np.int32)
        noise = rng.random(lab.shape) < 0.1
        lab[noise] = rng.integers(0, 50, int(noise.sum()))
        C = np.empty(n, np.int32)
        start = 0
        for s in sizes:
            half = rng.permutation(np.arange(start, start + s))
            C[half[: s // 2]] = half[0]
            C[half[s // 2:]] = half[s // 2]
            start += s
        iu, ju = np.triu_indices(n, 1)
        keep = (group[iu] == group[ju]) & (rng.random(len(iu)) < 0.8) | (rng.random(len(iu)) < 0.05)
        ro, col = csr_from_edges(n, iu[keep], ju[keep])
        F = oracle.objective(lab, C)
        with cc.Consensus(ro, col, lab, options(cc, sweep_mode=mode)) as job:
            job.set_cluster_ids(C)
            assert job.objective() == F
            Cs, Fs = C, F
            for _ in range(10):
                r = oracle.sync_step(ro, col, lab, Cs, Fs)
                assert job.sweep() == r.stats
                np.testing.assert_array_equal(job.cluster_ids(), r.C)
                seen += r.stats["fallback"]
                if r.stats["proposals"] == 0:
                    break
                Cs, Fs = r.C, r.stats["F"]
    assert seen >= 3


def test_errors_leave_state(cc):
    c = make_config("sbm", n=200, communities=4, k=3, seed=8)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    bad = col.copy()
    bad[5] = 200
    with pytest.raises(cc.CCError) as e:
        cc.Consensus(ro, bad, lab)
    assert e.value.status == 1
    ro_bad = ro.copy()
    ro_bad[10] = ro_bad[11] + 1
    with pytest.raises(cc.CCError):
        cc.Consensus(ro_bad, col, lab)
    with cc.Consensus(ro, col, lab) as job:
        job.sweep()
        before = job.cluster_ids().copy()
        F = job.objective()
        Cbad = before.copy()
        Cbad[3] = -1
        with pytest.raises(cc.CCError):
            job.set_cluster_ids(Cbad)
        np.testing.assert_array_equal(job.cluster_ids(), before)
        assert job.objective() == F == job.objective_recompute()


def test_table_full_is_reported(cc):
    """A contingency hash far too small: bounded probing reports CC_ERR_TABLE_FULL,
    at creation when the table is built there (staged deltas), else at the
    first sweep's rebuild."""
    c = make_config("sbm", n=200, communities=4, k=3, seed=8)
    with pytest.raises(cc.CCError) as e:
        cc.Consensus(c["row_off"], c["col"], c["labels"], options(cc, table_log2=6, sweep_mode=1))
    assert e.value.status == 5
    with cc.Consensus(c["row_off"], c["col"], c["labels"], options(cc, table_log2=6)) as job:
        with pytest.raises(cc.CCError) as e:
            job.run_until_converged(20)
        assert e.value.status == 5


def test_reset_and_options(cc):
    c = make_config("lfr", n=8000, k=6, cmin=20, cmax=500, max_deg=300, seed=31)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 20)
    o = cc.cc_default_options()
    o.debug_checks = 1
    with cc.Consensus(ro, col, lab, o) as job:
        a = job.run_until_converged(20)
        ha, Ca = job.history(), job.cluster_ids().copy()
        job.reset()
        assert job.history() == []
        b = job.run_until_converged(20)
        assert a == b == ref.sweeps
        assert job.history() == ha == ref.stats
        np.testing.assert_array_equal(job.cluster_ids(), Ca)
    # a larger table (fewer rebuilds) gives the same run
    g = gpu_run(cc, ro, col, lab, 20, table_log2=int(np.ceil(np.log2(3 * 6 * 8000 + 64))) + 2)
    assert_same(g, ref)


def test_create_from_device_buffers(cc):
    torch = pytest.importorskip("torch")
    c = make_config("sbm", n=1000, k=10, seed=77)
    ref = oracle.sync_run(c["row_off"], c["col"], c["labels"], 20)
    dev = torch.device("cuda:0")
    ro = torch.from_numpy(c["row_off"]).to(dev)
    col = torch.from_numpy(c["col"]).to(dev)
    lab = torch.from_numpy(np.ascontiguousarray(c["labels"])).to(dev)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    job = cc.Consensus.from_device(1000, len(c["col"]), ro.data_ptr(), col.data_ptr(), 10, lab.data_ptr(),
                                   stream=s.cuda_stream)
    try:
        assert job.run_until_converged(20) == ref.sweeps
        assert job.history() == ref.stats
        np.testing.assert_array_equal(job.cluster_ids(), ref.C)
    finally:
        job.close()


def test_run_timing_and_launch_count(cc):
    """Per-sweep device times come from events inside the run's graph; the
    launch counter counts the kernels outside the graph's conditional regions
    on every sweep body and the region kernels that ran."""
    c = make_config("sbm")
    with cc.Consensus(c["row_off"], c["col"], c["labels"]) as job:
        base = job.launch_count()
        done = job.run_until_converged(20)
        sweep_ms, prop_ms = job.last_run_timing()
        assert len(sweep_ms) == len(prop_ms) == done
        assert np.all(sweep_ms > 0) and np.all(prop_ms > 0) and np.all(prop_ms <= sweep_ms)
        bodies = ((done + 3) // 4) * 4  # graphs of 4 unrolled sweep bodies
        outside = 17  # per body: begin, own, edges, collect, route, 6 gates, bid, match keys, commit,
        #               match reset, end jobs, end
        rebuild = 9  # clear, 3 scan kernels, scatter, build, build check, summaries, done
        # heavy path, its second rebuild attempt, heavy evaluation, rollback,
        # light path, end-of-sweep rebuild
        regions = (2 + rebuild) + rebuild + 2 + (1 + rebuild) + 3 + rebuild
        delta = job.launch_count() - base
        assert 1 + bodies * outside < delta < 1 + bodies * (outside + regions)
        # a sweep runs the heavy or the light path, never both, and the
        # skipped bodies after the run stopped enter no region
        assert delta <= 1 + bodies * outside + done * (regions - 3)
        job.sweep()
        assert len(job.last_run_timing()[0]) == 1


def _hub_case(n_nbr, clusters_of, pair_with_leaf, seed):
    """Vertex 0 joined to vertices 1..n_nbr; the warm-start consensus puts the
    neighbours in the clusters given by clusters_of (optionally each with a
    private leaf), and vertex 0 in a two-member cluster with the last vertex."""
    rng = np.random.default_rng(seed)
    leaves = n_nbr if pair_with_leaf else 0
    n = 1 + n_nbr + leaves + 1
    pairs = [(0, i) for i in range(1, n_nbr + 1)]
    if pair_with_leaf:
        pairs += [(i, n_nbr + i) for i in range(1, n_nbr + 1)]
    pairs += [(0, n - 1)]
    ro, col = _edges(n, pairs)
    C = np.arange(n, dtype=np.int32)
    for i in range(1, n_nbr + 1):
        C[i] = clusters_of(i)
        if pair_with_leaf:
            C[n_nbr + i] = C[i]
    C[n - 1] = 0
    lab = rng.integers(0, 3, (7, n)).astype(np.int32)
    return ro, col, lab, C


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", ["own_plus_32_tables", "repeats_across_chunks", "seen_set_full"])
def test_warm_start_hubs(cc, case, mode):
    """Proposal edge cases: 33 table-scored clusters in one chunk (own cluster
    plus 32 neighbours' two-member clusters), candidates repeated across
    32-wide chunks, and more distinct candidates than the seen-set holds."""
    if case == "own_plus_32_tables":
        ro, col, lab, C = _hub_case(40, lambda i: i, True, 1)
    elif case == "repeats_across_chunks":
        ro, col, lab, C = _hub_case(100, lambda i: 1 + (i - 1) % 5, False, 2)
    else:
        ro, col, lab, C = _hub_case(200, lambda i: i, True, 3)
    F = oracle.objective(lab, C)
    with cc.Consensus(ro, col, lab, options(cc, sweep_mode=mode)) as job:
        job.set_cluster_ids(C)
        Cs, Fs = C, F
        for _ in range(8):
            r = oracle.sync_step(ro, col, lab, Cs, Fs)
            assert job.sweep() == r.stats
            np.testing.assert_array_equal(job.cluster_ids(), r.C)
            if r.stats["proposals"] == 0:
                break
            Cs, Fs = r.C, r.stats["F"]


def test_table_retry_path(cc):
    """A starting capacity too small for the first sweep's new keys: the sweep
    is abandoned before it commits, retried in twice the capacity, and the run
    equals the oracle's (including through later shrinks and rebuilds)."""
    c = make_config("lfr", n=28000, k=8, cmin=20, cmax=1000, max_deg=500, seed=11)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 20)
    o = cc.cc_default_options()
    # staged deltas from the start, in 262,144 slots for 224,000 keys: the
    # first sweep's ~16,000 new keys cross the 7/8 fill limit
    o.table_start_log2 = 18
    o.sweep_mode = 1
    with cc.Consensus(ro, col, lab, o) as job:
        assert job.run_until_converged(20) == ref.sweeps
        assert job.history() == ref.stats
        np.testing.assert_array_equal(job.cluster_ids(), ref.C)
        ts = job.table_stats()
        assert ts["retries"] >= 1 and ts["rebuilds"] >= 2
        assert ts["live_keys"] <= ts["used_slots"] <= ts["capacity"] <= ts["max_capacity"]
        assert job.objective_recompute() == ref.F


def test_full_size_lfr_as_benchmarked(cc):
    """The benchmark workload at full size (LFR-style n = 1,000,000, k = 20),
    launched as bench.py launches it (a caller stream, graphs of up to 4
    sweeps, reset then run to convergence, twice): every sweep record, the
    raw ids, the labels and F equal the oracle's."""
    import torch

    c = make_config("lfr")
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 20)
    stream = torch.cuda.Stream()
    with cc.Consensus(ro, col, lab) as job:
        job.set_stream(stream.cuda_stream)
        for _ in range(2):
            job.reset()
            assert job.run_until_converged(20) == ref.sweeps
            assert job.history() == ref.stats
            np.testing.assert_array_equal(job.cluster_ids(), ref.C)
        assert job.objective() == ref.F == job.objective_recompute()
        np.testing.assert_array_equal(job.consensus_labels(), oracle.renumber(ref.C))


def test_full_size_knn_as_benchmarked(cc):
    """The largest single-GPU workload at full size (kNN-15 of a 200-component
    Gaussian mixture in 50-D, n = 2,000,000, k = 50 graded partitions; lanes
    per item chosen automatically: 8), launched as bench.py launches it (a
    caller stream, reset then run to convergence, twice): every sweep record,
    the raw ids, the labels (n above 2^20, so the renumbering scans its block
    counts several per thread) and F equal the oracle's."""
    import torch

    c = make_config("knn", device="cuda")
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    assert lab.shape == (50, 2_000_000)
    ref = oracle.sync_run(ro, col, lab, 20)
    stream = torch.cuda.Stream()
    with cc.Consensus(ro, col, lab) as job:
        job.set_stream(stream.cuda_stream)
        for _ in range(2):
            job.reset()
            assert job.run_until_converged(20) == ref.sweeps
            assert job.history() == ref.stats
            np.testing.assert_array_equal(job.cluster_ids(), ref.C)
        assert job.objective() == ref.F == job.objective_recompute()
        np.testing.assert_array_equal(job.consensus_labels(), oracle.renumber(ref.C))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,k,seed", [(20000, 8, 11), (5003, 37, 12), (12000, 64, 14)])
def test_active_set_runs(cc, n, k, seed, mode):
    """With the active set, sweeps after the first re-score only the vertices
    near clusters that changed; the run still equals the oracle's, sweep by
    sweep, in every sweep mode."""
    c = make_config("lfr", n=n, k=k, cmin=20, cmax=min(1000, n), max_deg=min(1000, n // 4), seed=seed)
    ref = oracle.sync_run(c["row_off"], c["col"], c["labels"], 20)
    assert_same(gpu_run(cc, c["row_off"], c["col"], c["labels"], 20, sweep_mode=mode, active_set=1), ref)


def test_active_set_knn_and_reruns(cc):
    """kNN graph with the active set; a second run on the converged state
    scores everything in its first sweep and finds nothing; a reset repeats
    the run exactly."""
    c = make_config("knn", n=6000, comps=30, dim=20, k=12, seed=21)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 30)
    with cc.Consensus(ro, col, lab, options(cc, active_set=1)) as job:
        for _ in range(2):
            job.reset()
            assert job.run_until_converged(30) == ref.sweeps
            assert job.history() == ref.stats
            np.testing.assert_array_equal(job.cluster_ids(), ref.C)
        assert job.run_until_converged(30) == 1
        assert job.history()[-1]["proposals"] == 0
        assert job.objective() == ref.F == job.objective_recompute()


def test_active_set_limited_runs(cc):
    """Runs of 2 sweeps at a time: each run's first sweep scores everything,
    later ones only the active set; the trajectory equals the oracle's."""
    c = make_config("lfr", n=20000, k=8, cmin=20, cmax=1000, max_deg=1000, seed=11)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 20)
    with cc.Consensus(ro, col, lab, options(cc, active_set=1)) as job:
        for _ in range(12):
            job.run_until_converged(2)
        assert job.history()[: ref.sweeps] == ref.stats
        np.testing.assert_array_equal(job.cluster_ids(), ref.C)


def test_active_set_table_retry(cc):
    """The retry path (first sweep abandoned for lack of table space) with
    the active set on."""
    c = make_config("lfr", n=28000, k=8, cmin=20, cmax=1000, max_deg=500, seed=11)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 20)
    o = options(cc, table_start_log2=18, sweep_mode=1, active_set=1)
    with cc.Consensus(ro, col, lab, o) as job:
        assert job.run_until_converged(20) == ref.sweeps
        assert job.history() == ref.stats
        np.testing.assert_array_equal(job.cluster_ids(), ref.C)
        assert job.table_stats()["retries"] >= 1


@pytest.mark.parametrize("tight", [0, 1, 2])
@pytest.mark.parametrize("mode", [0, 2])
def test_tight_rebuild_same_results(cc, tight, mode):
    """The heavy sweep's rebuild first tries a tight capacity and builds again
    at the safe one when the keys do not fit (tight_rebuild = 2 drops every
    tight attempt, so the second attempt runs); every setting gives the
    oracle's run, and the tight attempt leaves a smaller table."""
    c = make_config("lfr", n=20000, k=8, cmin=20, cmax=1000, max_deg=1000, seed=11)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 20)
    assert_same(gpu_run(cc, ro, col, lab, 20, sweep_mode=mode, tight_rebuild=tight), ref)
    caps = []
    for t in (tight, 1):
        with cc.Consensus(ro, col, lab, options(cc, sweep_mode=mode, tight_rebuild=t)) as job:
            job.sweep()  # the singleton start: always the safe capacity
            assert job.sweep() == ref.stats[1]
            caps.append(job.table_stats()["capacity"])
    if tight == 0:
        assert caps[0] < caps[1]  # the second sweep is heavy and its tight attempt fits
    else:
        assert caps[0] == caps[1]


@pytest.mark.parametrize("mode", MODES)
def test_no_regions_same_results(cc, mode):
    """Sweep graphs without conditional regions (every kernel a plain node,
    for profilers) give the same runs; their launch count is 55 kernels per
    sweep body."""
    c = make_config("lfr", n=20000, k=8, cmin=20, cmax=1000, max_deg=1000, seed=11)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 20)
    assert_same(gpu_run(cc, ro, col, lab, 20, sweep_mode=mode, no_regions=1), ref)
    with cc.Consensus(ro, col, lab, options(cc, no_regions=1, sweep_mode=mode)) as job:
        base = job.launch_count()
        done = job.run_until_converged(20)
        assert job.launch_count() - base == 1 + ((done + 3) // 4) * 4 * 55


# --------------------------------------------- move-to-empty variant (option)


def _random_grouping(rng, n, groups):
    """A warm start: vertices grouped at random, each group's id a random
    member (so most ids are free for the move-to-empty variant)."""
    cls = rng.integers(0, groups, n)
    C = np.empty(n, np.int32)
    for g in np.unique(cls):
        mem = np.nonzero(cls == g)[0]
        C[mem] = rng.choice(mem)
    return C


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("active", [0, 1])
def test_empty_moves_warm_start(cc, mode, active):
    """cc_options.empty_moves from random groupings (many vertices in the
    wrong cluster, most ids free): sweep by sweep, the records and raw ids
    equal the oracle's variant, in every sweep mode, with and without the
    active set; the empty move is taken."""
    isolated = 0
    for seed, (n, k) in enumerate([(3000, 8), (1500, 37), (4000, 3)]):
        c = make_config("lfr", n=n, k=k, cmin=20, cmax=300, max_deg=min(300, n // 4), seed=40 + seed)
        ro, col, lab = c["row_off"], c["col"], c["labels"]
        rng = np.random.default_rng(50 + seed)
        C = _random_grouping(rng, n, n // 40)
        ref = oracle.sync_run(ro, col, lab, 30, C0=C, empty=True)
        with cc.Consensus(ro, col, lab, options(cc, sweep_mode=mode, active_set=active, empty_moves=1)) as job:
            job.set_cluster_ids(C)
            assert job.run_until_converged(30) == ref.sweeps
            assert job.history() == ref.stats
            np.testing.assert_array_equal(job.cluster_ids(), ref.C)
            assert job.objective() == ref.F == job.objective_recompute()
        sizes = np.bincount(ref.C, minlength=n)
        isolated += int(np.sum((ref.C == np.arange(n)) & (C != np.arange(n))))
    assert isolated > 0


@pytest.mark.parametrize("mode", MODES)
def test_empty_moves_from_singletons(cc, mode):
    """The variant from the singleton start on the small SBM and a kNN graph:
    equal to the oracle's variant, sweep by sweep."""
    for c in (make_config("sbm"), make_config("knn", n=6000, comps=30, dim=20, k=12, seed=21)):
        ro, col, lab = c["row_off"], c["col"], c["labels"]
        ref = oracle.sync_run(ro, col, lab, 30, empty=True)
        assert_same(gpu_run(cc, ro, col, lab, 30, sweep_mode=mode, empty_moves=1), ref)


def test_empty_moves_golden(cc):
    """The hand-worked sweep where a vertex leaves its cluster for a new one."""
    with open(os.path.join(GOLDEN, "empty_move_path3.json")) as f:
        g = json.load(f)
    ro, col = _edges(g["n"], g["edges"])
    lab = np.array(g["labels"], np.int32)
    with cc.Consensus(ro, col, lab, options(cc, empty_moves=1)) as job:
        job.set_cluster_ids(np.array(g["C0"], np.int32))
        assert job.objective() == g["F0"]
        for want in g["sweeps"]:
            info = job.sweep()
            assert info == {key: want[key] for key in info}
            np.testing.assert_array_equal(job.cluster_ids(), want["C"])


# ------------------------------------------- colour-batched variant (option)


@pytest.mark.parametrize("mode", MODES)
def test_colour_batched_runs(cc, mode):
    """cc_options.colour_batched: every sweep record (sums over the colour
    classes), the raw ids and F equal the oracle's colour-batched run, on the
    small SBM, an LFR-style graph with hubs and a kNN graph, in every sweep
    mode; with the move-to-empty variant too on one of them."""
    cases = [(make_config("sbm"), False),
             (make_config("lfr", n=20000, k=8, cmin=20, cmax=1000, max_deg=1000, seed=11), False),
             (make_config("knn", n=6000, comps=30, dim=20, k=12, seed=21), True)]
    for c, empty in cases:
        ro, col, lab = c["row_off"], c["col"], c["labels"]
        ref = oracle.colour_run(ro, col, lab, 20, empty=empty)
        assert_same(gpu_run(cc, ro, col, lab, 20, sweep_mode=mode, colour_batched=1,
                            empty_moves=1 if empty else 0), ref)


def test_colour_batched_stepwise_and_warm_start(cc):
    """One sweep at a time (cc_sweep runs every class once) from a random
    warm start, against the oracle sweep by sweep; then a reset repeats the
    run from the singleton start."""
    c = make_config("lfr", n=5003, k=37, cmin=20, cmax=1000, max_deg=1000, seed=12)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    rng = np.random.default_rng(3)
    C0 = _random_grouping(rng, 5003, 200)
    ref = oracle.colour_run(ro, col, lab, 25, C0=C0)
    with cc.Consensus(ro, col, lab, options(cc, colour_batched=1)) as job:
        job.set_cluster_ids(C0)
        for want in ref.stats:
            assert job.sweep() == want
        np.testing.assert_array_equal(job.cluster_ids(), ref.C)
        job.reset()
        ref2 = oracle.colour_run(ro, col, lab, 20)
        assert job.run_until_converged(20) == ref2.sweeps
        assert job.history() == ref2.stats


# ------------------------------------------------------------- autotune


def test_autotune_same_results_and_record(cc):
    """cc_options.autotune: the first run times the candidate lane counts on
    the state after its first sweep and keeps the fastest; the run equals the
    oracle's, the choice is recorded for the lane bin, and a second context of
    that bin reuses it with identical results."""
    from paper_2408_11331_gb300 import _native
    import ctypes

    c = make_config("lfr", n=20000, k=37, cmin=20, cmax=1000, max_deg=1000, seed=17)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 20)
    assert_same(gpu_run(cc, ro, col, lab, 20, autotune=1), ref)
    rec = (ctypes.c_int32 * 6)()
    _native._check(_native.lib.cc_autotune_record(6, rec), None)
    assert rec[2] in (2, 4, 8)  # k = 37 is in the bin of 21..40 partitions (4 lanes automatic)
    with cc.Consensus(ro, col, lab, options(cc, autotune=1)) as job:
        for _ in range(2):
            job.reset()
            assert job.run_until_converged(20) == ref.sweeps
            assert job.history() == ref.stats
            np.testing.assert_array_equal(job.cluster_ids(), ref.C)
