"""Partition distances on the GPU (Methods, Evaluation metrics) against the
oracle: Mirkin and split-join exact, Rand distance and variation of
information within fp64 summation error."""
import numpy as np
import pytest

import oracle
from workloads import make_config
from workloads.configs import make_job

pytestmark = pytest.mark.gpu

# VI is a difference of fp64 sums of up to n terms |c| log |c| <= n log n,
# accumulated in an unfixed order on the GPU: 1e-9 nats is far above that
# rounding at the sizes tested and far below any real difference.
VI_TOL = 1e-9


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2408_11331_gb300 as m

    return m


def _same(got, want):
    np.testing.assert_array_equal(got["mirkin"], want["mirkin"])
    np.testing.assert_array_equal(got["split_join"], want["split_join"])
    np.testing.assert_allclose(got["rand_distance"], want["rand_distance"], rtol=1e-14, atol=0)
    np.testing.assert_allclose(got["vi"], want["vi"], rtol=0, atol=VI_TOL)


@pytest.mark.parametrize("name,kw", [("sbm", {}), ("lfr", dict(n=20000, k=8, cmin=20, cmax=1000, max_deg=1000, seed=11)),
                                     ("lfr", dict(n=5003, k=37, cmin=20, cmax=1000, max_deg=1000, seed=12))])
def test_metrics_after_run(cc, name, kw):
    c = make_config(name, **kw)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    with cc.Consensus(ro, col, lab) as job:
        start = job.metrics()  # singleton start, before any table exists
        _same(start, oracle.metrics(lab, oracle.singletons(len(ro) - 1)))
        job.run_until_converged(20)
        C = job.cluster_ids()
        got = job.metrics()
        _same(got, oracle.metrics(lab, C))
        assert int(got["mirkin"].sum()) == job.objective()


def test_metrics_do_not_change_the_run(cc):
    c = make_config("lfr", n=20000, k=8, cmin=20, cmax=1000, max_deg=1000, seed=11)
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    ref = oracle.sync_run(ro, col, lab, 20)
    with cc.Consensus(ro, col, lab) as job:
        job.run_until_converged(2)
        job.metrics()
        job.run_until_converged(20)
        assert job.history() == ref.stats
        np.testing.assert_array_equal(job.cluster_ids(), ref.C)


def test_metrics_warm_start(cc):
    c = make_config("sbm")
    ro, col, lab = c["row_off"], c["col"], c["labels"]
    rng = np.random.default_rng(4)
    C0 = rng.integers(0, 50, len(ro) - 1).astype(np.int32)
    with cc.Consensus(ro, col, lab) as job:
        job.set_cluster_ids(C0)
        _same(job.metrics(), oracle.metrics(lab, C0))


def test_metrics_batch(cc):
    rng = np.random.default_rng(8)
    jobs = []
    for j in range(12):
        n = int(rng.integers(50, 3000))
        d = make_job(np.random.default_rng(int(rng.integers(0, 2 ** 62))), n, "lfr" if j % 2 else "sbm",
                     int(rng.integers(1, 40)))
        jobs.append((d["row_off"], d["col"], d["labels"]))
    with cc.ConsensusBatch(jobs) as b:
        b.run_until_converged(20)
        ids = b.cluster_ids()
        per_job = b.metrics()
        for j, (ro, col, lab) in enumerate(jobs):
            _same(per_job[j], oracle.metrics(lab, ids[b.offsets[j]:b.offsets[j + 1]]))
            assert int(per_job[j]["mirkin"].sum()) == b.objective(j)


def test_partition_distances_and_groups(cc):
    """Pairwise distances of the input partitions against the oracle, the
    consensus left untouched, and one consensus per group of homogeneous
    partitions (Methods, Grouping homogeneous partitions) equal to the
    oracle's run on that group alone."""
    rng = np.random.default_rng(12)
    c = make_config("lfr", n=6000, k=4, cmin=20, cmax=1000, max_deg=500, seed=31)
    ro, col, lab4 = c["row_off"], c["col"], c["labels"]
    # two families: the 4 perturbed partitions, and 3 partitions scrambled far from them
    far = np.stack([rng.permutation(lab4[0]) for _ in range(3)]).astype(np.int32)
    lab = np.concatenate([lab4, far])
    k = lab.shape[0]
    with cc.Consensus(ro, col, lab) as job:
        job.run_until_converged(20)
        C, F, hist = job.cluster_ids(), job.objective(), job.history()
        d = job.partition_distances()
        np.testing.assert_array_equal(job.cluster_ids(), C)
        assert job.objective() == F == job.objective_recompute()
        job.run_until_converged(20)  # continues as if nothing happened: nothing left to move
        assert job.history()[: len(hist)] == hist and job.history()[-1]["proposals"] == 0
    for a in range(k):
        want = oracle.metrics(lab, lab[a])
        np.testing.assert_array_equal(d["split_join"][a], want["split_join"])
        np.testing.assert_array_equal(d["mirkin"][a], want["mirkin"])
        np.testing.assert_allclose(d["vi"][a], want["vi"], rtol=0, atol=VI_TOL)
    assert (np.diag(d["split_join"]) == 0).all() and (d["split_join"] == d["split_join"].T).all()
    # a threshold between the within-family and the cross distances
    within = d["split_join"][:4, :4].max()
    lam = int(within)
    groups, ng = cc._native.cc_group_partitions(d["split_join"], lam)
    assert groups[:4].tolist() == [0] * 4
    if d["split_join"][:4, 4:].min() > within:
        assert ng >= 2
    members = [np.nonzero(groups == g)[0] for g in range(ng)]
    jobs = [(ro, col, lab[m]) for m in members]
    with cc.ConsensusBatch(jobs) as b:
        b.run_until_converged(20)
        ids = b.cluster_ids()
        for g, m in enumerate(members):
            ref = oracle.sync_run(ro, col, lab[m], 20)
            assert b.history(g) == ref.stats
            np.testing.assert_array_equal(ids[b.offsets[g]:b.offsets[g + 1]], ref.C)
