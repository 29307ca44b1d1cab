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
