"""Batched form: many independent jobs in one context, per job bit-exact.

Every job of a batch must end exactly where the oracle's synchronous run of
that job alone ends: the same number of sweeps, the same per-sweep records,
the same raw cluster ids and labels, the same objective.  The jobs differ in
n, k and structure so that they stop at different sweeps, share warps and
blocks of every kernel, and mix the sweep modes' heavy and light paths.
"""
import numpy as np
import pytest

import oracle
from workloads import csr_from_edges
from workloads.configs import make_job

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2408_11331_gb300 as m

    return m


def options(cc, **kw):
    o = cc.cc_default_options()
    for key, val in kw.items():
        setattr(o, key, val)
    return o


def _special_jobs():
    rng = np.random.default_rng(77)
    out = []
    # no edges: stops after one sweep with no proposal
    out.append((np.zeros(41, np.int64), np.zeros(0, np.int32), rng.integers(0, 3, (3, 40)).astype(np.int32)))
    # one vertex
    out.append((np.zeros(2, np.int64), np.zeros(0, np.int32), np.array([[4], [9], [1]], np.int32)))
    # star: the centre has 70 singleton neighbours
    e = np.array([(0, i) for i in range(1, 71)], np.int64)
    ro, col = csr_from_edges(71, e[:, 0], e[:, 1])
    out.append((ro, col, rng.integers(0, 2, (7, 71)).astype(np.int32)))
    # two cliques, identical labels
    pairs = [(i, j) for i in range(8) for j in range(i + 1, 8)] + \
            [(i, j) for i in range(8, 20) for j in range(i + 1, 20)] + [(7, 8)]
    e = np.array(pairs, np.int64)
    ro, col = csr_from_edges(20, e[:, 0], e[:, 1])
    out.append((ro, col, np.array([[0] * 8 + [1] * 12] * 4, np.int32)))
    return out


def _mixed_jobs(count, seed, nmax=3000):
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(count):
        n = int(np.exp(rng.uniform(np.log(60), np.log(nmax))))
        kind = "sbm" if j % 2 == 0 else "lfr"
        k = int(rng.integers(1, 70))
        d = make_job(np.random.default_rng(int(rng.integers(0, 2 ** 62))), n, kind, k)
        jobs.append((d["row_off"], d["col"], d["labels"]))
    return jobs


def _check_batch(b, jobs, refs):
    ids = b.cluster_ids()
    lab_all = b.consensus_labels()
    for j, ((ro, col, lab), ref) in enumerate(zip(jobs, refs)):
        lo, hi = b.offsets[j], b.offsets[j + 1]
        assert b.history(j) == ref.stats, f"job {j}"
        assert b.sweeps(j) == ref.sweeps, f"job {j}"
        assert b.objective(j) == ref.F, f"job {j}"
        np.testing.assert_array_equal(ids[lo:hi], ref.C, err_msg=f"job {j}")
        want = oracle.renumber(ref.C)
        np.testing.assert_array_equal(lab_all[lo:hi], want, err_msg=f"job {j}")
        np.testing.assert_array_equal(b.labels(j), want, err_msg=f"job {j}")


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_mixed_jobs(cc, mode):
    jobs = _special_jobs() + _mixed_jobs(24, 101)
    rng = np.random.default_rng(3)
    order = rng.permutation(len(jobs))
    jobs = [jobs[i] for i in order]
    refs = [oracle.sync_run(ro, col, lab, 20) for ro, col, lab in jobs]
    assert len({r.sweeps for r in refs}) > 2  # the jobs stop at different sweeps
    with cc.ConsensusBatch(jobs, options(cc, sweep_mode=mode)) as b:
        assert b.jobs == len(jobs)
        done = b.run_until_converged(20)
        assert done == max(r.sweeps for r in refs)
        _check_batch(b, jobs, refs)


@pytest.mark.parametrize("mode", [0, 2])
def test_batch_tight_attempt_dropped(cc, mode):
    """tight_rebuild = 2: every heavy rebuild's tight attempt is dropped and
    built again at the safe capacity (the second attempt, with the build's
    part of F' cleared); the jobs still match the oracle."""
    jobs = _special_jobs() + _mixed_jobs(24, 101)
    refs = [oracle.sync_run(ro, col, lab, 20) for ro, col, lab in jobs]
    with cc.ConsensusBatch(jobs, options(cc, sweep_mode=mode, tight_rebuild=2)) as b:
        assert b.run_until_converged(20) == max(r.sweeps for r in refs)
        _check_batch(b, jobs, refs)


def test_batch_run_and_result_names(cc):
    """cc_batch_run and cc_batch_result (the batch interface under its first
    names) give the oracle's run, as cc_run_until_converged, cc_job_labels and
    cc_job_objective do."""
    from paper_2408_11331_gb300 import _native

    jobs = _mixed_jobs(6, 303)
    refs = [oracle.sync_run(ro, col, lab, 20) for ro, col, lab in jobs]
    with cc.ConsensusBatch(jobs) as b:
        _native.cc_batch_run(b._ctx, 20)
        for j, ref in enumerate(refs):
            lab, F = _native.cc_batch_result(b._ctx, j, b.sizes[j])
            np.testing.assert_array_equal(lab, oracle.renumber(ref.C), err_msg=f"job {j}")
            assert F == ref.F, f"job {j}"
            assert b.sweeps(j) == ref.sweeps, f"job {j}"


def test_batch_many_small_jobs(cc):
    """Hundreds of jobs of a few hundred vertices: many jobs share each warp."""
    jobs = _mixed_jobs(300, 202, nmax=400)
    refs = [oracle.sync_run(ro, col, lab, 20) for ro, col, lab in jobs]
    with cc.ConsensusBatch(jobs) as b:
        b.run_until_converged(20)
        _check_batch(b, jobs, refs)


def test_batch_sweep_limit_and_continue(cc):
    """A run limited to 2 sweeps stops every job at 2; a second run continues
    each job from where it stopped, as the oracle does from that consensus."""
    jobs = _mixed_jobs(10, 303)
    with cc.ConsensusBatch(jobs) as b:
        assert b.run_until_converged(2) == 2
        ids = b.cluster_ids()
        firsts = []
        for j, (ro, col, lab) in enumerate(jobs):
            r = oracle.sync_run(ro, col, lab, 2)
            assert b.history(j) == r.stats
            np.testing.assert_array_equal(ids[b.offsets[j]:b.offsets[j + 1]], r.C)
            firsts.append(r)
        b.run_until_converged(20)
        ids = b.cluster_ids()
        for j, (ro, col, lab) in enumerate(jobs):
            r = oracle.sync_run(ro, col, lab, 20, C0=firsts[j].C)
            assert b.history(j) == firsts[j].stats + r.stats
            np.testing.assert_array_equal(ids[b.offsets[j]:b.offsets[j + 1]], r.C)


def test_batch_stepwise(cc):
    """Sweep by sweep (cc_sweep on a batch): each job follows the oracle step by step."""
    jobs = _special_jobs() + _mixed_jobs(6, 404)
    Cs = [oracle.singletons(len(ro) - 1) for ro, _, _ in jobs]
    Fs = [oracle.objective(lab, C) for (_, _, lab), C in zip(jobs, Cs)]
    stopped = [False] * len(jobs)
    with cc.ConsensusBatch(jobs, options(cc, sweep_mode=1)) as b:
        for j in range(len(jobs)):
            assert b.objective(j) == Fs[j]
        for _ in range(25):
            b.sweep()
            ids = b.cluster_ids()
            for j, (ro, col, lab) in enumerate(jobs):
                if stopped[j]:
                    continue
                r = oracle.sync_step(ro, col, lab, Cs[j], Fs[j])
                assert b.history(j)[-1] == r.stats
                np.testing.assert_array_equal(ids[b.offsets[j]:b.offsets[j + 1]], r.C)
                Cs[j], Fs[j] = r.C, r.stats["F"]
                stopped[j] = r.stats["proposals"] == 0
            if all(stopped):
                break
        assert all(stopped)


def test_batch_warm_start_job_local_ids(cc):
    """cc_set_cluster_ids takes job-local ids; the warm-started batch matches
    the oracle started from the same consensus."""
    jobs = _mixed_jobs(5, 505)
    rng = np.random.default_rng(9)
    C0 = []
    for ro, _, lab in jobs:
        n = len(ro) - 1
        C0.append(rng.integers(0, max(1, n // 5), n).astype(np.int32))
    with cc.ConsensusBatch(jobs) as b:
        b.set_cluster_ids(np.concatenate(C0))
        for j, (_, _, lab) in enumerate(jobs):
            assert b.objective(j) == oracle.objective(lab, C0[j])
        b.run_until_converged(20)
        ids = b.cluster_ids()
        for j, (ro, col, lab) in enumerate(jobs):
            r = oracle.sync_run(ro, col, lab, 20, C0=C0[j])
            assert b.history(j) == r.stats
            np.testing.assert_array_equal(ids[b.offsets[j]:b.offsets[j + 1]], r.C)


def test_batch_rejects_foreign_ids(cc):
    """An id outside its own job's range is rejected and the state is kept."""
    jobs = _mixed_jobs(3, 606)
    with cc.ConsensusBatch(jobs) as b:
        before = b.cluster_ids()
        bad = before.copy()
        bad[b.offsets[1]] = b.sizes[1]  # one past job 1's last vertex
        with pytest.raises(cc.CCError) as e:
            b.set_cluster_ids(bad)
        assert e.value.status == 1
        np.testing.assert_array_equal(b.cluster_ids(), before)
        b.run_until_converged(20)
        for j, (ro, col, lab) in enumerate(jobs):
            assert b.history(j) == oracle.sync_run(ro, col, lab, 20).stats


def test_batch_reset_repeats_the_run(cc):
    jobs = _mixed_jobs(8, 707)
    with cc.ConsensusBatch(jobs) as b:
        b.run_until_converged(20)
        first = [b.history(j) for j in range(b.jobs)]
        ids = b.cluster_ids()
        b.reset()
        for j in range(b.jobs):
            assert b.history(j) == []
        b.run_until_converged(20)
        assert [b.history(j) for j in range(b.jobs)] == first
        np.testing.assert_array_equal(b.cluster_ids(), ids)


def test_batch_single_job_calls_refused(cc):
    jobs = _mixed_jobs(2, 808)
    with cc.ConsensusBatch(jobs) as b:
        for call in (lambda: cc._native.cc_history(b._ctx), lambda: cc._native.cc_objective(b._ctx),
                     lambda: cc._native.cc_objective_recompute(b._ctx), lambda: cc._native.cc_sweep(b._ctx)):
            with pytest.raises(cc.CCError) as e:
                call()
            assert e.value.status == 1
        with pytest.raises(cc.CCError):
            cc._native.cc_job_objective(b._ctx, 2)


def test_batch_malformed_job_named(cc):
    jobs = _mixed_jobs(4, 909)
    ro, col, lab = jobs[2]
    col = col.copy()
    col[0] = len(ro) - 1  # out of range for its own job
    jobs[2] = (ro, col, lab)
    with pytest.raises(cc.CCError) as e:
        cc.ConsensusBatch(jobs)
    assert e.value.status == 1


def test_batch_of_one_equals_single(cc):
    ro, col, lab = _mixed_jobs(1, 1001)[0]
    with cc.ConsensusBatch([(ro, col, lab)]) as b, cc.Consensus(ro, col, lab) as s:
        b.run_until_converged(20)
        s.run_until_converged(20)
        assert b.history(0) == s.history()
        np.testing.assert_array_equal(b.cluster_ids(), s.cluster_ids())
        assert b.objective(0) == s.objective() == s.objective_recompute()


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_active_set(cc, mode):
    """A batch with the active set: jobs stop at different sweeps, and a
    stopped job's vertices never repeat an old bid."""
    jobs = _special_jobs() + _mixed_jobs(20, 111)
    refs = [oracle.sync_run(ro, col, lab, 20) for ro, col, lab in jobs]
    assert len({r.sweeps for r in refs}) > 2
    with cc.ConsensusBatch(jobs, options(cc, sweep_mode=mode, active_set=1)) as b:
        assert b.run_until_converged(20) == max(r.sweeps for r in refs)
        _check_batch(b, jobs, refs)


def test_batch_empty_moves(cc):
    """The move-to-empty variant in a batch from job-local warm starts: each
    job equals the oracle's variant started from the same consensus."""
    jobs = _mixed_jobs(4, 515)
    rng = np.random.default_rng(10)
    C0 = []
    for ro, _, lab in jobs:
        n = len(ro) - 1
        cls = rng.integers(0, max(1, n // 30), n)
        C = np.empty(n, np.int32)
        for g in np.unique(cls):
            mem = np.nonzero(cls == g)[0]
            C[mem] = rng.choice(mem)
        C0.append(C)
    o = cc.cc_default_options()
    o.empty_moves = 1
    with cc.ConsensusBatch(jobs, o) as b:
        b.set_cluster_ids(np.concatenate(C0))
        b.run_until_converged(30)
        ids = b.cluster_ids()
        for j, (ro, col, lab) in enumerate(jobs):
            r = oracle.sync_run(ro, col, lab, 30, C0=C0[j], empty=True)
            assert b.history(j) == r.stats
            np.testing.assert_array_equal(ids[b.offsets[j]:b.offsets[j + 1]], r.C)


def test_batch_colour_batched(cc):
    """Colour-batched sweeps over a batch: jobs with different numbers of
    colour classes run the classes in lockstep; each job equals the oracle's
    colour-batched run of that job alone."""
    jobs = _mixed_jobs(5, 525)
    o = cc.cc_default_options()
    o.colour_batched = 1
    with cc.ConsensusBatch(jobs, o) as b:
        b.run_until_converged(20)
        ids = b.cluster_ids()
        for j, (ro, col, lab) in enumerate(jobs):
            r = oracle.colour_run(ro, col, lab, 20)
            assert b.history(j) == r.stats
            np.testing.assert_array_equal(ids[b.offsets[j]:b.offsets[j + 1]], r.C)


def test_batch_autotune(cc):
    """Autotuned lanes in a batch: every job equals the oracle's run alone."""
    jobs = _mixed_jobs(6, 535)
    o = cc.cc_default_options()
    o.autotune = 1
    o.active_set = 1
    with cc.ConsensusBatch(jobs, o) as b:
        b.run_until_converged(20)
        ids = b.cluster_ids()
        for j, (ro, col, lab) in enumerate(jobs):
            r = oracle.sync_run(ro, col, lab, 20)
            assert b.history(j) == r.stats
            np.testing.assert_array_equal(ids[b.offsets[j]:b.offsets[j + 1]], r.C)
