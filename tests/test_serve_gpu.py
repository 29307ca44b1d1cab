"""Served form: jobs submitted while others run, continuously batched.

Each job's result must be what the oracle gives for that job alone, whatever
else was in flight with it: labels, objective and sweep count, bit-exact.
"""
import numpy as np
import pytest

import oracle
from workloads.configs import make_job

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2408_11331_gb300 as m

    return m


def _jobs(count, seed, nmin=100, nmax=4000, kmin=1, kmax=40):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        k = int(rng.integers(kmin, kmax + 1))
        d = make_job(np.random.default_rng(int(rng.integers(0, 2 ** 62))), n, "lfr" if j % 3 else "sbm", k)
        out.append((d["row_off"], d["col"], d["labels"]))
    return out


def _refs(jobs):
    return [oracle.sync_run(ro, col, lab, 20) for ro, col, lab in jobs]


def _check(srv, tickets, jobs, refs):
    for t, (ro, col, lab), ref in zip(tickets, jobs, refs):
        r = srv.result(t)
        assert r["done"] and r["status"] == 0, r
        assert r["sweeps"] == ref.sweeps
        assert r["F"] == ref.F
        np.testing.assert_array_equal(r["labels"], oracle.renumber(ref.C))


def test_serve_all_at_once(cc):
    jobs = _jobs(60, 1)
    refs = _refs(jobs)
    with cc.Server(max_active=4, max_batch_jobs=16) as srv:
        tickets = [srv.submit(*j) for j in jobs]
        order = srv.drain()
        assert sorted(order) == sorted(tickets)
        _check(srv, tickets, jobs, refs)
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 0
        assert st["batches"] >= len(jobs) // 16
        assert st["bytes_in_use"] == 0 and st["in_flight"] == 0


def test_serve_same_alone_and_in_mix(cc):
    """A job served alone and the same job served among others give the same result."""
    jobs = _jobs(30, 2)
    probe = jobs[7]
    with cc.Server() as srv:
        t = srv.submit(*probe)
        srv.drain()
        alone = srv.result(t)
    with cc.Server(max_active=3, max_batch_jobs=8) as srv:
        ts = [srv.submit(*j) for j in jobs]
        srv.drain()
        mixed = srv.result(ts[7])
    assert alone["F"] == mixed["F"] and alone["sweeps"] == mixed["sweeps"]
    np.testing.assert_array_equal(alone["labels"], mixed["labels"])
    ref = oracle.sync_run(*probe, 20)
    np.testing.assert_array_equal(mixed["labels"], oracle.renumber(ref.C))


def test_serve_arrivals_while_running(cc):
    """Jobs arrive in bursts between progress calls, so new contexts are
    admitted while earlier ones are still on the device."""
    jobs = _jobs(48, 3, nmax=20000)
    refs = _refs(jobs)
    with cc.Server(max_active=4, max_batch_jobs=6) as srv:
        tickets = []
        done = []
        for b in range(0, len(jobs), 6):
            tickets += [srv.submit(*j) for j in jobs[b:b + 6]]
            d, _ = srv.progress()
            done += d
        done += srv.drain()
        assert sorted(done) == sorted(tickets)
        _check(srv, tickets, jobs, refs)
        assert srv.stats()["max_in_flight"] >= 2


def test_serve_budget_limits_admission(cc):
    """A budget that holds about two jobs at a time: every job still finishes,
    and the bytes held never pass the budget."""
    jobs = _jobs(12, 4, nmin=3000, nmax=6000, kmin=10, kmax=20)
    refs = _refs(jobs)
    peaks = [cc._native.cc_estimate_bytes([(len(ro) - 1, len(col), lab.shape[0])])[1] for ro, col, lab in jobs]
    budget = int(2.2 * max(peaks))
    with cc.Server(budget_bytes=budget, max_active=8, max_batch_jobs=64) as srv:
        tickets = [srv.submit(*j) for j in jobs]
        srv.drain()
        _check(srv, tickets, jobs, refs)
        st = srv.stats()
        assert st["peak_bytes"] <= budget
        assert st["batches"] >= 4


def test_serve_oversize_job_fails_alone(cc):
    jobs = _jobs(5, 5, nmin=200, nmax=400)
    big = _jobs(1, 6, nmin=30000, nmax=30001, kmin=30, kmax=30)[0]
    small_peak = max(cc._native.cc_estimate_bytes([(len(ro) - 1, len(col), lab.shape[0])])[1] for ro, col, lab in jobs)
    big_peak = cc._native.cc_estimate_bytes([(len(big[0]) - 1, len(big[1]), big[2].shape[0])])[1]
    assert big_peak > 4 * small_peak
    with cc.Server(budget_bytes=4 * small_peak, max_batch_jobs=1) as srv:
        ts = [srv.submit(*j) for j in jobs[:2]] + [srv.submit(*big)] + [srv.submit(*j) for j in jobs[2:]]
        srv.drain()
        r = srv.result(ts[2])
        assert r["done"] and r["status"] == 2  # CC_ERR_OOM
        others = [t for i, t in enumerate(ts) if i != 2]
        _check(srv, others, jobs, _refs(jobs))
        assert srv.stats()["failed"] == 1


def test_serve_bins_by_k(cc):
    """Jobs of very different k go to different contexts (lane bins); with
    sizes alike, each bin is one context."""
    lo = _jobs(6, 7, nmin=1000, nmax=1100, kmin=2, kmax=5)
    hi = _jobs(6, 8, nmin=1000, nmax=1100, kmin=50, kmax=64)
    jobs = [j for pair in zip(lo, hi) for j in pair]
    refs = _refs(jobs)
    with cc.Server(max_active=2, max_batch_jobs=64) as srv:
        tickets = [srv.submit(*j) for j in jobs]
        srv.drain()
        _check(srv, tickets, jobs, refs)
        assert srv.stats()["batches"] == 2


def test_serve_size_classes(cc):
    """A job joins a context only if its n is within a factor 4 of the first
    job's, so a small job never waits for a large one."""
    small = _jobs(4, 10, nmin=200, nmax=220, kmin=10, kmax=10)
    large = _jobs(4, 11, nmin=5000, nmax=5200, kmin=10, kmax=10)
    jobs = [j for pair in zip(small, large) for j in pair]
    refs = _refs(jobs)
    with cc.Server(max_active=2, max_batch_jobs=64) as srv:
        tickets = [srv.submit(*j) for j in jobs]
        srv.drain()
        _check(srv, tickets, jobs, refs)
        assert srv.stats()["batches"] == 2


def test_estimate_covers_allocation(cc):
    """The bytes a context holds, seen as free device memory going down,
    match the estimate within allocation granularity."""
    import torch

    ro, col, lab = _jobs(1, 9, nmin=200000, nmax=200001, kmin=20, kmax=20)[0]
    est, peak = cc._native.cc_estimate_bytes([(len(ro) - 1, len(col), lab.shape[0])])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with cc.Consensus(ro, col, lab) as job:
        free1 = torch.cuda.mem_get_info()[0]
        held = free0 - free1
        assert 0.9 * est <= held <= est + (64 << 20)
        job.run_until_converged(20)


def _sweeps_and_job(seed, n, kind, k):
    d = make_job(np.random.default_rng(seed), n, kind, k)
    job = (d["row_off"], d["col"], d["labels"])
    return oracle.sync_run(*job, 20), job


def test_serve_releases_a_job_before_its_slowest_sibling(cc):
    """Two jobs of one context (same lane bin, sizes within a factor 4), one
    needing several sweeps fewer than the other: the short one is reported
    done while the context still runs the long one, and both equal the
    oracle's runs."""
    short = long_ = None
    for seed in range(200):
        ref, job = _sweeps_and_job(1000 + seed, 1500, "lfr" if seed % 2 else "sbm", 6)
        if short is None or ref.sweeps < short[0].sweeps:
            short = (ref, job)
        if long_ is None or ref.sweeps > long_[0].sweeps:
            long_ = (ref, job)
        if long_[0].sweeps - short[0].sweeps >= 4:
            break
    assert long_[0].sweeps - short[0].sweeps >= 4  # a graph launch runs 4 sweeps
    with cc.Server(max_active=1, max_batch_jobs=4) as srv:
        t_long = srv.submit(*long_[1])
        t_short = srv.submit(*short[1])
        seen = {}
        calls = 0
        while len(seen) < 2:
            done, _ = srv.progress(wait=True)
            calls += 1
            st = srv.stats()
            for t in done:
                seen[t] = (calls, st["in_flight"])
            assert calls < 10000
        assert srv.stats()["batches"] == 1  # both ran in one context
        assert seen[t_short][0] < seen[t_long][0]
        assert seen[t_short][1] == 1  # the context was still in flight
        for t, (ref, _) in ((t_short, short), (t_long, long_)):
            r = srv.result(t)
            assert r["status"] == 0 and r["sweeps"] == ref.sweeps and r["F"] == ref.F
            np.testing.assert_array_equal(r["labels"], oracle.renumber(ref.C))


def test_serve_loads_a_waiting_job_into_a_running_context(cc):
    """One context of two jobs (max_active 1): when its short job stops, a
    waiting job of the same lane bin that fits the short job's place is
    loaded into it while the long job keeps running (no new context), and
    every job equals the oracle's run of it alone.  The loaded job is
    smaller than the place, so the place's unused vertices and CSR entries
    are exercised."""
    cands = []
    for seed in range(200):
        ref, job = _sweeps_and_job(2000 + seed, 1500, "lfr" if seed % 2 else "sbm", 6)
        cands.append((ref, job))
    cands.sort(key=lambda rj: rj[0].sweeps)
    short, long_ = cands[0], cands[-1]
    assert long_[0].sweeps - short[0].sweeps >= 4
    ref_w, job_w = _sweeps_and_job(4242, 900, "lfr", 5)  # fewer vertices, edges, partitions
    assert len(job_w[0]) - 1 < len(short[1][0]) - 1 and len(job_w[1]) <= len(short[1][1])
    with cc.Server(max_active=1, max_batch_jobs=2) as srv:
        t_long = srv.submit(*long_[1])
        t_short = srv.submit(*short[1])
        srv.progress()  # both admitted into one context
        t_w = srv.submit(*job_w)
        srv.drain()
        st = srv.stats()
        assert st["batches"] == 1 and st["admitted_running"] == 1, st
        for t, ref in ((t_long, long_[0]), (t_short, short[0]), (t_w, ref_w)):
            r = srv.result(t)
            assert r["status"] == 0 and r["sweeps"] == ref.sweeps and r["F"] == ref.F, (t, r["F"], ref.F)
            np.testing.assert_array_equal(r["labels"], oracle.renumber(ref.C))


@pytest.mark.timeout(300)
def test_serve_many_loads_into_one_context(cc):
    """Forty jobs of similar size through one context of eight places: most
    jobs are loaded into the place of a finished one (the table keeps the
    other jobs' counts, or is rebuilt when it would run short), and every job
    equals the oracle's run of it alone."""
    rng = np.random.default_rng(77)
    jobs = []
    for j in range(40):
        d = make_job(np.random.default_rng(int(rng.integers(0, 2 ** 62))), int(rng.integers(1200, 1600)),
                     "lfr" if j % 2 else "sbm", int(rng.integers(8, 11)))
        jobs.append((d["row_off"], d["col"], d["labels"]))
    refs = _refs(jobs)
    with cc.Server(max_active=1, max_batch_jobs=8) as srv:
        tickets = [srv.submit(*j) for j in jobs]
        srv.drain()
        st = srv.stats()
        assert st["completed"] == 40 and st["failed"] == 0
        assert st["admitted_running"] >= 10, st
        _check(srv, tickets, jobs, refs)
