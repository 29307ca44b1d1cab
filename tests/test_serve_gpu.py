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
