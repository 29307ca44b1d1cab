"""GB300-native median consensus clustering sweep (arXiv 2408.11331).

The work runs in ``libcc.so`` (hand-written CUDA for sm_103a behind the C ABI
of ``include/cc.h``).  This package is the thin Python layer over it:

* ``_native``   one ctypes function per C entry point, same names
* ``Consensus`` a small object wrapper owning one context (one job)
* ``ConsensusBatch`` the same for a batch of independent jobs in one context
* ``Server``    the served form: jobs submitted as they arrive, continuously batched

Importing the package loads libcc.so and raises if it is missing.
"""
from __future__ import annotations

import numpy as np

from . import _native
from ._native import CCError, cc_options, cc_default_options  # noqa: F401


class Consensus:
    """One consensus job: graph + k input partitions, resident on the GPU.

    ``Consensus(row_off, col, labels)`` with host numpy arrays (row_off
    int64[n+1], col int32[nnz], labels int32[k, n]) or
    ``Consensus.from_device(...)`` with device buffers.
    """

    def __init__(self, row_off=None, col=None, labels=None, options=None, _ctx=None, _n=None, _k=None):
        if _ctx is not None:
            self._ctx, self.n, self.k = _ctx, _n, _k
            return
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        self.k, self.n = labels.shape
        self._ctx = _native.cc_create(row_off, col, labels, options)

    @classmethod
    def from_device(cls, n, nnz, row_off_ptr, col_ptr, k, labels_ptr, options=None, stream=0):
        ctx = _native.cc_create_dev(n, nnz, row_off_ptr, col_ptr, k, labels_ptr, options, stream)
        return cls(_ctx=ctx, _n=n, _k=k)

    def set_cluster_ids(self, C):
        if len(C) != self.n:
            raise ValueError("C must have n entries")
        _native.cc_set_cluster_ids(self._ctx, C)

    def sweep(self) -> dict:
        return _native.cc_sweep(self._ctx)

    def run_until_converged(self, max_sweeps: int = 0) -> int:
        return _native.cc_run_until_converged(self._ctx, max_sweeps)

    def last_run_timing(self):
        return _native.cc_last_run_timing(self._ctx)

    def table_stats(self) -> dict:
        return _native.cc_table_stats(self._ctx)

    def launch_count(self) -> int:
        return _native.cc_launch_count(self._ctx)

    def history(self) -> list:
        return _native.cc_history(self._ctx)

    def objective(self) -> int:
        return _native.cc_objective(self._ctx)

    def objective_recompute(self) -> int:
        return _native.cc_objective_recompute(self._ctx)

    def metrics(self) -> dict:
        """Mirkin, split-join, Rand and VI distances of the consensus to each input partition."""
        return _native.cc_metrics(self._ctx, self.k)

    def partition_distances(self) -> dict:
        """k x k distances between the input partitions (the consensus is left as it was)."""
        return _native.cc_partition_distances(self._ctx, self.k)

    def consensus_labels(self) -> np.ndarray:
        return _native.cc_consensus_labels(self._ctx, self.n)

    def cluster_ids(self) -> np.ndarray:
        return _native.cc_cluster_ids(self._ctx, self.n)

    def cluster_ids_dev(self) -> int:
        return _native.cc_cluster_ids_dev(self._ctx)

    def set_stream(self, stream: int = 0):
        _native.cc_set_stream(self._ctx, stream)

    def reset(self):
        _native.cc_reset(self._ctx)

    def close(self):
        if self._ctx is not None:
            _native.cc_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ConsensusBatch:
    """Many independent consensus jobs in one context (one disjoint union on
    the device; every sweep runs all jobs in the same launches).

    ``ConsensusBatch([(row_off, col, labels), ...])`` with host numpy arrays
    per job, as for ``Consensus``.  Per-job results come from ``objective(j)``,
    ``history(j)`` and ``labels(j)``; ``cluster_ids()`` / ``consensus_labels()``
    give all jobs at once, job after job, each local to its job.
    """

    def __init__(self, jobs, options=None):
        jobs = list(jobs)
        self.sizes = [int(np.asarray(lab).shape[1]) for _, _, lab in jobs]
        self.ks = [int(np.asarray(lab).shape[0]) for _, _, lab in jobs]
        self.n = sum(self.sizes)
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self._ctx = _native.cc_batch_create(jobs, options)

    @property
    def jobs(self) -> int:
        return len(self.sizes)

    def sweep(self):
        _native.cc_sweep(self._ctx, info=False)

    def run_until_converged(self, max_sweeps: int = 0) -> int:
        return _native.cc_run_until_converged(self._ctx, max_sweeps)

    def last_run_timing(self):
        return _native.cc_last_run_timing(self._ctx)

    def table_stats(self) -> dict:
        return _native.cc_table_stats(self._ctx)

    def launch_count(self) -> int:
        return _native.cc_launch_count(self._ctx)

    def objective(self, job: int) -> int:
        return _native.cc_job_objective(self._ctx, job)[0]

    def sweeps(self, job: int) -> int:
        return _native.cc_job_objective(self._ctx, job)[1]

    def history(self, job: int) -> list:
        return _native.cc_job_history(self._ctx, job)

    def labels(self, job: int) -> np.ndarray:
        return _native.cc_job_labels(self._ctx, job, self.sizes[job])

    def metrics(self) -> list:
        """Per job, the distances of its consensus to each of its input partitions."""
        m = _native.cc_metrics(self._ctx, int(sum(self.ks)))
        out, at = [], 0
        for k in self.ks:
            out.append({f: v[at:at + k] for f, v in m.items()})
            at += k
        return out

    def consensus_labels(self) -> np.ndarray:
        return _native.cc_consensus_labels(self._ctx, self.n)

    def cluster_ids(self) -> np.ndarray:
        return _native.cc_cluster_ids(self._ctx, self.n)

    def set_cluster_ids(self, C):
        if len(C) != self.n:
            raise ValueError("C must have sum n_j entries")
        _native.cc_set_cluster_ids(self._ctx, C)

    def set_stream(self, stream: int = 0):
        _native.cc_set_stream(self._ctx, stream)

    def reset(self):
        _native.cc_reset(self._ctx)

    def close(self):
        if self._ctx is not None:
            _native.cc_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop with continuous batching (the library's cc_server).

    ``submit(row_off, col, labels)`` queues a job and returns its ticket; the
    arrays are kept referenced here until the job is done.  ``progress()``
    advances the server and returns the tickets finished since the last call;
    ``result(ticket)`` gives the labels, objective, sweeps and status.
    """

    def __init__(self, budget_bytes: int = 0, max_active: int = 0, max_batch_jobs: int = 0, options=None):
        so = _native.cc_server_default_options()
        so.budget_bytes = budget_bytes
        if max_active:
            so.max_active = max_active
        if max_batch_jobs:
            so.max_batch_jobs = max_batch_jobs
        self._srv = _native.cc_server_create(so, options)
        self._live = {}
        self._out = {}

    def submit(self, row_off, col, labels) -> int:
        keep = []
        desc = _native._job_desc(row_off, col, labels, keep)
        out = np.empty(desc.n, np.int32)
        t = _native.cc_server_submit(self._srv, desc, out)
        self._live[t] = (keep, desc)
        self._out[t] = out
        return t

    def progress(self, wait: bool = False):
        done, pending = _native.cc_server_progress(self._srv, wait)
        for t in done:
            self._live.pop(t, None)
        return done, pending

    def result(self, ticket: int, pop: bool = False) -> dict:
        """Labels, objective, sweeps and status of a job; pop=True also drops
        the labels buffer kept here once the job is done."""
        r = _native.cc_server_job(self._srv, ticket)
        r["labels"] = (self._out.pop(ticket) if pop else self._out[ticket]) if r["done"] else None
        return r

    def drain(self):
        """Runs until every submitted job is done; returns the tickets in finishing order."""
        order = []
        while True:
            done, pending = self.progress(wait=True)
            order += done
            if pending == 0:
                done, _ = self.progress()
                return order + done

    def stats(self) -> dict:
        return _native.cc_server_stats(self._srv)

    def close(self):
        if self._srv is not None:
            _native.cc_server_destroy(self._srv)
            self._srv = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
