"""GB300-native median consensus clustering sweep (arXiv 2408.11331).

The work runs in ``libcc.so`` (hand-written CUDA for sm_103a behind the C ABI
of ``include/cc.h``).  This package is the thin Python layer over it:

* ``_native``   one ctypes function per C entry point, same names
* ``Consensus`` a small object wrapper owning one context

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
