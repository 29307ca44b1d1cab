"""ctypes binding of libcc.so -- argument marshalling only.

Every function here mirrors one entry point of include/cc.h under the same
name; the work itself runs in the library's CUDA kernels.  There is no CPU
fallback: if libcc.so is missing or cannot be loaded, importing this module
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcc.so")

CC_OK = 0
STATUS_NAMES = {0: "CC_OK", 1: "CC_ERR_INVALID", 2: "CC_ERR_OOM", 3: "CC_ERR_CUDA", 4: "CC_ERR_OVERFLOW",
                5: "CC_ERR_TABLE_FULL", 6: "CC_ERR_TIMEOUT"}

# Every symbol include/cc.h declares; the CPU test suite checks the library exports them.
EXPORTS = ("cc_default_options", "cc_create", "cc_create_dev", "cc_set_stream", "cc_reset", "cc_set_cluster_ids", "cc_sweep",
           "cc_run_until_converged", "cc_last_run_timing", "cc_table_stats", "cc_launch_count", "cc_history", "cc_objective", "cc_objective_recompute",
           "cc_consensus_labels", "cc_cluster_ids", "cc_cluster_ids_dev", "cc_last_error", "cc_destroy",
           "cc_batch_create", "cc_job_count", "cc_job_objective", "cc_job_history", "cc_job_labels",
           "cc_batch_run", "cc_batch_result",
           "cc_metrics", "cc_partition_distances", "cc_group_partitions", "cc_estimate_bytes", "cc_plan_batches", "cc_server_default_options", "cc_server_create", "cc_server_submit",
           "cc_server_progress", "cc_server_job", "cc_server_stats", "cc_server_last_error", "cc_server_destroy",
           "cc_renumber_noalloc", "cc_noalloc_max_n", "cc_autotune_record")


class CCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class cc_options(ctypes.Structure):
    _fields_ = [("max_sweeps", ctypes.c_int32), ("debug_checks", ctypes.c_int32),
                ("table_log2", ctypes.c_int32), ("table_start_log2", ctypes.c_int32),
                ("sweep_mode", ctypes.c_int32), ("lanes", ctypes.c_int32), ("active_set", ctypes.c_int32),
                ("no_regions", ctypes.c_int32), ("empty_moves", ctypes.c_int32),
                ("colour_batched", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("tight_rebuild", ctypes.c_int32)]


class cc_table_info(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("max_capacity", ctypes.c_int64), ("live_keys", ctypes.c_int64),
                ("used_slots", ctypes.c_int64), ("rebuilds", ctypes.c_int64), ("retries", ctypes.c_int64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class cc_sweep_info(ctypes.Structure):
    _fields_ = [("proposals", ctypes.c_int64), ("p1", ctypes.c_int64), ("dF_p1", ctypes.c_int64),
                ("fallback", ctypes.c_int64), ("moves", ctypes.c_int64), ("F", ctypes.c_int64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class cc_partition_metrics(ctypes.Structure):
    _fields_ = [("mirkin", ctypes.c_int64), ("split_join", ctypes.c_int64), ("rand_distance", ctypes.c_double),
                ("vi", ctypes.c_double)]


class cc_job_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_off", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("k", ctypes.c_int32), ("labels", ctypes.c_void_p)]


class cc_server_options(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("max_batch_jobs", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class cc_server_info(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "admitted", "completed", "failed", "batches",
                                              "max_in_flight", "in_flight", "queued", "budget_bytes",
                                              "bytes_in_use", "peak_bytes", "admitted_running")]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing; build it with `python paper_2408_11331_gb300/build.py` "
                          "(nvcc, sm_103a). There is no CPU fallback.")
    lib = ctypes.CDLL(path)
    c = ctypes
    P = c.c_void_p
    lib.cc_default_options.restype = None
    lib.cc_default_options.argtypes = [c.POINTER(cc_options)]
    lib.cc_create.restype = c.c_int
    lib.cc_create.argtypes = [c.c_int32, c.c_int64, P, P, c.c_int32, P, c.POINTER(cc_options), c.POINTER(P)]
    lib.cc_create_dev.restype = c.c_int
    lib.cc_create_dev.argtypes = [c.c_int32, c.c_int64, P, P, c.c_int32, P, c.POINTER(cc_options), P,
                                  c.POINTER(P)]
    lib.cc_set_stream.restype = c.c_int
    lib.cc_set_stream.argtypes = [P, P]
    lib.cc_reset.restype = c.c_int
    lib.cc_reset.argtypes = [P]
    lib.cc_set_cluster_ids.restype = c.c_int
    lib.cc_set_cluster_ids.argtypes = [P, P]
    lib.cc_sweep.restype = c.c_int
    lib.cc_sweep.argtypes = [P, c.POINTER(cc_sweep_info)]
    lib.cc_run_until_converged.restype = c.c_int
    lib.cc_run_until_converged.argtypes = [P, c.c_int32, c.POINTER(c.c_int32)]
    lib.cc_last_run_timing.restype = c.c_int
    lib.cc_last_run_timing.argtypes = [P, c.c_int32, P, P, c.POINTER(c.c_int32)]
    lib.cc_table_stats.restype = c.c_int
    lib.cc_table_stats.argtypes = [P, c.POINTER(cc_table_info)]
    lib.cc_launch_count.restype = c.c_int
    lib.cc_launch_count.argtypes = [P, c.POINTER(c.c_int64)]
    lib.cc_history.restype = c.c_int
    lib.cc_history.argtypes = [P, c.c_int32, c.POINTER(cc_sweep_info), c.POINTER(c.c_int32)]
    lib.cc_objective.restype = c.c_int
    lib.cc_objective.argtypes = [P, c.POINTER(c.c_int64)]
    lib.cc_objective_recompute.restype = c.c_int
    lib.cc_objective_recompute.argtypes = [P, c.POINTER(c.c_int64)]
    lib.cc_consensus_labels.restype = c.c_int
    lib.cc_consensus_labels.argtypes = [P, P]
    lib.cc_cluster_ids.restype = c.c_int
    lib.cc_cluster_ids.argtypes = [P, P]
    lib.cc_cluster_ids_dev.restype = c.c_int
    lib.cc_cluster_ids_dev.argtypes = [P, c.POINTER(P)]
    lib.cc_last_error.restype = c.c_char_p
    lib.cc_last_error.argtypes = [P]
    lib.cc_destroy.restype = None
    lib.cc_destroy.argtypes = [P]
    lib.cc_batch_create.restype = c.c_int
    lib.cc_batch_create.argtypes = [c.c_int32, c.POINTER(cc_job_desc), c.POINTER(cc_options), c.POINTER(P)]
    lib.cc_job_count.restype = c.c_int
    lib.cc_job_count.argtypes = [P, c.POINTER(c.c_int32)]
    lib.cc_job_objective.restype = c.c_int
    lib.cc_job_objective.argtypes = [P, c.c_int32, c.POINTER(c.c_int64), c.POINTER(c.c_int32)]
    lib.cc_job_history.restype = c.c_int
    lib.cc_job_history.argtypes = [P, c.c_int32, c.c_int32, c.POINTER(cc_sweep_info), c.POINTER(c.c_int32)]
    lib.cc_job_labels.restype = c.c_int
    lib.cc_job_labels.argtypes = [P, c.c_int32, P]
    lib.cc_batch_run.restype = c.c_int
    lib.cc_batch_run.argtypes = [P, c.c_int32]
    lib.cc_batch_result.restype = c.c_int
    lib.cc_batch_result.argtypes = [P, c.c_int32, P, c.POINTER(c.c_int64)]
    lib.cc_metrics.restype = c.c_int
    lib.cc_metrics.argtypes = [P, c.POINTER(cc_partition_metrics)]
    lib.cc_partition_distances.restype = c.c_int
    lib.cc_partition_distances.argtypes = [P, c.POINTER(cc_partition_metrics)]
    lib.cc_group_partitions.restype = c.c_int
    lib.cc_group_partitions.argtypes = [c.c_int32, P, c.c_int64, P, c.POINTER(c.c_int32)]
    lib.cc_estimate_bytes.restype = c.c_int
    lib.cc_estimate_bytes.argtypes = [c.c_int32, c.POINTER(cc_job_desc), c.POINTER(cc_options),
                                      c.POINTER(c.c_int64), c.POINTER(c.c_int64)]
    lib.cc_plan_batches.restype = c.c_int
    lib.cc_plan_batches.argtypes = [c.c_int32, c.POINTER(cc_job_desc), c.POINTER(cc_options), c.c_int64, c.c_int32,
                                    P, c.POINTER(c.c_int32)]
    lib.cc_server_default_options.restype = None
    lib.cc_server_default_options.argtypes = [c.POINTER(cc_server_options)]
    lib.cc_server_create.restype = c.c_int
    lib.cc_server_create.argtypes = [c.POINTER(cc_server_options), c.POINTER(cc_options), c.POINTER(P)]
    lib.cc_server_submit.restype = c.c_int
    lib.cc_server_submit.argtypes = [P, c.POINTER(cc_job_desc), P, c.POINTER(c.c_int64)]
    lib.cc_server_progress.restype = c.c_int
    lib.cc_server_progress.argtypes = [P, c.c_int32, P, c.c_int32, c.POINTER(c.c_int32), c.POINTER(c.c_int64)]
    lib.cc_server_job.restype = c.c_int
    lib.cc_server_job.argtypes = [P, c.c_int64, c.POINTER(c.c_int32), c.POINTER(c.c_int64), c.POINTER(c.c_int32),
                                  c.POINTER(c.c_int32)]
    lib.cc_server_stats.restype = c.c_int
    lib.cc_server_stats.argtypes = [P, c.POINTER(cc_server_info)]
    lib.cc_server_last_error.restype = c.c_char_p
    lib.cc_server_last_error.argtypes = [P]
    lib.cc_server_destroy.restype = None
    lib.cc_server_destroy.argtypes = [P]
    lib.cc_renumber_noalloc.restype = c.c_int
    lib.cc_renumber_noalloc.argtypes = [c.c_int32, P, P, P]
    lib.cc_noalloc_max_n.restype = c.c_int32
    lib.cc_noalloc_max_n.argtypes = []
    lib.cc_autotune_record.restype = c.c_int
    lib.cc_autotune_record.argtypes = [c.c_int32, P]
    return lib


lib = load_library()

# Largest n accepted by cc_renumber_noalloc, as compiled into the library
# (its built-in scratch holds about 2 n ints).
CC_NOALLOC_MAX_N = int(lib.cc_noalloc_max_n())


def _check(status: int, ctx=None):
    if status != CC_OK:
        msg = lib.cc_last_error(ctx)
        raise CCError(status, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def cc_default_options() -> cc_options:
    o = cc_options()
    lib.cc_default_options(ctypes.byref(o))
    return o


def cc_create(row_off, col, labels, options: cc_options | None = None):
    """Host arrays: row_off int64[n+1], col int32[nnz], labels int32[k, n] -> ctx handle."""
    row_off = np.ascontiguousarray(row_off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    if labels.ndim != 2:
        raise ValueError("labels must be int32[k, n]")
    k, n = labels.shape
    if len(row_off) != n + 1:
        raise ValueError("row_off must have n + 1 entries")
    ctx = ctypes.c_void_p()
    st = lib.cc_create(n, len(col), _ptr(row_off), _ptr(col), k, _ptr(labels),
                       ctypes.byref(options) if options is not None else None, ctypes.byref(ctx))
    _check(st, None)
    return ctx


def cc_create_dev(n: int, nnz: int, row_off_ptr: int, col_ptr: int, k: int, labels_ptr: int,
                  options: cc_options | None = None, stream: int = 0):
    """Device pointers (integers, e.g. torch ``data_ptr()``) -> ctx handle."""
    ctx = ctypes.c_void_p()
    st = lib.cc_create_dev(n, nnz, ctypes.c_void_p(row_off_ptr), ctypes.c_void_p(col_ptr), k,
                           ctypes.c_void_p(labels_ptr), ctypes.byref(options) if options is not None else None,
                           ctypes.c_void_p(stream or None), ctypes.byref(ctx))
    _check(st, None)
    return ctx


def cc_batch_create(jobs, options: cc_options | None = None):
    """jobs: sequence of (row_off int64[n+1], col int32[nnz], labels int32[k, n]) host arrays -> ctx handle."""
    keep = []
    descs = (cc_job_desc * max(len(jobs), 1))()
    for j, (row_off, col, labels) in enumerate(jobs):
        row_off = np.ascontiguousarray(row_off, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        if labels.ndim != 2:
            raise ValueError(f"job {j}: labels must be int32[k, n]")
        k, n = labels.shape
        if len(row_off) != n + 1:
            raise ValueError(f"job {j}: row_off must have n + 1 entries")
        keep += [row_off, col, labels]
        descs[j] = cc_job_desc(n, len(col), _ptr(row_off).value, _ptr(col).value, k, _ptr(labels).value)
    ctx = ctypes.c_void_p()
    st = lib.cc_batch_create(len(jobs), descs, ctypes.byref(options) if options is not None else None,
                             ctypes.byref(ctx))
    _check(st, None)
    return ctx


def cc_job_count(ctx) -> int:
    out = ctypes.c_int32(0)
    _check(lib.cc_job_count(ctx, ctypes.byref(out)), ctx)
    return out.value


def cc_job_objective(ctx, job: int):
    """(F, sweeps recorded) of one job."""
    out = ctypes.c_int64(0)
    sw = ctypes.c_int32(0)
    _check(lib.cc_job_objective(ctx, job, ctypes.byref(out), ctypes.byref(sw)), ctx)
    return out.value, sw.value


def cc_job_history(ctx, job: int) -> list:
    count = ctypes.c_int32(0)
    _check(lib.cc_job_history(ctx, job, 0, None, ctypes.byref(count)), ctx)
    buf = (cc_sweep_info * max(count.value, 1))()
    _check(lib.cc_job_history(ctx, job, count.value, buf, ctypes.byref(count)), ctx)
    return [buf[i].as_dict() for i in range(min(count.value, len(buf)))]


def cc_job_labels(ctx, job: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
    out = np.empty(n, np.int32) if out is None else out
    _check(lib.cc_job_labels(ctx, job, _ptr(out)), ctx)
    return out


def cc_batch_run(ctx, max_sweeps: int = 0):
    _check(lib.cc_batch_run(ctx, max_sweeps), ctx)


def cc_batch_result(ctx, job: int, n: int) -> tuple[np.ndarray, int]:
    """(labels int32[n], objective) of job `job`."""
    out = np.empty(n, np.int32)
    obj = ctypes.c_int64(0)
    _check(lib.cc_batch_result(ctx, job, _ptr(out), ctypes.byref(obj)), ctx)
    return out, int(obj.value)


def cc_set_stream(ctx, stream: int = 0):
    _check(lib.cc_set_stream(ctx, ctypes.c_void_p(stream or None)), ctx)


def cc_reset(ctx):
    _check(lib.cc_reset(ctx), ctx)


def cc_set_cluster_ids(ctx, C):
    C = np.ascontiguousarray(C, dtype=np.int32)
    _check(lib.cc_set_cluster_ids(ctx, _ptr(C)), ctx)


def cc_sweep(ctx, info: bool = True) -> dict | None:
    """One sweep; its record for a single-job context (info=False for a batch)."""
    if not info:
        _check(lib.cc_sweep(ctx, None), ctx)
        return None
    rec = cc_sweep_info()
    _check(lib.cc_sweep(ctx, ctypes.byref(rec)), ctx)
    return rec.as_dict()


def cc_run_until_converged(ctx, max_sweeps: int = 0) -> int:
    done = ctypes.c_int32(0)
    _check(lib.cc_run_until_converged(ctx, max_sweeps, ctypes.byref(done)), ctx)
    return done.value


def cc_last_run_timing(ctx):
    """(sweep_ms float32[s], propose_ms float32[s]) of the last run."""
    count = ctypes.c_int32(0)
    _check(lib.cc_last_run_timing(ctx, 0, None, None, ctypes.byref(count)), ctx)
    a = np.zeros(max(count.value, 1), np.float32)
    b = np.zeros(max(count.value, 1), np.float32)
    _check(lib.cc_last_run_timing(ctx, count.value, _ptr(a), _ptr(b), ctypes.byref(count)), ctx)
    return a[: count.value], b[: count.value]


def cc_table_stats(ctx) -> dict:
    out = cc_table_info()
    _check(lib.cc_table_stats(ctx, ctypes.byref(out)), ctx)
    return out.as_dict()


def cc_launch_count(ctx) -> int:
    out = ctypes.c_int64(0)
    _check(lib.cc_launch_count(ctx, ctypes.byref(out)), ctx)
    return out.value


def cc_history(ctx) -> list:
    count = ctypes.c_int32(0)
    _check(lib.cc_history(ctx, 0, None, ctypes.byref(count)), ctx)
    buf = (cc_sweep_info * max(count.value, 1))()
    _check(lib.cc_history(ctx, count.value, buf, ctypes.byref(count)), ctx)
    return [buf[i].as_dict() for i in range(count.value)]


def cc_objective(ctx) -> int:
    out = ctypes.c_int64(0)
    _check(lib.cc_objective(ctx, ctypes.byref(out)), ctx)
    return out.value


def cc_objective_recompute(ctx) -> int:
    out = ctypes.c_int64(0)
    _check(lib.cc_objective_recompute(ctx, ctypes.byref(out)), ctx)
    return out.value


def cc_consensus_labels(ctx, n: int, out: np.ndarray | None = None) -> np.ndarray:
    out = np.empty(n, np.int32) if out is None else out
    _check(lib.cc_consensus_labels(ctx, _ptr(out)), ctx)
    return out


def cc_cluster_ids(ctx, n: int, out: np.ndarray | None = None) -> np.ndarray:
    out = np.empty(n, np.int32) if out is None else out
    _check(lib.cc_cluster_ids(ctx, _ptr(out)), ctx)
    return out


def cc_cluster_ids_dev(ctx) -> int:
    p = ctypes.c_void_p()
    _check(lib.cc_cluster_ids_dev(ctx, ctypes.byref(p)), ctx)
    return p.value or 0


def cc_last_error(ctx=None) -> str:
    m = lib.cc_last_error(ctx)
    return m.decode() if m else ""


def cc_destroy(ctx):
    lib.cc_destroy(ctx)


def cc_renumber_noalloc(n: int, ids_ptr: int, labels_ptr: int, stream: int = 0):
    """Renumbers n device ids (ids_ptr) into labels_ptr without allocating device memory."""
    _check(lib.cc_renumber_noalloc(n, ctypes.c_void_p(ids_ptr), ctypes.c_void_p(labels_ptr),
                                   ctypes.c_void_p(stream or None)), None)


def _job_desc(row_off, col, labels, keep):
    row_off = np.ascontiguousarray(row_off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    if labels.ndim != 2:
        raise ValueError("labels must be int32[k, n]")
    k, n = labels.shape
    if len(row_off) != n + 1:
        raise ValueError("row_off must have n + 1 entries")
    keep += [row_off, col, labels]
    return cc_job_desc(n, len(col), _ptr(row_off).value, _ptr(col).value, k, _ptr(labels).value)


def cc_metrics(ctx, parts: int) -> dict:
    """Distances of the consensus to every input partition (parts = sum of k over jobs):
    arrays mirkin, split_join (int64), rand_distance, vi (float64), job after job."""
    buf = (cc_partition_metrics * max(parts, 1))()
    _check(lib.cc_metrics(ctx, buf), ctx)
    return {f: np.array([getattr(buf[i], f) for i in range(parts)],
                        dtype=np.float64 if f in ("rand_distance", "vi") else np.int64)
            for f, _ in cc_partition_metrics._fields_}


def cc_partition_distances(ctx, k: int) -> dict:
    """k x k distances between the job's input partitions (fields as cc_metrics)."""
    buf = (cc_partition_metrics * (k * k))()
    _check(lib.cc_partition_distances(ctx, buf), ctx)
    return {f: np.array([getattr(buf[i], f) for i in range(k * k)],
                        dtype=np.float64 if f in ("rand_distance", "vi") else np.int64).reshape(k, k)
            for f, _ in cc_partition_metrics._fields_}


def cc_group_partitions(distance, lam: int):
    """Connected components of the partitions joined by distance <= lam: (group of each, count)."""
    d = np.ascontiguousarray(distance, dtype=np.int64)
    k = d.shape[0]
    out = np.empty(k, np.int32)
    ng = ctypes.c_int32(0)
    _check(lib.cc_group_partitions(k, _ptr(d), int(lam), _ptr(out), ctypes.byref(ng)), None)
    return out, ng.value


def cc_estimate_bytes(sizes, options: cc_options | None = None):
    """sizes: sequence of (n, nnz, k) -> (persistent bytes, peak bytes) of a context for those jobs."""
    descs = (cc_job_desc * max(len(sizes), 1))()
    for j, (n, nnz, k) in enumerate(sizes):
        descs[j] = cc_job_desc(n, nnz, None, None, k, None)
    a = ctypes.c_int64(0)
    b = ctypes.c_int64(0)
    _check(lib.cc_estimate_bytes(len(sizes), descs, ctypes.byref(options) if options is not None else None,
                                 ctypes.byref(a), ctypes.byref(b)), None)
    return a.value, b.value


def cc_plan_batches(sizes, budget_bytes: int, max_jobs: int = 0, options: cc_options | None = None):
    """sizes: sequence of (n, nnz, k) -> (batch index of every job (-1: over the budget), number of batches)."""
    descs = (cc_job_desc * max(len(sizes), 1))()
    for j, (n, nnz, k) in enumerate(sizes):
        descs[j] = cc_job_desc(n, nnz, None, None, k, None)
    out = np.empty(max(len(sizes), 1), np.int32)
    nb = ctypes.c_int32(0)
    _check(lib.cc_plan_batches(len(sizes), descs, ctypes.byref(options) if options is not None else None,
                               budget_bytes, max_jobs, _ptr(out), ctypes.byref(nb)), None)
    return out[: len(sizes)], nb.value


def _check_server(status: int, srv=None):
    if status != CC_OK:
        msg = lib.cc_server_last_error(srv)
        raise CCError(status, msg.decode() if msg else "")


def cc_server_default_options() -> cc_server_options:
    o = cc_server_options()
    lib.cc_server_default_options(ctypes.byref(o))
    return o


def cc_server_create(server_options: cc_server_options | None = None, options: cc_options | None = None):
    srv = ctypes.c_void_p()
    st = lib.cc_server_create(ctypes.byref(server_options) if server_options is not None else None,
                              ctypes.byref(options) if options is not None else None, ctypes.byref(srv))
    _check_server(st, None)
    return srv


def cc_server_submit(srv, desc: cc_job_desc, out: np.ndarray) -> int:
    """desc: a cc_job_desc whose arrays the caller keeps alive until the job is done; out: int32[n]."""
    t = ctypes.c_int64(0)
    _check_server(lib.cc_server_submit(srv, ctypes.byref(desc), _ptr(out), ctypes.byref(t)), srv)
    return t.value


def cc_server_progress(srv, wait: bool = False, max_done: int = 4096):
    """-> (tickets done since the last report, jobs pending)."""
    buf = np.empty(max_done, np.int64)
    nd = ctypes.c_int32(0)
    pend = ctypes.c_int64(0)
    _check_server(lib.cc_server_progress(srv, 1 if wait else 0, _ptr(buf), max_done, ctypes.byref(nd),
                                         ctypes.byref(pend)), srv)
    return buf[: nd.value].tolist(), pend.value


def cc_server_job(srv, ticket: int) -> dict:
    done = ctypes.c_int32(0)
    F = ctypes.c_int64(0)
    sw = ctypes.c_int32(0)
    st = ctypes.c_int32(0)
    _check_server(lib.cc_server_job(srv, ticket, ctypes.byref(done), ctypes.byref(F), ctypes.byref(sw),
                                    ctypes.byref(st)), srv)
    return {"done": bool(done.value), "F": F.value, "sweeps": sw.value, "status": st.value}


def cc_server_stats(srv) -> dict:
    out = cc_server_info()
    _check_server(lib.cc_server_stats(srv, ctypes.byref(out)), srv)
    return out.as_dict()


def cc_server_destroy(srv):
    lib.cc_server_destroy(srv)
