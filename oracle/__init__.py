"""CPU oracle for the consensus-clustering sweep -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never calls it.

The arithmetic lives in ``oracle.c`` (plain C, integers only); this module
loads it with ctypes, compiling it with gcc on first use if the shared object
is missing.  Every function follows the definitions in the paper's Methods
section and Appendix; the header of ``oracle.c`` states each one and the
readings taken where the paper leaves a choice open.

Functions with a pin in ``tests/test_oracle_*.py``:

* ``objective``      F(C) = sum_i Mirkin(C, P_i), ordered pairs      (Eq. objective1)
* ``mirkin_pairs``   Mirkin distance by pair enumeration              (Appendix Eq. distance)
* ``gain_member`` / ``gain_closed``  dD(v: a -> b) two ways           (Eq. objective3)
* ``sync_propose``   best move of every vertex against one state      (Eq. objective4)
* ``sync_step`` / ``sync_run``  synchronous sweeps with the singleton and
                     exact-objective guards and the matching fallback (Parallel algorithm)
* ``match``          the locally dominant matching used by the fallback
* ``colour`` / ``colour_run``  colour-batched greedy: the synchronous rule applied
                     one colour class of a greedy colouring at a time (a variant)
* ``seq_run``        sequential greedy, one move at a time            (The algorithm)
* ``brute_force``    exact optimum over all set partitions, n <= 12
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


class SweepStats(ctypes.Structure):
    _fields_ = [("proposals", ctypes.c_int64), ("p1", ctypes.c_int64), ("dF_p1", ctypes.c_int64),
                ("fallback", ctypes.c_int64), ("moves", ctypes.c_int64), ("F", ctypes.c_int64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    c = ctypes
    lib.orc_objective.restype = c.c_int64
    lib.orc_objective.argtypes = [c.c_int32, c.c_int32, i32p, i32p]
    lib.orc_partition_sq.restype = c.c_int64
    lib.orc_partition_sq.argtypes = [c.c_int32, c.c_int32, i32p]
    lib.orc_mirkin_pairs.restype = c.c_int64
    lib.orc_mirkin_pairs.argtypes = [c.c_int32, i32p, i32p]
    for f in (lib.orc_gain_member, lib.orc_gain_closed):
        f.restype = c.c_int64
        f.argtypes = [c.c_int32, c.c_int32, i32p, i32p, c.c_int32, c.c_int32]
    lib.orc_sync_propose.restype = c.c_int64
    lib.orc_sync_propose.argtypes = [c.c_int32, i64p, i32p, c.c_int32, i32p, i32p, i32p, i64p,
                                     c.c_int32, c.c_int32]
    lib.orc_sync_propose_range.restype = c.c_int64
    lib.orc_sync_propose_range.argtypes = [c.c_int32, i64p, i32p, c.c_int32, i32p, i32p, c.c_int32, c.c_int32,
                                           i32p, i64p, c.c_int32, c.c_int32]
    lib.orc_sync_step.restype = c.c_int32
    lib.orc_sync_step.argtypes = [c.c_int32, i64p, i32p, c.c_int32, i32p, i32p, c.c_int64, c.c_int32,
                                  c.POINTER(SweepStats), i32p, i64p, i32p]
    lib.orc_sync_run.restype = c.c_int32
    lib.orc_sync_run.argtypes = [c.c_int32, i64p, i32p, c.c_int32, i32p, i32p, c.c_int32, c.c_int32,
                                 c.c_int32, c.POINTER(SweepStats), c.POINTER(c.c_int32)]
    lib.orc_priority.restype = c.c_uint64
    lib.orc_priority.argtypes = [c.c_uint64]
    lib.orc_colour.restype = c.c_int32
    lib.orc_colour.argtypes = [c.c_int32, i64p, i32p, i32p]
    lib.orc_colour_run.restype = c.c_int32
    lib.orc_colour_run.argtypes = [c.c_int32, i64p, i32p, c.c_int32, i32p, i32p, i32p, c.c_int32, c.c_int32,
                                   c.c_int32, c.c_int32, c.POINTER(SweepStats), c.POINTER(c.c_int32)]
    lib.orc_seq_run.restype = c.c_int32
    lib.orc_seq_run.argtypes = [c.c_int32, i64p, i32p, c.c_int32, i32p, i32p, c.c_int32, i64p, i64p,
                                c.POINTER(c.c_int32)]
    lib.orc_match.restype = c.c_int64
    lib.orc_match.argtypes = [c.c_int32, i32p, i32p, i64p, i32p]
    lib.orc_brute_force.restype = c.c_int64
    lib.orc_brute_force.argtypes = [c.c_int32, c.c_int32, i32p, i32p]
    f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
    lib.orc_metrics.restype = c.c_int32
    lib.orc_metrics.argtypes = [c.c_int32, c.c_int32, i32p, i32p, i64p, i64p, f64p]
    _lib = lib
    return lib


def _labels(labels):
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    if lab.ndim != 2:
        raise ValueError("labels must be int32[k, n]")
    return lab


def singletons(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.int32)


def objective(labels, C) -> int:
    lab = _labels(labels)
    k, n = lab.shape
    r = _load().orc_objective(n, k, lab, np.ascontiguousarray(C, dtype=np.int32))
    if r < 0:
        raise ValueError("invalid consensus (ids must lie in [0, n))")
    return int(r)


def partition_sq(labels) -> int:
    lab = _labels(labels)
    k, n = lab.shape
    return int(_load().orc_partition_sq(n, k, lab))


def metrics(labels, C) -> dict:
    """Distances between C and each input partition (Methods, Evaluation
    metrics): Mirkin over ordered pairs, Rand distance (Mirkin / n(n-1)),
    van Dongen's split-join distance, Meila's variation of information (nats)."""
    lab = _labels(labels)
    k, n = lab.shape
    C = np.ascontiguousarray(C, dtype=np.int32)
    mir = np.zeros(k, np.int64)
    sj = np.zeros(k, np.int64)
    vi = np.zeros(k, np.float64)
    rc = _load().orc_metrics(n, k, lab, C, mir, sj, vi)
    if rc != 0:
        raise RuntimeError(f"oracle metrics failed ({rc})")
    pairs = n * (n - 1)
    rand = mir / pairs if pairs else np.zeros(k)
    return {"mirkin": mir, "rand_distance": rand, "split_join": sj, "vi": vi}


def mirkin_pairs(X, Y) -> int:
    X = np.ascontiguousarray(X, dtype=np.int32)
    Y = np.ascontiguousarray(Y, dtype=np.int32)
    return int(_load().orc_mirkin_pairs(len(X), X, Y))


def gain_member(labels, C, v: int, b: int) -> int:
    lab = _labels(labels)
    k, n = lab.shape
    return int(_load().orc_gain_member(n, k, lab, np.ascontiguousarray(C, dtype=np.int32), v, b))


def gain_closed(labels, C, v: int, b: int) -> int:
    lab = _labels(labels)
    k, n = lab.shape
    return int(_load().orc_gain_closed(n, k, lab, np.ascontiguousarray(C, dtype=np.int32), v, b))


# mode: 0 gains from the contingency counts, 1 by member iteration (the same
# values); empty=True adds the move-to-empty candidate (mode bit 2)
EMPTY = 2


def sync_propose(row_off, col, labels, C, mode: int = 0, threads: int = 0, empty: bool = False):
    """(target int32[n], gain int64[n], count): each vertex's proposal against C."""
    mode = mode | (EMPTY if empty else 0)
    lab = _labels(labels)
    k, n = lab.shape
    target = np.empty(n, np.int32)
    gain = np.empty(n, np.int64)
    cnt = _load().orc_sync_propose(n, np.ascontiguousarray(row_off, dtype=np.int64),
                                   np.ascontiguousarray(col, dtype=np.int32), k, lab,
                                   np.ascontiguousarray(C, dtype=np.int32), target, gain, mode, threads)
    if cnt < 0:
        raise RuntimeError("oracle proposal pass failed")
    return target, gain, int(cnt)


def sync_propose_range(row_off, col, labels, C, v0: int, v1: int, mode: int = 0, threads: int = 0,
                       empty: bool = False):
    """As sync_propose, for the vertices in [v0, v1) only (the rest propose nothing)."""
    mode = mode | (EMPTY if empty else 0)
    lab = _labels(labels)
    k, n = lab.shape
    target = np.empty(n, np.int32)
    gain = np.empty(n, np.int64)
    cnt = _load().orc_sync_propose_range(n, np.ascontiguousarray(row_off, dtype=np.int64),
                                         np.ascontiguousarray(col, dtype=np.int32), k, lab,
                                         np.ascontiguousarray(C, dtype=np.int32), v0, v1, target, gain, mode,
                                         threads)
    if cnt < 0:
        raise RuntimeError("oracle proposal pass failed")
    return target, gain, int(cnt)


@dataclass
class StepResult:
    C: np.ndarray
    stats: dict
    target: np.ndarray
    gain: np.ndarray
    moved: np.ndarray


def sync_step(row_off, col, labels, C, F=None, mode: int = 0, empty: bool = False) -> StepResult:
    """One synchronous sweep from state C (not modified); returns the new state."""
    mode = mode | (EMPTY if empty else 0)
    lab = _labels(labels)
    k, n = lab.shape
    C1 = np.array(C, dtype=np.int32, copy=True)
    F = objective(lab, C1) if F is None else F
    st = SweepStats()
    target = np.empty(n, np.int32)
    gain = np.empty(n, np.int64)
    moved = np.empty(n, np.int32)
    rc = _load().orc_sync_step(n, np.ascontiguousarray(row_off, dtype=np.int64),
                               np.ascontiguousarray(col, dtype=np.int32), k, lab, C1, int(F), mode,
                               ctypes.byref(st), target, gain, moved)
    if rc != 0:
        raise RuntimeError(f"oracle sweep failed ({rc})")
    return StepResult(C1, st.as_dict(), target, gain, moved.astype(bool))


@dataclass
class RunResult:
    C: np.ndarray
    stats: list
    sweeps: int
    F0: int

    @property
    def F(self):
        return self.stats[-1]["F"] if self.stats else self.F0


def sync_run(row_off, col, labels, max_sweeps: int = 20, C0=None, mode: int = 0, threads: int = 0,
             empty: bool = False):
    """Synchronous sweeps from C0 (default: singletons) until no proposal or max_sweeps."""
    mode = mode | (EMPTY if empty else 0)
    lab = _labels(labels)
    k, n = lab.shape
    C = singletons(n) if C0 is None else np.array(C0, dtype=np.int32, copy=True)
    F0 = objective(lab, C)
    stats = (SweepStats * max(max_sweeps, 1))()
    done = ctypes.c_int32(0)
    rc = _load().orc_sync_run(n, np.ascontiguousarray(row_off, dtype=np.int64),
                              np.ascontiguousarray(col, dtype=np.int32), k, lab, C, max_sweeps, mode,
                              threads, stats, ctypes.byref(done))
    if rc != 0:
        raise RuntimeError(f"oracle run failed ({rc})")
    return RunResult(C, [stats[s].as_dict() for s in range(done.value)], done.value, F0)


def priority(v: int) -> int:
    """Colouring priority of vertex v: the first splitmix64 output seeded with v."""
    return int(_load().orc_priority(v))


def colour(row_off, col):
    """(colour int32[n], number of colours): greedy colouring in decreasing priority."""
    n = len(row_off) - 1
    out = np.empty(n, np.int32)
    cnt = _load().orc_colour(n, np.ascontiguousarray(row_off, dtype=np.int64),
                             np.ascontiguousarray(col, dtype=np.int32), out)
    if cnt < 0:
        raise RuntimeError("oracle colouring failed")
    return out, int(cnt)


def colour_run(row_off, col, labels, max_sweeps: int = 20, C0=None, mode: int = 0, threads: int = 0,
               empty: bool = False):
    """Colour-batched greedy sweeps from C0 (default: singletons) until no proposal or max_sweeps."""
    mode = mode | (EMPTY if empty else 0)
    lab = _labels(labels)
    k, n = lab.shape
    C = singletons(n) if C0 is None else np.array(C0, dtype=np.int32, copy=True)
    F0 = objective(lab, C)
    cls, ncol = colour(row_off, col)
    stats = (SweepStats * max(max_sweeps, 1))()
    done = ctypes.c_int32(0)
    rc = _load().orc_colour_run(n, np.ascontiguousarray(row_off, dtype=np.int64),
                                np.ascontiguousarray(col, dtype=np.int32), k, lab, C, cls, ncol, max_sweeps,
                                mode, threads, stats, ctypes.byref(done))
    if rc != 0:
        raise RuntimeError(f"oracle colour-batched run failed ({rc})")
    return RunResult(C, [stats[s].as_dict() for s in range(done.value)], done.value, F0)


def seq_run(row_off, col, labels, max_sweeps: int = 20, C0=None):
    """Sequential greedy; returns (C, F_trace, moves_trace)."""
    lab = _labels(labels)
    k, n = lab.shape
    C = singletons(n) if C0 is None else np.array(C0, dtype=np.int32, copy=True)
    Ft = np.zeros(max(max_sweeps, 1), np.int64)
    Mt = np.zeros(max(max_sweeps, 1), np.int64)
    done = ctypes.c_int32(0)
    rc = _load().orc_seq_run(n, np.ascontiguousarray(row_off, dtype=np.int64),
                             np.ascontiguousarray(col, dtype=np.int32), k, lab, C, max_sweeps, Ft, Mt,
                             ctypes.byref(done))
    if rc != 0:
        raise RuntimeError(f"oracle sequential run failed ({rc})")
    return C, Ft[: done.value].copy(), Mt[: done.value].copy()


def match(C, target, gain):
    """Locally dominant matching of a proposal set: bool[n], True for kept moves."""
    C = np.ascontiguousarray(C, dtype=np.int32)
    n = len(C)
    moved = np.empty(n, np.int32)
    r = _load().orc_match(n, C, np.ascontiguousarray(target, dtype=np.int32),
                          np.ascontiguousarray(gain, dtype=np.int64), moved)
    if r < 0:
        raise MemoryError("oracle matching")
    return moved.astype(bool)


def brute_force(labels):
    """(F*, C*) over all set partitions; n <= 12."""
    lab = _labels(labels)
    k, n = lab.shape
    best = np.zeros(n, np.int32)
    F = _load().orc_brute_force(n, k, lab, best)
    if F < 0:
        raise ValueError("brute force needs 1 <= n <= 12")
    return int(F), best


def renumber(C) -> np.ndarray:
    """Cluster ids renumbered 0..b-1 in order of first appearance by vertex index."""
    C = np.asarray(C)
    out = np.empty(len(C), np.int32)
    seen = {}
    for v, c in enumerate(C.tolist()):
        if c not in seen:
            seen[c] = len(seen)
        out[v] = seen[c]
    return out
