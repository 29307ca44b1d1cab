"""The C ABI without a GPU: the library loads, exports every function that
include/cc.h declares, and rejects malformed arguments on the host before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(cc_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def native():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2408_11331_gb300 import _native

    return _native


def test_exports_every_declared_symbol(native):
    declared = _declared()
    assert declared, "no declarations found"
    missing = [s for s in sorted(declared) if not hasattr(native.lib, s)]
    assert not missing, missing
    assert set(native.EXPORTS) == declared


def test_noalloc_limit_matches_header(native):
    """The no-allocation renumbering's size limit, as the library reports it,
    is the one include/cc.h states (bindings read it from the library)."""
    text = open(os.path.join(ROOT, "include", "cc.h")).read()
    m = re.search(r"#define\s+CC_NOALLOC_MAX_N\s+\(1\s*<<\s*(\d+)\)", text)
    assert m, "CC_NOALLOC_MAX_N not found in cc.h"
    assert native.lib.cc_noalloc_max_n() == 1 << int(m.group(1)) == native.CC_NOALLOC_MAX_N


def test_default_options(native):
    o = native.cc_default_options()
    assert o.max_sweeps == 20 and o.debug_checks == 0 and o.table_log2 == 0 and o.table_start_log2 == 0
    assert o.sweep_mode == 0 and o.lanes == 0 and o.active_set == 0 and o.no_regions == 0
    assert o.empty_moves == 0 and o.colour_batched == 0 and o.autotune == 0 and o.tight_rebuild == 0


def _create_status(native, n, nnz, row_off, col, k, labels, opt=None):
    ctx = ctypes.c_void_p()
    st = native.lib.cc_create(n, nnz, row_off, col, k, labels, opt, ctypes.byref(ctx))
    assert not ctx.value
    return st, native.cc_last_error()


def test_host_validation(native):
    P = ctypes.c_void_p
    ok = P(1)
    assert _create_status(native, 0, 0, ok, None, 1, ok)[0] == 1
    assert _create_status(native, 5, 0, ok, None, 0, ok)[0] == 1
    assert _create_status(native, 5, -1, ok, None, 1, ok)[0] == 1
    assert _create_status(native, 5, 0, None, None, 1, ok)[0] == 1
    assert _create_status(native, 5, 0, ok, None, 1, None)[0] == 1
    assert _create_status(native, 5, 3, ok, None, 1, ok)[0] == 1       # nnz > 0 needs col
    assert _create_status(native, 5, 0, ok, None, 5000, ok)[0] == 1    # k above the limit
    st, msg = _create_status(native, 300_000_000, 0, ok, None, 3, ok)  # 3 k n + k >= 2^31
    assert st == 4 and "2^31" in msg
    opt = native.cc_default_options()
    opt.no_regions = 7
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.sweep_mode = 3
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.active_set = 2
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.autotune = 3
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.tight_rebuild = 3
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.colour_batched = 2
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.colour_batched = 1
    opt.active_set = 1
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.empty_moves = 2
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.lanes = 3
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt.lanes = 64
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.table_log2 = 99
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1


def test_null_context_calls(native):
    lib = native.lib
    assert lib.cc_sweep(None, None) == 1
    assert lib.cc_reset(None) == 1
    assert lib.cc_run_until_converged(None, 3, None) == 1
    out = ctypes.c_int64()
    assert lib.cc_objective(None, ctypes.byref(out)) == 1
    lib.cc_destroy(None)


def test_python_binding_checks_shapes(native):
    with pytest.raises(ValueError):
        native.cc_create(np.zeros(3, np.int64), np.zeros(0, np.int32), np.zeros(4, np.int32))
    with pytest.raises(ValueError):
        native.cc_create(np.zeros(3, np.int64), np.zeros(0, np.int32), np.zeros((1, 4), np.int32))


def test_batch_host_validation(native):
    """cc_batch_create checks every job on the host before any device work."""
    lib = native.lib
    ctx = ctypes.c_void_p(123)
    assert lib.cc_batch_create(0, None, None, ctypes.byref(ctx)) == 1
    assert ctx.value is None
    ok = 1
    good = native.cc_job_desc(5, 0, ok, None, 2, ok)
    descs = (native.cc_job_desc * 3)(good, good, native.cc_job_desc(0, 0, ok, None, 2, ok))
    assert lib.cc_batch_create(3, descs, None, ctypes.byref(ctx)) == 1
    assert "job 2" in native.cc_last_error(None)
    descs = (native.cc_job_desc * 2)(good, native.cc_job_desc(5, 0, ok, None, 4097, ok))
    assert lib.cc_batch_create(2, descs, None, ctypes.byref(ctx)) == 1
    assert "job 1" in native.cc_last_error(None)
    descs = (native.cc_job_desc * 2)(native.cc_job_desc(300_000_000, 0, ok, None, 3, ok), good)
    assert lib.cc_batch_create(2, descs, None, ctypes.byref(ctx)) == 4
    # a job count the union cannot index: 2^31 vertices in all
    big = native.cc_job_desc(100_000_000, 0, ok, None, 1, ok)
    descs = (native.cc_job_desc * 22)(*([big] * 22))
    assert lib.cc_batch_create(22, descs, None, ctypes.byref(ctx)) == 4
    opt = native.cc_default_options()
    opt.sweep_mode = 7
    descs = (native.cc_job_desc * 1)(good)
    assert lib.cc_batch_create(1, descs, ctypes.byref(opt), ctypes.byref(ctx)) == 1


def test_batch_null_context_calls(native):
    lib = native.lib
    out = ctypes.c_int64()
    n = ctypes.c_int32()
    assert lib.cc_job_count(None, ctypes.byref(n)) == 1
    assert lib.cc_job_objective(None, 0, ctypes.byref(out), None) == 1
    assert lib.cc_job_history(None, 0, 0, None, ctypes.byref(n)) == 1
    assert lib.cc_job_labels(None, 0, None) == 1
    assert lib.cc_batch_run(None, 0) == 1
    assert lib.cc_batch_result(None, 0, None, ctypes.byref(out)) == 1


def test_python_batch_binding_checks_shapes(native):
    with pytest.raises(ValueError):
        native.cc_batch_create([(np.zeros(3, np.int64), np.zeros(0, np.int32), np.zeros(4, np.int32))])
    with pytest.raises(ValueError):
        native.cc_batch_create([(np.zeros(3, np.int64), np.zeros(0, np.int32), np.zeros((1, 4), np.int32))])


def test_estimate_bytes_host(native):
    """The footprint estimate is host arithmetic: it grows with every size,
    counts the creation temporaries on top, and sizes the contingency hash
    at 2 k n slots (4 k n when every sweep is staged) rounded up to a power
    of two, 16 bytes a slot."""
    p1, k1 = native.cc_estimate_bytes([(1000, 20000, 10)])
    assert k1 > p1 > 0
    assert native.cc_estimate_bytes([(2000, 20000, 10)])[0] > p1
    assert native.cc_estimate_bytes([(1000, 40000, 10)])[0] > p1
    assert native.cc_estimate_bytes([(1000, 20000, 20)])[0] > p1
    # a batch does not depend on the order of its jobs and holds more than its largest job
    a = native.cc_estimate_bytes([(1000, 20000, 10), (3000, 50000, 7)])[0]
    assert a == native.cc_estimate_bytes([(3000, 50000, 7), (1000, 20000, 10)])[0]
    assert a > native.cc_estimate_bytes([(3000, 50000, 7), (3000, 0, 1)])[0] - native.cc_estimate_bytes([(3000, 0, 1)])[0]
    # staged-only sweeps double the hash: 2kn + 64 = 20064 -> 32768 slots, 4kn + 64 -> 65536
    o = native.cc_default_options()
    o.sweep_mode = 1
    s1 = native.cc_estimate_bytes([(1000, 20000, 10)], o)[0]
    assert s1 - p1 == 16 * (65536 - 32768)
    with pytest.raises(native.CCError):
        native.cc_estimate_bytes([(0, 0, 3)])


def test_server_host_validation(native):
    lib = native.lib
    srv = ctypes.c_void_p(7)
    so = native.cc_server_default_options()
    assert so.max_active == 8 and so.max_batch_jobs == 256 and so.budget_bytes == 0
    so.reserved[1] = 3
    assert lib.cc_server_create(ctypes.byref(so), None, ctypes.byref(srv)) == 1
    assert srv.value is None
    so = native.cc_server_default_options()
    so.max_active = 65
    assert lib.cc_server_create(ctypes.byref(so), None, ctypes.byref(srv)) == 1
    so = native.cc_server_default_options()
    so.budget_bytes = -1
    assert lib.cc_server_create(ctypes.byref(so), None, ctypes.byref(srv)) == 1
    o = native.cc_default_options()
    o.sweep_mode = 5
    assert lib.cc_server_create(None, ctypes.byref(o), ctypes.byref(srv)) == 1
    assert lib.cc_server_submit(None, None, None, None) == 1
    assert lib.cc_server_progress(None, 0, None, 0, None, None) == 1
    lib.cc_server_destroy(None)


def test_plan_batches_host(native):
    """Batches hold one lane bin each, keep job order within a bin, fit the
    budget, respect the job cap, and mark jobs over the budget with -1."""
    sizes = [(1000, 20000, 10), (500, 8000, 3), (2000, 40000, 9), (800, 9000, 60), (700, 7000, 4),
             (3000, 60000, 8), (900, 9000, 50), (100000, 2000000, 30)]
    one = [native.cc_estimate_bytes([s])[1] for s in sizes]
    budget = 3 * max(one[:7])
    batch, nb = native.cc_plan_batches(sizes, budget)
    assert batch[7] == -1  # the big job alone exceeds the budget
    bins = {}
    for j, b in enumerate(batch[:7]):
        bins.setdefault(int(b), []).append(j)
    assert len(bins) == nb
    lanes = lambda k: next(g for g in (1, 2, 4, 8, 16, 32) if g * 10 >= k or g == 32)  # noqa: E731
    for b, members in bins.items():
        assert len({lanes(sizes[j][2]) for j in members}) == 1
        assert native.cc_estimate_bytes([sizes[j] for j in members])[1] <= budget
    # bins in increasing order of lanes: k <= 10 first
    assert batch[1] == batch[4] == 0
    capped, nb2 = native.cc_plan_batches(sizes[:7], 1 << 40, max_jobs=1)
    assert nb2 == 7 and sorted(capped.tolist()) == list(range(7))
    whole, nb3 = native.cc_plan_batches(sizes[:7], 1 << 40)
    assert nb3 == 2  # bins of k: {10, 3, 9, 4, 8}, {60, 50}
    with pytest.raises(native.CCError):
        native.cc_plan_batches([(0, 0, 1)], 1 << 30)


def test_group_partitions_host(native):
    """Components of the threshold graph over partitions (host only)."""
    d = np.array([[0, 2, 9, 9, 9],
                  [2, 0, 9, 3, 9],
                  [9, 9, 0, 9, 9],
                  [9, 3, 9, 0, 1],
                  [9, 9, 9, 1, 0]], np.int64)
    g, n = native.cc_group_partitions(d, 3)
    assert n == 2 and g.tolist() == [0, 0, 1, 0, 0]
    g, n = native.cc_group_partitions(d, 2)
    assert n == 3 and g.tolist() == [0, 0, 1, 2, 2]
    g, n = native.cc_group_partitions(d, 0)
    assert n == 5 and g.tolist() == [0, 1, 2, 3, 4]
    g, n = native.cc_group_partitions(d, 100)
    assert n == 1 and g.tolist() == [0] * 5
    rng = np.random.default_rng(3)
    for _ in range(20):
        k = int(rng.integers(1, 12))
        m = rng.integers(0, 20, (k, k))
        m = np.minimum(m, m.T)
        np.fill_diagonal(m, 0)
        lam = int(rng.integers(0, 20))
        g, n = native.cc_group_partitions(m, lam)
        # same group iff joined by a path of edges <= lam (closure by repeated squaring)
        adj = (m <= lam).astype(np.int64)
        reach = adj.copy()
        for _ in range(k):
            reach = np.minimum(1, reach + reach @ adj)
        assert ((g[:, None] == g[None, :]) == (reach > 0)).all()
        assert n == len(set(g.tolist()))
    with pytest.raises(native.CCError):
        native.cc_group_partitions(np.zeros((0, 0), np.int64), 1)
