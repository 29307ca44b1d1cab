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


def test_default_options(native):
    o = native.cc_default_options()
    assert o.max_sweeps == 20 and o.debug_checks == 0 and o.table_log2 == 0 and o.table_start_log2 == 0
    assert o.sweep_mode == 0 and list(o.reserved) == [0] * 3


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
    opt.reserved[2] = 7
    assert _create_status(native, 5, 0, ok, None, 1, ok, ctypes.byref(opt))[0] == 1
    opt = native.cc_default_options()
    opt.sweep_mode = 3
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
