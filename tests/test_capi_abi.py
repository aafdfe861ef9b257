"""The C ABI library: it loads without a GPU, exports every function that
include/lopc.h declares, and its host-only entry points agree with the oracle."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lopc.h")


@pytest.fixture(scope="module")
def L():
    from paper_2603_26968_b300 import build, lopc
    build.build()
    return lopc


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lopc_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "lopc_compress" in names and "lopc_decompress" in names and len(names) >= 10
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", str(L.LIB_PATH)], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s(lopc_\w+)$", out, flags=re.M))
    assert set(names) <= exported
    assert all(e in names for e in exported), exported - set(names)


def test_strerror_and_invalid_args(L):
    lib = L.lib()
    assert lib.lopc_strerror(0) == b"ok"
    assert lib.lopc_strerror(-5) == b"corrupt stream"
    bad = L.make_desc((4, 4), "f32", L.NOA, 1e-3)
    bad.ndim = 4
    assert lib.lopc_compress_bound(C.byref(bad)) == 0
    assert lib.lopc_compress_workspace_size(C.byref(bad)) == 0
    size = C.c_size_t()
    rc = lib.lopc_compress(C.byref(bad), None, None, 0, C.byref(size), None, 0, None)
    assert rc == -1
    good = L.make_desc((4, 4), "f32", L.NOA, 1e-3)
    good.eb = 0.0
    assert lib.lopc_compress(C.byref(good), None, None, 0, C.byref(size), None, 0, None) == -1
    assert lib.lopc_peek(None, 0, C.byref(good)) == -1


def test_bounds_cover_the_oracle_streams(L, orc):
    rng = np.random.default_rng(0)
    for shape, dt in [((70, 90), np.float32), ((9, 17, 33), np.float64), ((1, 300), np.float32)]:
        x = np.cumsum(rng.standard_normal(shape), axis=-1).astype(dt)
        st = orc.compress(x, 1, 1e-4)
        d = L.make_desc(shape, x.dtype == np.float32 and "f32" or "f64", L.NOA, 1e-4)
        assert L.compress_bound(d) >= len(st)
        assert L.compress_workspace_size(d) > 0 and L.decompress_workspace_size(d) > 0


def test_peek_reads_oracle_headers(L, orc):
    x = np.linspace(-1, 1, 5 * 6 * 7).reshape(5, 6, 7)
    st = orc.compress(x, 0, 1e-3)
    d = L.peek(st)
    assert (d.dtype, d.ndim, d.shape, d.mode, d.eb) == (1, 3, (5, 6, 7), 0, 1e-3)
    with pytest.raises(L.LopcError):
        L.peek(b"XXXX" + st[4:128])


def test_verify_host_checks(L):
    lib = L.lib()
    # the report's layout: 15 int64 counts, 6 doubles, two int32
    assert C.sizeof(L.VerifyReport) == 15 * 8 + 6 * 8 + 8
    bad = L.make_desc((4, 4), "f32", L.NOA, 1e-3)
    bad.ndim = 4
    assert lib.lopc_verify_workspace_size(C.byref(bad)) == 0
    r = L.VerifyReport()
    assert lib.lopc_verify(C.byref(bad), None, None, None, None, C.byref(r), None, 0, None) == -1
    good = L.make_desc((300, 200, 100), "f64", L.ABS, 0.5)
    ws = lib.lopc_verify_workspace_size(C.byref(good))
    assert ws >= (1 << 14) and ws % 256 == 0
    assert lib.lopc_verify(C.byref(good), None, None, None, None, C.byref(r), None, 0, None) == -1


def test_repair_mode_knob(L):
    lib = L.lib()
    assert lib.lopc_set_repair_mode(7) == -1
    prev = lib.lopc_set_repair_mode(L.REPAIR_WORKLIST)
    assert prev == L.REPAIR_TILES
    d = L.make_desc((30, 40, 50), "f32", L.NOA, 1e-3)
    wl = lib.lopc_compress_workspace_size(C.byref(d))
    assert lib.lopc_set_repair_mode(L.REPAIR_TILES) == L.REPAIR_WORKLIST
    tiles = lib.lopc_compress_workspace_size(C.byref(d))
    assert wl >= tiles + 12 * 30 * 40 * 50
    # batches always use tiles
    assert lib.lopc_batch_compress_workspace_size(1, C.byref(d)) == tiles


def test_tuning_knobs_clamp_and_read_back(L):
    saved = (L.tune_get(), L.tune_get_budget(), L.tune_get_dense(), L.tune_get_pass_order())
    try:
        assert saved[3] == (L.PASS_ORDER_AUTO,) * 4  # the default: each field decides
        L.tune_set_pass_order([-3, 1, 2, 9])
        assert L.tune_get_pass_order() == (0, 1, 2, 2)
        L.tune_set([0, 3, 17, 5])
        assert L.tune_get() == (1, 3, 16, 5)
        L.tune_set_budget([0, 64, 5000, 7])
        assert L.tune_get_budget() == (1, 64, 4096, 7)
        L.tune_set_dense([-1, 8, 18, 17])
        assert L.tune_get_dense() == (0, 8, 17, 17)
    finally:
        L.tune_set(saved[0])
        L.tune_set_budget(saved[1])
        L.tune_set_dense(saved[2])
        L.tune_set_pass_order(saved[3])


def test_batch_field_limit(L):
    """A compression batch holds at most LOPC_MAX_BATCH_FIELDS fields: the limit is
    checked on the host, before any launch."""
    lib = L.lib()
    d = L.make_desc((8, 8), "f32", L.NOA, 1e-3)
    for n, ok in ((65535, True), (65536, False)):
        descs = (type(d) * n)(*([d] * n))
        assert (lib.lopc_batch_compress_workspace_size(n, descs) > 0) == ok
    n = 65536
    descs = (type(d) * n)(*([d] * n))
    ptrs = (C.c_void_p * n)(*([1] * n))
    caps = (C.c_size_t * n)(*([4096] * n))
    plan = L.plan_default()
    for pl in (None, C.byref(plan)):
        rc = lib.lopc_batch_compress(n, descs, ptrs, ptrs, caps, C.c_void_p(1), C.c_void_p(1), pl, C.c_void_p(1),
                                     1 << 40, None)
        assert rc == -1


def test_plan_default_and_current(L):
    """lopc_plan: the defaults, and the thread's current plan following lopc_tune_*."""
    d = L.plan_default().as_dict()
    assert d == {"rerun_blocks_per_sm": [4, 4, 6, 6], "pass_budget16": [64] * 4, "pass_dense16": [8] * 4,
                 "pass_order": [0] * 4}
    saved = L.tune_get()
    try:
        L.tune_set([2, 5, 7, 9])
        assert L.plan_get().as_dict()["rerun_blocks_per_sm"] == [2, 5, 7, 9]
        assert L.Plan.of(d).as_dict() == d
    finally:
        L.tune_set(saved)


def test_fixpoint_work_reports_seven_values(L):
    """Pass and rerun evaluations and raises, rerun tiles and idle ones, and the pass
    order taken: the count is part of the ABI, so a caller can size its array."""
    v = (C.c_int64 * 9)(*([-7] * 9))
    assert L.lib().lopc_last_fixpoint_work(v, 9) == 7
    assert v[7] == v[8] == -7  # nothing past the seventh value is written
    assert set(L.last_fixpoint_work()) == {"pass_evals", "pass_raises", "rerun_evals", "rerun_raises",
                                           "rerun_tiles", "rerun_idle", "pass_ordered"}
