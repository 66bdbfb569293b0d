"""C ABI checks that need no GPU: the library loads, exports every function
that include/mocd.h declares, and rejects malformed graphs before touching
the device; the product path fails loudly when the library is missing."""
import os
import re

import numpy as np
import pytest

import paper_2506_01752_gb300 as mocd
import synth
from paper_2506_01752_gb300 import build as cuda_build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mocd.h")


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return mocd.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mocd_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "mocd_graph_upload" in names and "mocd_generation" in names
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert mocd.status_string(0) == "ok"
    assert "symmetric" in mocd.status_string(-2)
    assert mocd.status_string(-99) == "unknown status"


def _upload_status(rp, ci):
    import ctypes
    ctx = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    rc = mocd.load().mocd_graph_upload(ctypes.byref(ctx), rp.size - 1, rp.ctypes.data_as(ctypes.c_void_p),
                                       ci.ctypes.data_as(ctypes.c_void_p), None)
    if rc == 0:
        mocd.destroy(ctx)
    return rc


@pytest.mark.parametrize("rp,ci,status", [
    ([0, 1, 2], [0, 1], -3),              # self loops
    ([0, 2, 4], [1, 1, 0, 0], -4),        # repeated edge
    ([0, 0, 0], [], -5),                  # no edges
    ([0, 1, 2], [1, 5], -1),              # neighbour out of range
    ([0, 2, 1], [1, 0], -1),              # row_ptr decreasing
])
def test_graph_validation_before_device(lib, rp, ci, status):
    assert _upload_status(rp, ci) == status


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(mocd, "_lib", None)
    monkeypatch.setattr(mocd, "library_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        mocd.load()


def test_server_host_side(lib):
    """Queueing and job bookkeeping happen on the host only."""
    srv = mocd.Server(1 << 30, max_running=2, depth=1)
    try:
        jid = srv.submit([0, 1, 2], [1, 0], mocd.Params(pop_size=4), 3)
        assert jid == 1 and srv.state(jid) == (mocd.Server.QUEUED, 0)
        with pytest.raises(mocd.MocdError) as e:
            srv.result(jid)
        assert e.value.status == -9
        with pytest.raises(mocd.MocdError):
            srv.state(99)
    finally:
        srv.close()
    import ctypes
    h = ctypes.c_void_p()
    assert mocd.load().mocd_server_create(ctypes.byref(h), 0, 1, 1) == -1


def _big_graph():
    rp, ci, _ = synth.lfr_style(20000, 20, 50, 0.3, seed=4)  # ~400k entries: several threads
    return rp.astype(np.int64), ci.astype(np.int32).copy()


def _validation_codes():
    return {-1, -2, -3, -4, -5}


def test_large_graph_validation_passes_with_shuffled_rows(lib):
    """Rows in any order are accepted (a sorted copy is made); sorted rows are
    used as given. Without a GPU the call then fails at the device step, not
    in validation."""
    rp, ci = _big_graph()
    assert _upload_status(rp, ci) not in _validation_codes()
    rng = np.random.default_rng(0)
    for v in range(0, rp.size - 1, 7):
        seg = ci[rp[v]:rp[v + 1]].copy()
        rng.shuffle(seg)
        ci[rp[v]:rp[v + 1]] = seg
    assert _upload_status(rp, ci) not in _validation_codes()


@pytest.mark.parametrize("defect", ["self_loop_first", "range_first", "dup_unsorted", "sorted_order_decides",
                                    "hidden_repeat"])
def test_large_graph_first_failing_row_decides(lib, defect):
    """Defects in rows handled by different threads: the status is that of
    the lowest-numbered failing row, as in a sequential scan. (Symmetry is
    checked on the device after every row passed; see the GPU tests.)"""
    rp, ci = _big_graph()
    lo, hi = 10, rp.size - 50  # first and last thread ranges
    if defect == "self_loop_first":
        ci[rp[lo]] = lo           # row lo: self loop (also breaks symmetry)
        ci[rp[hi]] = rp.size + 5  # row hi: out of range
        want = -3
    elif defect == "range_first":
        ci[rp[lo]] = -7
        ci[rp[hi]] = hi
        want = -1
    elif defect == "dup_unsorted":
        seg = ci[rp[hi]:rp[hi + 1]].copy()
        seg[-1] = seg[0]           # repeated neighbour
        ci[rp[hi]:rp[hi + 1]] = seg[::-1]
        want = -4
    elif defect == "sorted_order_decides":
        # Row lo as given meets a repeat before an out-of-range id; in sorted
        # order the negative id comes first, so the row fails as out of range.
        v = next(u for u in range(lo, hi) if rp[u + 1] - rp[u] >= 4)
        a = ci[rp[v]]
        b = ci[rp[v] + 1]
        ci[rp[v]:rp[v] + 4] = [a, b, b, -1]
        ci[rp[hi]] = hi            # a later row with a self loop
        want = -1
    else:
        # Row lo repeats a neighbour non-adjacently (unsorted): only the
        # sorted order shows the repeat.
        v = next(u for u in range(lo, hi) if rp[u + 1] - rp[u] >= 3)
        seg = ci[rp[v]:rp[v + 1]].copy()
        seg[2] = seg[0]
        seg[0], seg[1] = seg[1], seg[0]
        ci[rp[v]:rp[v + 1]] = seg
        ci[rp[hi]] = -3            # a later row out of range
        want = -4
    assert _upload_status(rp, ci) == want


def test_debug_build_loads_and_exports_every_symbol():
    """The bounds-checked variant (-DMOCD_DEBUG_CHECKS) builds and exports
    the same C ABI."""
    lib = mocd.load_library(cuda_build.build(debug=True))
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_concurrent_validation_from_several_threads(lib):
    """Host threads validating graphs at the same time (as the server's
    admission threads do) share the library's worker threads or run their
    checks themselves; every call still reports its own graph's status."""
    from concurrent.futures import ThreadPoolExecutor

    rp, ci = _big_graph()
    cases = []
    for k in range(12):
        c = ci.copy()
        if k % 3 == 0:
            c[rp[10 + k]] = 10 + k  # self loop
            want = -3
        elif k % 3 == 1:
            c[rp[500 + k]] = -1     # out of range
            want = -1
        else:
            want = None             # valid: fails later, at the device step, without a GPU
        cases.append((c, want))

    def upload(case):
        c, want = case
        return _upload_status(rp, c), want

    with ThreadPoolExecutor(max_workers=6) as ex:
        for _ in range(3):
            for got, want in ex.map(upload, cases):
                if want is None:
                    assert got not in _validation_codes()
                else:
                    assert got == want


def _validate_in_child(conn):
    rp, ci = _big_graph()
    c = ci.copy()
    c[rp[123]] = 123  # self loop
    conn.send(_upload_status(rp, c))
    conn.close()


@pytest.mark.filterwarnings("ignore::DeprecationWarning")  # forking a threaded process is the point
def test_validation_in_a_forked_child(lib):
    """A process forked after the library's worker threads exist (they do not
    survive the fork) makes its own: validation in the child completes."""
    import multiprocessing as mp

    rp, ci = _big_graph()
    assert _upload_status(rp, ci) not in _validation_codes()  # the parent's workers exist now
    ctx = mp.get_context("fork")
    parent, child = ctx.Pipe()
    p = ctx.Process(target=_validate_in_child, args=(child,))
    p.start()
    try:
        assert parent.poll(120), "validation in the forked child did not finish"
        assert parent.recv() == -3
    finally:
        p.join(30)
        if p.is_alive():
            p.kill()
