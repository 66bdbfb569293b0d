"""GB300 (sm_103a) engine for HP-MOCD (arXiv 2506.01752): one NSGA-II
generation of Alg. 1 -- crossover, mutation, evaluation of both objectives and
environmental selection -- batched over the whole population on one GPU.

This module is a thin ctypes binding of the C ABI in ``include/mocd.h``: it
only marshals arguments. Every step runs in the CUDA library
``_build/libmocd.so`` (built by ``paper_2506_01752_gb300.build.build()``); if
that library is missing, loading fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

__all__ = [
    "MocdError", "Params", "Front", "library_path", "load",
    "graph_upload", "population_init", "generation", "pareto_front",
    "get_population", "get_offspring", "set_population", "evaluate", "synchronize",
    "set_timing", "kernel_times", "info", "destroy", "status_string", "evaluate_noalloc",
    "batch_create", "batch_generation", "batch_autotune", "batch_synchronize", "batch_destroy",
    "batch_configure", "batch_form",
    "Server", "FrontStats", "front_stats", "select_solution", "job_footprint", "debug_inject",
    "debug_pool_usage", "debug_checks", "load_library", "use_library", "SITE_DEVICE_ALLOC", "SITE_GENERATION",
    "SELECT_MODULARITY", "SELECT_COMMUNITIES", "SELECT_SIZE_VARIANCE", "SELECT_MEAN_CONDUCTANCE",
    "SELECT_MAX_CONDUCTANCE", "STAGES",
]

STAGES = ("crossover", "mutation", "evaluate", "select")

OK = 0
ERR_BUFFER_TOO_SMALL = -7


class MocdError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class _CParams(ctypes.Structure):
    _fields_ = [("pop_size", ctypes.c_int32), ("n_parents", ctypes.c_int32),
                ("p_crossover", ctypes.c_double), ("p_mutation", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("init_mode", ctypes.c_int32)]


@dataclass
class Params:
    """Alg. 1 parameters; defaults are the paper's (N_p 100, E_S 4, C_P 0.8, M_P 0.2)."""
    pop_size: int = 100
    n_parents: int = 4
    p_crossover: float = 0.8
    p_mutation: float = 0.2
    seed: int = 0
    init_mode: int = 0

    def _c(self) -> _CParams:
        return _CParams(self.pop_size, self.n_parents, self.p_crossover, self.p_mutation,
                        self.seed, self.init_mode)


@dataclass
class Front:
    """Pareto front F_1 in P order and the recommended member (Alg. 3)."""
    labels: np.ndarray   # [count][n] int32
    f1: np.ndarray
    f2: np.ndarray
    intra: np.ndarray
    sumsq: np.ndarray
    best: int


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = load_library(library_path())
    return _lib


def load_library(path: str):
    """A ctypes handle of the library at ``path`` (e.g. the debug build) with
    every function's signature declared; ``use_library`` makes the module's
    calls go through it."""
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_2506_01752_gb300.build.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    sig = {
        "mocd_graph_upload": (ctypes.c_int, [ctypes.POINTER(P), i64, P, P, P]),
        "mocd_population_init": (ctypes.c_int, [P, ctypes.POINTER(_CParams)]),
        "mocd_generation": (ctypes.c_int, [P, i32]),
        "mocd_pareto_front": (ctypes.c_int, [P, i32, P, P, P, P, P, P, P]),
        "mocd_front_stats": (ctypes.c_int, [P, i32, P, P, P, P, P]),
        "mocd_select_solution": (ctypes.c_int, [P, i32, i64, P]),
        "mocd_get_population": (ctypes.c_int, [P, P, P, P, P]),
        "mocd_get_offspring": (ctypes.c_int, [P, P, P, P]),
        "mocd_set_population": (ctypes.c_int, [P, ctypes.POINTER(_CParams), P, i32]),
        "mocd_evaluate": (ctypes.c_int, [P, i32, P, P, P]),
        "mocd_synchronize": (ctypes.c_int, [P]),
        "mocd_set_timing": (ctypes.c_int, [P, i32]),
        "mocd_kernel_times": (ctypes.c_int, [P, P, i32]),
        "mocd_info": (ctypes.c_int, [P, P, P, P, P]),
        "mocd_generation_kernels": (ctypes.c_int, [P, P]),
        "mocd_destroy": (None, [P]),
        "mocd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "mocd_evaluate_noalloc": (ctypes.c_int, [P, P, i64, P, i32, P, P, P]),
        "mocd_batch_create": (ctypes.c_int, [ctypes.POINTER(P), i32, P, P]),
        "mocd_batch_generation": (ctypes.c_int, [P, i32]),
        "mocd_batch_autotune": (ctypes.c_int, [P, i32, P]),
        "mocd_batch_synchronize": (ctypes.c_int, [P]),
        "mocd_batch_destroy": (None, [P]),
        "mocd_batch_configure": (ctypes.c_int, [P, i32, i32]),
        "mocd_batch_form": (ctypes.c_int, [P, P, P]),
        "mocd_server_create": (ctypes.c_int, [ctypes.POINTER(P), i64, i32, i32]),
        "mocd_server_submit": (ctypes.c_int, [P, i64, P, P, ctypes.POINTER(_CParams), i32, P]),
        "mocd_server_start": (ctypes.c_int, [P, i32, i32]),
        "mocd_server_step": (ctypes.c_int, [P, P, P, P]),
        "mocd_server_job_state": (ctypes.c_int, [P, i64, P, P]),
        "mocd_server_result": (ctypes.c_int, [P, i64, i32, P, P, P, P, P, P, P]),
        "mocd_server_destroy": (None, [P]),
        "mocd_server_cancel": (ctypes.c_int, [P, i64]),
        "mocd_job_footprint": (ctypes.c_int, [i64, P, i32, P]),
        "mocd_debug_inject": (ctypes.c_int, [i32, i32, i32, i32]),
        "mocd_debug_pool_usage": (ctypes.c_int, [i32, P, P]),
        "mocd_pool_trim": (ctypes.c_int, [i64]),
        "mocd_debug_checks": (ctypes.c_int, [P, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def use_library(lib):
    """Route this module's calls through ``lib`` (a load_library handle);
    returns the handle used before."""
    global _lib
    old, _lib = _lib, lib
    return old


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != OK:
        raise MocdError(rc, what)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return int(getattr(stream, "cuda_stream")) or None


def status_string(status: int) -> str:
    return load().mocd_status_string(status).decode()


def graph_upload(row_ptr, col_idx, stream=None):
    """Validate and upload a symmetric CSR graph; returns a context handle."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    ctx = ctypes.c_void_p()
    _check(load().mocd_graph_upload(ctypes.byref(ctx), rp.size - 1, _p(rp), _p(ci),
                                    _stream_handle(stream)), "mocd_graph_upload")
    return ctx


def population_init(ctx, params: Params):
    c = params._c()
    _check(load().mocd_population_init(ctx, ctypes.byref(c)), "mocd_population_init")


def generation(ctx, n_generations: int = 1):
    _check(load().mocd_generation(ctx, int(n_generations)), "mocd_generation")


def info(ctx):
    n = ctypes.c_int64()
    m = ctypes.c_int64()
    np_ = ctypes.c_int32()
    g = ctypes.c_int32()
    _check(load().mocd_info(ctx, ctypes.byref(n), ctypes.byref(m), ctypes.byref(np_), ctypes.byref(g)),
           "mocd_info")
    return dict(n=n.value, m=m.value, pop_size=np_.value, generation=g.value)


def generation_kernels(ctx) -> int:
    """Kernel launches in one generation of this context's graph."""
    k = ctypes.c_int32()
    _check(load().mocd_generation_kernels(ctx, ctypes.byref(k)), "mocd_generation_kernels")
    return k.value


def pareto_front(ctx, with_labels: bool = True) -> Front:
    d = info(ctx)
    n, cap = d["n"], max(d["pop_size"], 1)
    count = ctypes.c_int32()
    best = ctypes.c_int32()
    labels = np.zeros((cap, n), dtype=np.int32) if with_labels else None
    f1 = np.zeros(cap, dtype=np.float64)
    f2 = np.zeros(cap, dtype=np.float64)
    intra = np.zeros(cap, dtype=np.int64)
    sumsq = np.zeros(cap, dtype=np.int64)
    _check(load().mocd_pareto_front(ctx, cap, ctypes.byref(count), _p(labels), _p(f1), _p(f2), _p(intra),
                                    _p(sumsq), ctypes.byref(best)), "mocd_pareto_front")
    k = count.value
    return Front(labels[:k] if labels is not None else None, f1[:k], f2[:k], intra[:k], sumsq[:k], best.value)


SELECT_MODULARITY = 0
SELECT_COMMUNITIES = 1
SELECT_SIZE_VARIANCE = 2
SELECT_MEAN_CONDUCTANCE = 3
SELECT_MAX_CONDUCTANCE = 4


@dataclass
class FrontStats:
    """Community statistics of each front member, in pareto_front order."""
    communities: np.ndarray       # int64: number of non-empty communities k
    size_sumsq: np.ndarray        # int64: sum_c n_c^2
    mean_conductance: np.ndarray  # float64: (exact sum_c phi_c, rounded once) / k
    max_conductance: np.ndarray   # float64: max_c phi_c


def front_stats(ctx) -> FrontStats:
    cap = max(info(ctx)["pop_size"], 1)
    count = ctypes.c_int32()
    k = np.zeros(cap, np.int64)
    sq = np.zeros(cap, np.int64)
    mean = np.zeros(cap, np.float64)
    mx = np.zeros(cap, np.float64)
    _check(load().mocd_front_stats(ctx, cap, ctypes.byref(count), _p(k), _p(sq), _p(mean), _p(mx)),
           "mocd_front_stats")
    c = count.value
    return FrontStats(k[:c], sq[:c], mean[:c], mx[:c])


def select_solution(ctx, criterion: int = SELECT_MODULARITY, target: int = 0) -> int:
    """Index into pareto_front of the member `criterion` prefers."""
    idx = ctypes.c_int32()
    _check(load().mocd_select_solution(ctx, int(criterion), int(target), ctypes.byref(idx)),
           "mocd_select_solution")
    return idx.value


def get_population(ctx):
    """(labels [N_p][n], k1, k2, generation) of P in P order."""
    d = info(ctx)
    labels = np.zeros((d["pop_size"], d["n"]), dtype=np.int32)
    k1 = np.zeros(d["pop_size"], dtype=np.int64)
    k2 = np.zeros(d["pop_size"], dtype=np.int64)
    g = ctypes.c_int32()
    _check(load().mocd_get_population(ctx, _p(labels), _p(k1), _p(k2), ctypes.byref(g)), "mocd_get_population")
    return labels, k1, k2, g.value


def get_offspring(ctx):
    """(labels [N_p][n], k1, k2) of the most recent generation's children Q."""
    d = info(ctx)
    labels = np.zeros((d["pop_size"], d["n"]), dtype=np.int32)
    k1 = np.zeros(d["pop_size"], dtype=np.int64)
    k2 = np.zeros(d["pop_size"], dtype=np.int64)
    _check(load().mocd_get_offspring(ctx, _p(labels), _p(k1), _p(k2)), "mocd_get_offspring")
    return labels, k1, k2


def set_population(ctx, params: Params, labels, generation: int = 0):
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    c = params._c()
    _check(load().mocd_set_population(ctx, ctypes.byref(c), _p(lab), int(generation)), "mocd_set_population")


def evaluate(ctx, labels):
    """Exact (intra, S) of each labelling in ``labels`` ([count][n])."""
    lab = np.ascontiguousarray(np.atleast_2d(labels), dtype=np.int32)
    intra = np.zeros(lab.shape[0], dtype=np.int64)
    sumsq = np.zeros(lab.shape[0], dtype=np.int64)
    _check(load().mocd_evaluate(ctx, lab.shape[0], _p(lab), _p(intra), _p(sumsq)), "mocd_evaluate")
    return intra, sumsq


NOALLOC_MAX_CELLS = 4194304


def evaluate_noalloc(row_ptr_dev: int, col_idx_dev: int, n: int, labels_dev: int, count: int,
                     intra_dev: int, sumsq_dev: int, stream=None):
    """Objective evaluation that allocates no device memory (see
    ``mocd_evaluate_noalloc`` in include/mocd.h). Every argument except ``n``,
    ``count`` and ``stream`` is a raw device pointer (an int); ``labels_dev``
    is node-major ``[n][W]`` with ``W`` = ``count`` rounded up to 4. The call
    is asynchronous on ``stream``."""
    _check(load().mocd_evaluate_noalloc(row_ptr_dev, col_idx_dev, int(n), labels_dev, int(count), intra_dev,
                                        sumsq_dev, _stream_handle(stream)), "mocd_evaluate_noalloc")


def batch_create(ctxs, stream=None):
    """Group initialised contexts; one CUDA-graph launch then runs a
    generation of every one of them (see mocd_batch_create)."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    b = ctypes.c_void_p()
    _check(load().mocd_batch_create(ctypes.byref(b), len(ctxs), ctypes.cast(arr, ctypes.c_void_p),
                                    _stream_handle(stream)), "mocd_batch_create")
    b._members = list(ctxs)
    return b


def batch_generation(b, n_generations: int = 1):
    _check(load().mocd_batch_generation(b, int(n_generations)), "mocd_batch_generation")


def batch_autotune(b, generations_per_trial: int = 3) -> int:
    out = ctypes.c_int32()
    _check(load().mocd_batch_autotune(b, int(generations_per_trial), ctypes.byref(out)), "mocd_batch_autotune")
    return out.value


def batch_configure(b, nodes_per_warp: int = 1, form: int = 0):
    """Launch shape and form of a batch (see mocd_batch_configure): form 0 per
    member, 1 merged selection, 2 merged crossover, votes, evaluation and
    selection."""
    _check(load().mocd_batch_configure(b, int(nodes_per_warp), int(form)), "mocd_batch_configure")


def batch_form(b):
    """(nodes per warp, form) of a batch."""
    npw = ctypes.c_int32()
    form = ctypes.c_int32()
    _check(load().mocd_batch_form(b, ctypes.byref(npw), ctypes.byref(form)), "mocd_batch_form")
    return npw.value, form.value


def batch_synchronize(b):
    _check(load().mocd_batch_synchronize(b), "mocd_batch_synchronize")


def batch_destroy(b):
    if b is not None and b.value:
        load().mocd_batch_destroy(b)
        b.value = None


class Server:
    """Continuous-batching detection server (mocd_server_* in include/mocd.h)."""

    QUEUED, RUNNING, DONE, FAILED, CANCELLED = 0, 1, 2, 3, 4

    def __init__(self, hbm_budget_bytes: int, max_running: int = 64, depth: int = 2):
        self.h = ctypes.c_void_p()
        _check(load().mocd_server_create(ctypes.byref(self.h), int(hbm_budget_bytes), int(max_running),
                                         int(depth)), "mocd_server_create")
        self._n = {}
        self._np = {}

    def start(self, admission_threads: int = 2, policy: int = 0):
        """Background mode: scheduler thread plus admission workers."""
        _check(load().mocd_server_start(self.h, int(admission_threads), int(policy)), "mocd_server_start")

    def submit(self, row_ptr, col_idx, params: Params, generations: int = 100) -> int:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        c = params._c()
        jid = ctypes.c_int64()
        _check(load().mocd_server_submit(self.h, rp.size - 1, _p(rp), _p(ci), ctypes.byref(c), int(generations),
                                         ctypes.byref(jid)), "mocd_server_submit")
        self._n[jid.value] = rp.size - 1
        self._np[jid.value] = params.pop_size
        return jid.value

    def step(self):
        r = ctypes.c_int32()
        q = ctypes.c_int32()
        d = ctypes.c_int32()
        _check(load().mocd_server_step(self.h, ctypes.byref(r), ctypes.byref(q), ctypes.byref(d)), "mocd_server_step")
        return r.value, q.value, d.value

    def cancel(self, job_id: int):
        """Cancel a queued or running job (retired by a later round)."""
        _check(load().mocd_server_cancel(self.h, int(job_id)), "mocd_server_cancel")

    def state(self, job_id: int):
        st = ctypes.c_int32()
        status = ctypes.c_int32()
        _check(load().mocd_server_job_state(self.h, int(job_id), ctypes.byref(st), ctypes.byref(status)),
               "mocd_server_job_state")
        return st.value, status.value

    def result(self, job_id: int) -> Front:
        n, cap = self._n[job_id], self._np[job_id]
        count = ctypes.c_int32()
        best = ctypes.c_int32()
        labels = np.zeros((cap, n), dtype=np.int32)
        f1 = np.zeros(cap)
        f2 = np.zeros(cap)
        intra = np.zeros(cap, dtype=np.int64)
        sumsq = np.zeros(cap, dtype=np.int64)
        _check(load().mocd_server_result(self.h, int(job_id), cap, ctypes.byref(count), _p(labels), _p(f1), _p(f2),
                                         _p(intra), _p(sumsq), ctypes.byref(best)), "mocd_server_result")
        k = count.value
        return Front(labels[:k], f1[:k], f2[:k], intra[:k], sumsq[:k], best.value)

    def close(self):
        if self.h is not None and self.h.value:
            load().mocd_server_destroy(self.h)
            self.h.value = None


def job_footprint(row_ptr, pop_size: int = 100) -> int:
    """Device bytes the server accounts for a job on this graph while it runs."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    out = ctypes.c_int64()
    _check(load().mocd_job_footprint(rp.size - 1, _p(rp), int(pop_size), ctypes.byref(out)), "mocd_job_footprint")
    return out.value


SITE_DEVICE_ALLOC = 0
SITE_GENERATION = 1


def debug_inject(site: int, skip: int = 0, count: int = 1, status: int = -8):
    """Host-side failure injection (test support): after `skip` calls at
    `site` pass, the next `count` fail; count 0 disarms."""
    _check(load().mocd_debug_inject(int(site), int(skip), int(count), int(status)), "mocd_debug_inject")


def debug_checks(reset: bool = True):
    """(built with checks, failures, first code, first index) of the bounds
    checks of the debug build (all zero in the normal build)."""
    out = np.zeros(3, dtype=np.uint64)
    rc = load().mocd_debug_checks(_p(out), 1 if reset else 0)
    if rc < 0:
        raise MocdError(rc, "mocd_debug_checks")
    return bool(rc), int(out[0]), int(out[1]), int(out[2])


def debug_pool_usage(reset_peak: bool = False):
    """(bytes in use, high-water mark) of the device's default memory pool."""
    cur = ctypes.c_int64()
    peak = ctypes.c_int64()
    _check(load().mocd_debug_pool_usage(1 if reset_peak else 0, ctypes.byref(cur), ctypes.byref(peak)),
           "mocd_debug_pool_usage")
    return cur.value, peak.value


def pool_trim(keep_bytes: int = 0) -> None:
    """Release the device memory the library's pool keeps for later contexts
    (down to keep_bytes)."""
    _check(load().mocd_pool_trim(int(keep_bytes)), "mocd_pool_trim")


def synchronize(ctx):
    _check(load().mocd_synchronize(ctx), "mocd_synchronize")


def set_timing(ctx, enable: bool):
    _check(load().mocd_set_timing(ctx, 1 if enable else 0), "mocd_set_timing")


def kernel_times(ctx) -> dict:
    """Milliseconds of each stage of the most recent generation."""
    ms = np.zeros(len(STAGES), dtype=np.float32)
    rc = load().mocd_kernel_times(ctx, _p(ms), len(STAGES))
    if rc < 0:
        raise MocdError(rc, "mocd_kernel_times")
    return dict(zip(STAGES, ms.tolist()))


def destroy(ctx):
    if ctx is not None and ctx.value:
        load().mocd_destroy(ctx)
        ctx.value = None
