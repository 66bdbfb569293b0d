"""ctypes wrapper around the plain C oracle in ``mocd_oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline / reference leg are the only users. The CUDA library
neither imports nor links this package. Labels here are individual-major
arrays ``[count][n]`` of int32; keys are ``k1 = m - intra`` and ``k2 = S``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mocd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmocd_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                    "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


class _Params(ctypes.Structure):
    _fields_ = [("pop_size", ctypes.c_int32), ("n_parents", ctypes.c_int32),
                ("p_crossover", ctypes.c_double), ("p_mutation", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("init_mode", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        sig = {
            "orc_philox4x32_10": (None, [P, P, P]),
            "orc_pick": (u32, [u32, u32]),
            "orc_threshold": (ctypes.c_uint64, [ctypes.c_double]),
            "orc_objectives": (ctypes.c_int, [i64, P, P, P, P, P]),
            "orc_nondominated_sort": (ctypes.c_int, [i32, P, P, P]),
            "orc_crowding": (ctypes.c_int, [i32, P, P, P, P]),
            "orc_sort_rank_crowd": (ctypes.c_int, [i32, P, P, P]),
            "orc_rank_crowd_order": (ctypes.c_int, [i32, P, P, P, P, P]),
            "orc_mode_pick": (i32, [i32, P, u32]),
            "orc_operators_forced": (ctypes.c_int, [i64, P, P, i32, P, P, P, P, P, P]),
            "orc_init_population": (ctypes.c_int, [i64, P, P]),
            "orc_select_parents": (ctypes.c_int, [P, u32, P, P, P, P, P]),
            "orc_make_offspring": (ctypes.c_int, [i64, P, P, P, u32, P, P, P, P, P, P]),
            "orc_make_offspring_range": (ctypes.c_int, [i64, P, P, P, u32, P, P, P, i32, i32, P, P, P]),
            "orc_env_select": (ctypes.c_int, [i32, P, P, P]),
            "orc_run": (ctypes.c_int, [i64, P, P, P, u32, i32, P, P, P]),
            "orc_population_init": (ctypes.c_int, [i64, P, P, P, P, P, P]),
            "orc_pareto_front": (ctypes.c_int, [i32, P, P, i64, P, P, P]),
            "orc_objective_values": (None, [i64, i64, i64, P, P]),
            "orc_community_stats": (ctypes.c_int, [i64, P, P, i32, P, P, P, P, P]),
            "orc_select_solution": (ctypes.c_int32, [i32, i64, i64, P, P, P, P, P, P, i32, i64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


@dataclass
class Params:
    """Alg. 1 parameters: N_p, E_S, C_P, M_P (defaults: the paper's table)."""
    pop_size: int = 100
    n_parents: int = 4
    p_crossover: float = 0.8
    p_mutation: float = 0.2
    seed: int = 0
    init_mode: int = 0

    def _c(self):
        return _Params(self.pop_size, self.n_parents, self.p_crossover,
                       self.p_mutation, self.seed, self.init_mode)


@dataclass
class State:
    """P in P order: labels [N_p][n], keys k1 = m - intra, k2 = S, generation."""
    labels: np.ndarray
    k1: np.ndarray
    k2: np.ndarray
    generation: int


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def pick(u: int, k: int) -> int:
    return int(_load().orc_pick(u, k))


def threshold(p: float) -> int:
    return int(_load().orc_threshold(p))


def _graph(row_ptr, col_idx):
    return (np.ascontiguousarray(row_ptr, dtype=np.int64),
            np.ascontiguousarray(col_idx, dtype=np.int32))


def objectives(row_ptr, col_idx, labels):
    """Exact (intra, S) of each labelling in ``labels`` ([count][n] or [n])."""
    rp, ci = _graph(row_ptr, col_idx)
    n = rp.size - 1
    lab = np.ascontiguousarray(np.atleast_2d(labels), dtype=np.int32)
    intra = np.zeros(lab.shape[0], dtype=np.int64)
    sumsq = np.zeros(lab.shape[0], dtype=np.int64)
    one_i = np.zeros(1, np.int64)
    one_s = np.zeros(1, np.int64)
    for r in range(lab.shape[0]):
        row = np.ascontiguousarray(lab[r])
        _check(_load().orc_objectives(n, _p(rp), _p(ci), _p(row), _p(one_i), _p(one_s)), "objectives")
        intra[r], sumsq[r] = one_i[0], one_s[0]
    return intra, sumsq


def objective_values(m: int, k1: int, k2: int):
    f1 = ctypes.c_double()
    f2 = ctypes.c_double()
    _load().orc_objective_values(m, k1, k2, ctypes.byref(f1), ctypes.byref(f2))
    return f1.value, f2.value


def nondominated_sort(k1, k2):
    a = np.ascontiguousarray(k1, dtype=np.int64)
    b = np.ascontiguousarray(k2, dtype=np.int64)
    rank = np.zeros(a.size, dtype=np.int32)
    _check(_load().orc_nondominated_sort(a.size, _p(a), _p(b), _p(rank)), "sort")
    return rank


def crowding(k1, k2, rank):
    a = np.ascontiguousarray(k1, dtype=np.int64)
    b = np.ascontiguousarray(k2, dtype=np.int64)
    r = np.ascontiguousarray(rank, dtype=np.int32)
    out = np.zeros(a.size, dtype=np.float64)
    _check(_load().orc_crowding(a.size, _p(a), _p(b), _p(r), _p(out)), "crowding")
    return out


def rank_crowd_order(k1, k2):
    a = np.ascontiguousarray(k1, dtype=np.int64)
    b = np.ascontiguousarray(k2, dtype=np.int64)
    rank = np.zeros(a.size, dtype=np.int32)
    crowd = np.zeros(a.size, dtype=np.float64)
    order = np.zeros(a.size, dtype=np.int32)
    _check(_load().orc_rank_crowd_order(a.size, _p(a), _p(b), _p(rank), _p(crowd), _p(order)), "rank")
    return rank, crowd, order


def mode_pick(x, u: int) -> int:
    a = np.ascontiguousarray(x, dtype=np.int32)
    return int(_load().orc_mode_pick(a.size, _p(a), u))


def operators_forced(row_ptr, col_idx, parents, xtie, sel, mtie):
    """Crossover of the given parents then mutation of the nodes in ``sel``."""
    rp, ci = _graph(row_ptr, col_idx)
    n = rp.size - 1
    par = np.ascontiguousarray(parents, dtype=np.int32)
    xt = np.ascontiguousarray(xtie, dtype=np.uint32)
    se = np.ascontiguousarray(sel, dtype=np.uint8)
    mt = np.ascontiguousarray(mtie, dtype=np.uint32)
    child = np.zeros(n, dtype=np.int32)
    q = np.zeros(n, dtype=np.int32)
    _check(_load().orc_operators_forced(n, _p(rp), _p(ci), par.shape[0], _p(par), _p(xt),
                                        _p(se), _p(mt), _p(child), _p(q)), "operators")
    return child, q


def init_population(n: int, params: Params):
    P = np.zeros((params.pop_size, n), dtype=np.int32)
    pr = params._c()
    _check(_load().orc_init_population(n, ctypes.byref(pr), _p(P)), "init")
    return P


def population_init(row_ptr, col_idx, params: Params) -> State:
    rp, ci = _graph(row_ptr, col_idx)
    n = rp.size - 1
    P = np.zeros((params.pop_size, n), dtype=np.int32)
    k1 = np.zeros(params.pop_size, dtype=np.int64)
    k2 = np.zeros(params.pop_size, dtype=np.int64)
    pr = params._c()
    _check(_load().orc_population_init(n, _p(rp), _p(ci), ctypes.byref(pr), _p(P), _p(k1), _p(k2)),
           "population_init")
    return State(P, k1, k2, 0)


def select_parents(params: Params, gen: int, k1, k2):
    Np, E = params.pop_size, params.n_parents
    a = np.ascontiguousarray(k1, dtype=np.int64)
    b = np.ascontiguousarray(k2, dtype=np.int64)
    par = np.zeros((Np, E), dtype=np.int32)
    xo = np.zeros(Np, dtype=np.int32)
    skip = np.zeros(Np, dtype=np.int32)
    pr = params._c()
    _check(_load().orc_select_parents(ctypes.byref(pr), gen, _p(a), _p(b), _p(par), _p(xo), _p(skip)),
           "select_parents")
    return par, xo, skip


def make_offspring(row_ptr, col_idx, params: Params, gen: int, state: State):
    """Q of generation ``gen`` from P = state (labels and keys)."""
    rp, ci = _graph(row_ptr, col_idx)
    n = rp.size - 1
    Np = params.pop_size
    P = np.ascontiguousarray(state.labels, dtype=np.int32)
    k1 = np.ascontiguousarray(state.k1, dtype=np.int64)
    k2 = np.ascontiguousarray(state.k2, dtype=np.int64)
    Q = np.zeros((Np, n), dtype=np.int32)
    qk1 = np.zeros(Np, dtype=np.int64)
    qk2 = np.zeros(Np, dtype=np.int64)
    pr = params._c()
    _check(_load().orc_make_offspring(n, _p(rp), _p(ci), ctypes.byref(pr), gen, _p(P), _p(k1), _p(k2),
                                      _p(Q), _p(qk1), _p(qk2)), "make_offspring")
    return Q, qk1, qk2


def _threads(threads):
    if threads is None:
        threads = min(16, os.cpu_count() or 1)
    return max(1, int(threads))


def make_offspring_parallel(row_ptr, col_idx, params: Params, gen: int, state: State, threads=None):
    """As make_offspring, with the children split over host threads (the C
    oracle releases the GIL; every child is computed by the same sequential
    code, so the result does not depend on the thread count)."""
    from concurrent.futures import ThreadPoolExecutor

    rp, ci = _graph(row_ptr, col_idx)
    n = rp.size - 1
    Np = params.pop_size
    P = np.ascontiguousarray(state.labels, dtype=np.int32)
    k1 = np.ascontiguousarray(state.k1, dtype=np.int64)
    k2 = np.ascontiguousarray(state.k2, dtype=np.int64)
    Q = np.zeros((Np, n), dtype=np.int32)
    qk1 = np.zeros(Np, dtype=np.int64)
    qk2 = np.zeros(Np, dtype=np.int64)
    T = min(_threads(threads), Np)
    cuts = [Np * t // T for t in range(T + 1)]

    def work(t):
        pr = params._c()
        return _load().orc_make_offspring_range(n, _p(rp), _p(ci), ctypes.byref(pr), gen, _p(P), _p(k1),
                                                _p(k2), cuts[t], cuts[t + 1], _p(Q), _p(qk1), _p(qk2))

    with ThreadPoolExecutor(T) as ex:
        for rc in ex.map(work, range(T)):
            _check(rc, "make_offspring_range")
    return Q, qk1, qk2


def objectives_parallel(row_ptr, col_idx, labels, threads=None):
    """As objectives, with the labellings split over host threads."""
    from concurrent.futures import ThreadPoolExecutor

    rp, ci = _graph(row_ptr, col_idx)
    n = rp.size - 1
    lab = np.ascontiguousarray(np.atleast_2d(labels), dtype=np.int32)
    intra = np.zeros(lab.shape[0], dtype=np.int64)
    sumsq = np.zeros(lab.shape[0], dtype=np.int64)

    def work(r):
        row = np.ascontiguousarray(lab[r])
        a, b = np.zeros(1, np.int64), np.zeros(1, np.int64)
        _check(_load().orc_objectives(n, _p(rp), _p(ci), _p(row), _p(a), _p(b)), "objectives")
        intra[r], sumsq[r] = a[0], b[0]

    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(work, range(lab.shape[0])))
    return intra, sumsq


def next_state(state: State, Q, qk1, qk2) -> State:
    """EnvironmentalSelection (Alg. 1) of R = P u Q: the next P in the order
    env_select keeps it (the step orc_run takes after the offspring)."""
    Np = state.k1.size
    rk1 = np.concatenate([np.asarray(state.k1, np.int64), np.asarray(qk1, np.int64)])
    rk2 = np.concatenate([np.asarray(state.k2, np.int64), np.asarray(qk2, np.int64)])
    keep = env_select(rk1, rk2)
    P = np.empty_like(state.labels)
    for k, r in enumerate(keep):
        P[k] = state.labels[r] if r < Np else Q[r - Np]
    return State(P, rk1[keep].copy(), rk2[keep].copy(), state.generation + 1)


def run_parallel(row_ptr, col_idx, params: Params, state: State, generations: int, threads=None) -> State:
    """As run, each generation's children split over host threads; the same
    steps in the same order (offspring, then environmental selection)."""
    for _ in range(generations):
        Q, qk1, qk2 = make_offspring_parallel(row_ptr, col_idx, params, state.generation + 1, state, threads)
        state = next_state(state, Q, qk1, qk2)
    return state


def make_offspring_range(row_ptr, col_idx, params: Params, gen: int, state: State, i0: int, i1: int):
    """Children i0 <= i < i1 of generation ``gen`` (a bounded sample of one
    generation); rows outside the range are left zero."""
    rp, ci = _graph(row_ptr, col_idx)
    n = rp.size - 1
    Np = params.pop_size
    P = np.ascontiguousarray(state.labels, dtype=np.int32)
    k1 = np.ascontiguousarray(state.k1, dtype=np.int64)
    k2 = np.ascontiguousarray(state.k2, dtype=np.int64)
    Q = np.zeros((Np, n), dtype=np.int32)
    qk1 = np.zeros(Np, dtype=np.int64)
    qk2 = np.zeros(Np, dtype=np.int64)
    pr = params._c()
    _check(_load().orc_make_offspring_range(n, _p(rp), _p(ci), ctypes.byref(pr), gen, _p(P), _p(k1), _p(k2),
                                            i0, i1, _p(Q), _p(qk1), _p(qk2)), "make_offspring_range")
    return Q, qk1, qk2


def env_select(rk1, rk2):
    a = np.ascontiguousarray(rk1, dtype=np.int64)
    b = np.ascontiguousarray(rk2, dtype=np.int64)
    keep = np.zeros(a.size // 2, dtype=np.int32)
    _check(_load().orc_env_select(a.size // 2, _p(a), _p(b), _p(keep)), "env_select")
    return keep


def run(row_ptr, col_idx, params: Params, state: State, generations: int) -> State:
    """``generations`` generations of Alg. 1 after ``state`` (a new State)."""
    rp, ci = _graph(row_ptr, col_idx)
    n = rp.size - 1
    P = np.array(state.labels, dtype=np.int32, copy=True, order="C")
    k1 = np.array(state.k1, dtype=np.int64, copy=True)
    k2 = np.array(state.k2, dtype=np.int64, copy=True)
    pr = params._c()
    _check(_load().orc_run(n, _p(rp), _p(ci), ctypes.byref(pr), state.generation, generations,
                           _p(P), _p(k1), _p(k2)), "run")
    return State(P, k1, k2, state.generation + generations)


def pareto_front(state: State, m: int):
    """(members as P positions, index of the recommended member in that list)."""
    Np = state.k1.size
    k1 = np.ascontiguousarray(state.k1, dtype=np.int64)
    k2 = np.ascontiguousarray(state.k2, dtype=np.int64)
    members = np.zeros(Np, dtype=np.int32)
    count = ctypes.c_int32()
    best = ctypes.c_int32()
    _check(_load().orc_pareto_front(Np, _p(k1), _p(k2), m, ctypes.byref(count), _p(members),
                                    ctypes.byref(best)), "pareto_front")
    return members[: count.value].copy(), best.value


def community_stats(row_ptr, col_idx, labels):
    """Per labeling: (communities k, sum_c n_c^2, mean conductance, max
    conductance), Sec. 4.4; see orc_community_stats."""
    rp, ci = _graph(row_ptr, col_idx)
    n = rp.size - 1
    L = np.ascontiguousarray(np.atleast_2d(labels), dtype=np.int32)
    cnt = L.shape[0]
    k = np.zeros(cnt, np.int64)
    sq = np.zeros(cnt, np.int64)
    mean = np.zeros(cnt, np.float64)
    mx = np.zeros(cnt, np.float64)
    _check(_load().orc_community_stats(n, _p(rp), _p(ci), cnt, _p(L), _p(k), _p(sq), _p(mean), _p(mx)),
           "community_stats")
    return k, sq, mean, mx


def select_solution(m: int, n: int, k1, k2, stats, criterion: int, target: int = 0) -> int:
    """Index of the preferred front member (Alg. 3 / Sec. 4.4 criteria 0-4)."""
    k1 = np.ascontiguousarray(k1, dtype=np.int64)
    k2 = np.ascontiguousarray(k2, dtype=np.int64)
    k, sq, mean, mx = (np.ascontiguousarray(a) for a in stats)
    return int(_load().orc_select_solution(k1.size, m, n, _p(k1), _p(k2), _p(k), _p(sq), _p(mean), _p(mx),
                                           criterion, target))
