"""Seeded synthetic graphs in symmetric CSR form, plus random label vectors.

Workloads (stand-ins for the paper's networkx LFR graphs, Sec. 5.2, and its
planted-community examples; the paper's real-world datasets are not used):

* ``planted_partition``: ``k`` equal communities, each pair of nodes joined with
  probability ``p_in`` inside a community and ``p_out`` across.
* ``lfr_style``: an LFR-like generator written here (not networkx's): node
  degrees from a truncated power law (exponent ``tau1``, mean ``avg_deg``,
  maximum ``max_deg``), community sizes from a truncated power law (exponent
  ``tau2`` in ``[cmin, cmax]``), nodes assigned to communities at random, a
  fraction ``1 - mu`` of each node's stubs wired inside its community and the
  rest across communities by configuration-model pairing; self loops and
  repeated edges are dropped.

Everything is drawn from ``numpy.random.default_rng(seed)``; node ids are not
ordered by community.
"""
from __future__ import annotations

import math

import numpy as np


def csr_from_edges(n: int, u, v):
    """Symmetric CSR of the undirected simple graph with edges ``{u[k], v[k]}``.

    Self loops and repeated edges are removed and every adjacency list is
    sorted. Returns ``(row_ptr int64[n+1], col_idx int32[2m])``.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = np.unique(a * n + b)
    a, b = key // n, key % n
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(src, minlength=n))
    return row_ptr, dst.astype(np.int32)


def _distinct_pairs(rng, s: int, k: int):
    """``k`` distinct unordered pairs of distinct integers in ``[0, s)``."""
    if k <= 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    have = np.zeros(0, dtype=np.int64)
    while have.size < k:
        need = k - have.size
        a = rng.integers(0, s, size=2 * need + 16)
        b = rng.integers(0, s, size=2 * need + 16)
        ok = a != b
        lo, hi = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        have = np.unique(np.concatenate([have, lo * s + hi]))
    pick = rng.permutation(have.size)[:k]
    key = have[pick]
    return key // s, key % s


def planted_partition(n_comm: int = 10, size: int = 100, p_in: float = 0.1,
                      p_out: float = 0.002, seed: int = 0):
    """Planted-partition graph: ``n_comm`` communities of ``size`` nodes.

    Returns ``(row_ptr, col_idx, truth)`` where ``truth[v]`` is the planted
    community of node ``v``; node ids are randomly permuted.
    """
    rng = np.random.default_rng(seed)
    n = n_comm * size
    us, vs = [], []
    pairs_in = size * (size - 1) // 2
    for c in range(n_comm):
        k = int(rng.binomial(pairs_in, p_in))
        a, b = _distinct_pairs(rng, size, k)
        us.append(a + c * size)
        vs.append(b + c * size)
    pairs_out = n * (n - 1) // 2 - n_comm * pairs_in
    k_out = int(rng.binomial(pairs_out, p_out))
    got_u = np.zeros(0, np.int64)
    got_v = np.zeros(0, np.int64)
    while got_u.size < k_out:
        need = k_out - got_u.size
        a = rng.integers(0, n, size=2 * need + 16)
        b = rng.integers(0, n, size=2 * need + 16)
        ok = (a // size) != (b // size)
        lo, hi = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        key = np.unique(np.concatenate([got_u * n + got_v, lo * n + hi]))
        got_u, got_v = key // n, key % n
    pick = rng.permutation(got_u.size)[:k_out]
    us.append(got_u[pick])
    vs.append(got_v[pick])
    perm = rng.permutation(n)  # node id relabelling
    u = perm[np.concatenate(us)]
    v = perm[np.concatenate(vs)]
    truth = np.empty(n, dtype=np.int32)
    truth[perm] = np.repeat(np.arange(n_comm, dtype=np.int32), size)
    row_ptr, col_idx = csr_from_edges(n, u, v)
    return row_ptr, col_idx, truth


def _powerlaw_mean(xmin: float, xmax: float, tau: float) -> float:
    if abs(tau - 1.0) < 1e-12:
        return (xmax - xmin) / math.log(xmax / xmin)
    if abs(tau - 2.0) < 1e-12:
        return math.log(xmax / xmin) / (1.0 / xmin - 1.0 / xmax)
    return ((1 - tau) / (2 - tau) * (xmax ** (2 - tau) - xmin ** (2 - tau))
            / (xmax ** (1 - tau) - xmin ** (1 - tau)))


def _powerlaw_sample(rng, size: int, xmin: float, xmax: float, tau: float):
    """Inverse-CDF samples of the density ``~ x^-tau`` on ``[xmin, xmax]``."""
    r = rng.random(size)
    if abs(tau - 1.0) < 1e-12:
        return xmin * (xmax / xmin) ** r
    e = 1.0 - tau
    return (xmin ** e + r * (xmax ** e - xmin ** e)) ** (1.0 / e)


def _solve_xmin(mean: float, xmax: float, tau: float) -> float:
    lo, hi = 1.0, float(xmax)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _powerlaw_mean(mid, xmax, tau) < mean:
            lo = mid
        else:
            hi = mid
    return lo


def _accept(accepted, a, b, n):
    """Merge candidate edges ``{a[k], b[k]}`` into the sorted key array.

    A candidate is rejected (``bad[k]``) when it is a self loop, repeats an
    accepted edge, or repeats an earlier candidate of the same batch.
    """
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = lo * n + hi
    bad = lo == hi
    if accepted.size:
        at = np.searchsorted(accepted, key)
        at = np.minimum(at, accepted.size - 1)
        bad |= accepted[at] == key
    _, first = np.unique(key, return_index=True)
    dup = np.ones(key.size, dtype=bool)
    dup[first] = False
    bad |= dup
    good = np.sort(key[~bad])
    merged = np.concatenate([accepted, good])
    merged.sort(kind="stable")  # two sorted runs: merged in linear time
    return merged, bad


def lfr_style(n: int, avg_deg: float, max_deg: int, mu: float,
              tau1: float = 2.0, tau2: float = 1.0, cmin: int = 20,
              cmax: int = 100, seed: int = 0):
    """LFR-style benchmark graph (see module docstring).

    Returns ``(row_ptr, col_idx, truth)``.
    """
    rng = np.random.default_rng(seed)
    kmin = _solve_xmin(avg_deg, max_deg, tau1)
    deg = np.rint(_powerlaw_sample(rng, n, kmin, max_deg, tau1)).astype(np.int64)
    deg = np.clip(deg, 1, max_deg)

    sizes = []
    total = 0
    while total < n:
        s = int(np.rint(_powerlaw_sample(rng, 1, cmin, cmax, tau2)[0]))
        sizes.append(s)
        total += s
    sizes = np.array(sizes, dtype=np.int64)
    excess = int(total - n)
    sizes[-1] -= excess
    if sizes[-1] < cmin and sizes.size > 1:
        spare = int(sizes[-1])
        sizes = sizes[:-1]
        bump = rng.choice(sizes.size, size=spare, replace=True)
        np.add.at(sizes, bump, 1)
    n_comm = sizes.size
    member = rng.permutation(np.repeat(np.arange(n_comm, dtype=np.int64), sizes))

    kin = np.rint((1.0 - mu) * deg).astype(np.int64)
    kin = np.minimum(kin, sizes[member] - 1)
    kout = deg - kin

    # Internal wiring: stubs grouped by community and paired in random order;
    # stubs of self loops and repeated edges go back to the pool for a few
    # more rounds, then are dropped.
    accepted = np.zeros(0, dtype=np.int64)
    pool = np.repeat(np.arange(n, dtype=np.int64), kin)
    for _ in range(6):
        if pool.size < 2:
            break
        comm = member[pool]
        tag = (comm << 32) | rng.integers(0, 1 << 32, size=pool.size, dtype=np.int64)
        order = np.argsort(tag)
        pool, comm = pool[order], comm[order]
        counts = np.bincount(comm, minlength=n_comm)
        starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
        pos = np.arange(pool.size) - starts[comm]
        first = (pos % 2 == 0) & (pos + 1 < counts[comm])
        idx = np.nonzero(first)[0]
        a, b = pool[idx], pool[idx + 1]
        accepted, bad = _accept(accepted, a, b, n)
        paired = np.zeros(pool.size, dtype=bool)
        paired[idx] = True
        paired[idx + 1] = True
        pool = np.concatenate([pool[~paired], a[bad], b[bad]])

    # External wiring: all outside stubs paired at random; pairs that land in
    # one community, self loops and repeats are re-paired for a few rounds.
    ext = np.repeat(np.arange(n, dtype=np.int64), kout)
    for _ in range(6):
        if ext.size < 2:
            break
        ext = rng.permutation(ext)
        if ext.size % 2:
            ext = ext[:-1]
        a, b = ext[0::2], ext[1::2]
        same = member[a] == member[b]
        accepted_x, bad = _accept(accepted, a[~same], b[~same], n)
        accepted = accepted_x
        a2, b2 = a[~same], b[~same]
        ext = np.concatenate([a[same], b[same], a2[bad], b2[bad]])
    u, v = accepted // n, accepted % n
    row_ptr, col_idx = csr_from_edges(n, u, v)
    return row_ptr, col_idx, member.astype(np.int32)


def random_labels(n: int, count: int, seed: int, n_distinct: int | None = None):
    """``count`` label vectors of length ``n`` (int32, row per individual).

    Labels are uniform in ``[0, n)``; with ``n_distinct`` they are drawn from a
    random set of ``n_distinct`` ids in ``[0, n)`` (few large communities).
    """
    rng = np.random.default_rng(seed)
    if n_distinct is None:
        return rng.integers(0, n, size=(count, n), dtype=np.int64).astype(np.int32)
    ids = rng.choice(n, size=min(n_distinct, n), replace=False)
    return ids[rng.integers(0, ids.size, size=(count, n))].astype(np.int32)


def batch_instances(count: int = 64, seed: int = 0):
    """Many uneven detection jobs: n log-uniform in [1e3, 5e4], average degree
    uniform in [10, 30], mixing mu uniform in [0.2, 0.5]; even-numbered jobs are
    planted-partition graphs (communities of 20-100 nodes), odd ones
    LFR-style graphs (maximum degree 2.5x the average). Returns a list of
    (row_ptr, col_idx, truth, description)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(1e3), math.log(5e4)))))
        d = float(rng.uniform(10, 30))
        mu = float(rng.uniform(0.2, 0.5))
        s = int(rng.integers(0, 1 << 31))
        if k % 2 == 0:
            size = int(rng.integers(20, 101))
            n_comm = max(2, n // size)
            nn = n_comm * size
            p_in = min(1.0, (1 - mu) * d / (size - 1))
            p_out = mu * d / (nn - size)
            rp, ci, tr = planted_partition(n_comm, size, p_in, p_out, seed=s)
            desc = f"planted n={nn} d={d:.1f} mu={mu:.2f}"
        else:
            rp, ci, tr = lfr_style(n, d, int(round(2.5 * d)), mu, seed=s)
            desc = f"lfr n={n} d={d:.1f} mu={mu:.2f}"
        out.append((rp, ci, tr, desc))
    return out


def serving_pool(count: int = 12, seed: int = 0, n_min: float = 1e3, n_max: float = 1e6):
    """Graphs for a request stream: n log-spaced in [n_min, n_max], LFR-style
    (average degree 16, maximum 200, communities 20-2000), mixing mu uniform
    in [0.1, 0.6]. Returns a list of (row_ptr, col_idx, description)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(math.log(n_min) + k * (math.log(n_max) - math.log(n_min)) / max(1, count - 1))))
        mu = float(rng.uniform(0.1, 0.6))
        rp, ci, _ = lfr_style(n, 16, 200 if n >= 20_000 else 50, mu, cmin=20,
                              cmax=2000 if n >= 20_000 else 100, seed=int(rng.integers(0, 1 << 31)))
        out.append((rp, ci, f"lfr n={n} mu={mu:.2f}"))
    return out


# Named workloads: shapes of the paper's experiments (Sec. 5.2, Table of
# parameters: N_p = 100, G = 100, C_P = 0.8, M_P = 0.2, E_S = 4).
WORKLOADS = {
    "planted-1k": dict(kind="planted", n_comm=10, size=100, p_in=0.1, p_out=0.002),
    "lfr-40k": dict(kind="lfr", n=40_000, avg_deg=20, max_deg=50, mu=0.3,
                    tau1=2.0, tau2=1.0, cmin=20, cmax=100),
    "lfr-1m": dict(kind="lfr", n=1_000_000, avg_deg=16, max_deg=200, mu=0.3,
                   tau1=2.0, tau2=1.0, cmin=20, cmax=2000),
}


def workload(name: str, seed: int = 0, **overrides):
    """Build the named workload graph; returns ``(row_ptr, col_idx, truth)``."""
    spec = dict(WORKLOADS[name])
    spec.update(overrides)
    kind = spec.pop("kind")
    if kind == "planted":
        return planted_partition(seed=seed, **spec)
    return lfr_style(seed=seed, **spec)
