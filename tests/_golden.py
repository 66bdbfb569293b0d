"""Reader for the small text fixtures under tests/golden (paper examples)."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            out[key] = rest.strip()
    return out


def graph(d):
    """(row_ptr, col_idx) of the fixture's 1-based edge list, as 0-based CSR."""
    n = int(d["nodes"])
    adj = [[] for _ in range(n)]
    for e in d["edges"].split():
        a, b = (int(x) - 1 for x in e.split("-"))
        adj[a].append(b)
        adj[b].append(a)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for v in range(n):
        row_ptr[v + 1] = row_ptr[v] + len(adj[v])
    col_idx = np.array([u for v in range(n) for u in sorted(adj[v])], dtype=np.int32)
    return row_ptr, col_idx


def ints(s):
    return np.array([int(x) for x in s.split()], dtype=np.int32)


def frac(s):
    return Fraction(s)
