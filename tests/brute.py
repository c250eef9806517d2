"""Independent brute-force formulations used to pin the oracle.

Each helper restates a definition in a different form from the oracle's code
(flat sets instead of recursion, exact rationals instead of FP64, string bit
interleaving instead of shifts), so that a slip in either shows up as a
mismatch.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

TWO32 = 1 << 32


def quantize_exact(v: float, box: float = 1.0) -> int:
    """floor(frac(v/box) * 2^32) with the FP64 quotient and exact rationals after it."""
    t = Fraction(v / box)
    frac = t - (t.numerator // t.denominator)          # in [0, 1) for either sign
    q = (frac * TWO32).numerator // (frac * TWO32).denominator
    return int(q)


def morton_string(x: int, y: int, z: int) -> int:
    """Interleave the top 21 bits of x, y, z as binary strings, x first."""
    bx, by, bz = (format(v, "032b")[:21] for v in (x, y, z))
    return int("".join(a + b + c for a, b, c in zip(bx, by, bz)), 2)


def node_set(skey: np.ndarray, leaf_max: int = 1):
    """All octree nodes as (level, begin, end) from the flat definition:
    the root, plus every cell (level >= 1) holding more than leaf_max sorted
    particles whose particles are not all in one child octant (or level 21)."""
    n = skey.shape[0]
    skey = skey.astype(np.uint64)
    out = {(0, 0, n)}
    for lev in range(1, 22):
        pre = skey >> np.uint64(3 * (21 - lev))
        starts = np.flatnonzero(np.r_[True, pre[1:] != pre[:-1]])
        ends = np.r_[starts[1:], n]
        for b, e in zip(starts, ends):
            if e - b <= leaf_max:
                continue
            if lev < 21:
                sub = skey[b:e] >> np.uint64(3 * (21 - lev - 1))
                if sub[0] == sub[-1]:
                    continue
            out.add((lev, int(b), int(e)))
    return out


def deepest_containing(nodes, lo, hi):
    """Among nodes (level, b, e) containing [lo, hi) pick the deepest."""
    best = None
    for (lev, b, e) in nodes:
        if b <= lo and hi <= e and (best is None or lev > best[0]):
            best = (lev, b, e)
    return best


def groups_flat(nodes, n: int, G: int):
    """Groups from the flat reading: each particle's frontier node is the
    deepest node with more than G particles containing it (the root if none).
    When the frontier node holds at most 8G particles, maximal runs of
    consecutive particles with the same frontier node are cut into pieces of
    G; otherwise the particles of each child of the frontier node (a node of
    at most G particles, or a single particle) form one group."""
    big = [nd for nd in nodes if nd[2] - nd[1] > G or nd[0] == 0]
    big.sort(key=lambda t: (t[1], t[0]))
    front, unit = [], []
    for i in range(n):
        f = deepest_containing(big, i, i + 1)
        front.append(f)
        # the child of f containing i: the shallowest node below f containing i
        below = [nd for nd in nodes if nd[0] > f[0] and nd[1] <= i < nd[2]
                 and f[1] <= nd[1] and nd[2] <= f[2]]
        unit.append(min(below, key=lambda t: t[0]) if below else ("p", i))
    groups = []
    i = 0
    while i < n:
        j = i
        if front[i][2] - front[i][1] <= 8 * G:
            while j < n and front[j] == front[i]:
                j += 1
            for s in range(i, j, G):
                groups.append((s, min(s + G, j)))
        else:
            while j < n and front[j] == front[i] and unit[j] == unit[i]:
                j += 1
            groups.append((i, j))
        i = j
    return groups


def exact_com(xs, ms):
    """Exact rational centre of mass of integer coordinates with FP64 masses."""
    M = sum(Fraction(m) for m in ms)
    return [sum(Fraction(m) * int(x) for m, x in zip(ms, col)) / M for col in xs]


def min_image_int(a: np.ndarray) -> np.ndarray:
    """Two's-complement 32-bit wrap of integer differences."""
    a = np.asarray(a, dtype=np.int64)
    return ((a + (1 << 31)) % (1 << 32)) - (1 << 31)
