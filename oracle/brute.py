"""Brute-force restatement of the method for tiny inputs (pure Python ints).

TEST INFRASTRUCTURE ONLY.  It re-derives Section 2 of the paper with triple
loops and no cell hash, sharing nothing with oracle.c, so that the oracle can
be pinned against an independent evaluation of the same definition:

* seeds: unordered pairs with seed_min^2 <= |d|^2 < seed_max^2, lo = the grain
  that comes first in lexicographic (x, y, z) order;
* count: grains k of the whole view with |(g_k - g_lo) x w|^2 <= r^2 |w|^2;
* candidates: count >= min_hits, visited by (count desc, lo key, hi key);
  each keeps its unused tube grains and is accepted iff >= min_hits remain.

Cost is O(N^3); keep N at a few hundred.
"""
from __future__ import annotations


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def in_tube(g, a, w, r):
    c = _cross(_sub(g, a), w)
    return _dot(c, c) <= r * r * _dot(w, w)


def find(xyz, seed_min, seed_max, tube_r, min_hits):
    """Returns (seeds {(lo, hi): count}, tracks [(lo, hi, nhits, members tuple)])."""
    pts = [tuple(int(v) for v in p) for p in xyz]
    n = len(pts)
    seeds = {}
    for i in range(n):
        for j in range(n):
            if not pts[i] < pts[j]:           # lexicographic order of the coordinates
                continue
            d = _sub(pts[j], pts[i])
            dd = _dot(d, d)
            if seed_min * seed_min <= dd < seed_max * seed_max:
                seeds[(i, j)] = sum(1 for k in range(n) if in_tube(pts[k], pts[i], d, tube_r))
    cands = [(s, c) for s, c in seeds.items() if c >= min_hits]
    cands.sort(key=lambda sc: (-sc[1], pts[sc[0][0]], pts[sc[0][1]]))
    used = [False] * n
    tracks = []
    for (i, j), _ in cands:
        w = _sub(pts[j], pts[i])
        free = [k for k in range(n) if in_tube(pts[k], pts[i], w, tube_r) and not used[k]]
        if len(free) >= min_hits:
            for k in free:
                used[k] = True
            tracks.append((i, j, len(free), tuple(sorted(free))))
    return seeds, tracks
