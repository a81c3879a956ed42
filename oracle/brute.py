"""Brute-force restatement of the method for tiny inputs (pure Python ints).

TEST INFRASTRUCTURE ONLY.  It re-derives Section 2 of the paper with triple
loops and no cell hash, sharing nothing with oracle.c, so that the oracle can
be pinned against an independent evaluation of the same definition:

* seeds: unordered pairs with seed_min^2 <= |d|^2 < seed_max^2, lo = the grain
  that comes first in lexicographic (x, y, z) order;
* count: grains k of the whole view with |(g_k - g_lo) x w|^2 <= r^2 |w|^2;
* candidates: count >= min_hits, visited by (count desc, lo key, hi key);
  each keeps its unused tube grains and is accepted iff >= min_hits remain;
* the single-pass association and the grain-count cut variants.

Cost is O(N^3); keep N at a few hundred.
"""
from __future__ import annotations

from fractions import Fraction


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def in_tube(g, a, w, r):
    c = _cross(_sub(g, a), w)
    return _dot(c, c) <= r * r * _dot(w, w)


def keeps_angle_cut(w, nhits, cut):
    """Grain-count cut of Section 3 (Fig. 9c): nhits >= base + slope * min(tan theta, tan_max),
    tan theta = |w_xy| / |w_z| (infinite for w_z = 0), with exact rational arithmetic."""
    base, slope, tan_max = cut
    txy = w[0] * w[0] + w[1] * w[1]
    if w[2] == 0 or Fraction(txy, w[2] * w[2]) >= tan_max * tan_max:
        bound = Fraction(slope * tan_max)
        return nhits >= base + bound
    # nhits - base >= slope * sqrt(txy) / |w_z|, compared squared (both sides >= 0)
    need = nhits - base
    return need >= 0 and need * need * w[2] * w[2] >= slope * slope * txy


def find(xyz, seed_min, seed_max, tube_r, min_hits, single_pass=False, cut=None):
    """Returns (seeds {(lo, hi): count}, tracks [(lo, hi, nhits, members tuple)]).

    single_pass: each grain goes to the first candidate (candidate order) whose
    tube holds it; a candidate is a track iff at least min_hits grains chose it.
    cut: (base, slope, tan_max) of the grain-count cut, applied to the tracks."""
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
    tubes = [[k for k in range(n) if in_tube(pts[k], pts[i], _sub(pts[j], pts[i]), tube_r)]
             for (i, j), _ in cands]
    tracks = []
    if single_pass:
        choice = [None] * n
        for ci, tube in enumerate(tubes):
            for k in tube:
                if choice[k] is None:
                    choice[k] = ci
        for ci, ((i, j), _) in enumerate(cands):
            mine = [k for k in tubes[ci] if choice[k] == ci]
            if len(mine) >= min_hits:
                tracks.append((i, j, len(mine), tuple(sorted(mine))))
    else:
        used = [False] * n
        for ci, ((i, j), _) in enumerate(cands):
            free = [k for k in tubes[ci] if not used[k]]
            if len(free) >= min_hits:
                for k in free:
                    used[k] = True
                tracks.append((i, j, len(free), tuple(sorted(free))))
    if cut is not None:
        tracks = [t for t in tracks if keeps_angle_cut(_sub(pts[t[1]], pts[t[0]]), t[2], cut)]
    return seeds, tracks
