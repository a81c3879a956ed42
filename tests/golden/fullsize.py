"""Digests of full-size results, for parity checks whose expected values are
too large to store: the per-seed table (seed_i, seed_j, count) as a multiset
hash, the accepted track list as SHA-256 of its tuples in acceptance order,
and the grain input as SHA-256 of its bytes (so that a test can tell when the
input generator drew different grains on another platform).

This module serialises and hashes; it holds none of the method's arithmetic.
"""
from __future__ import annotations

import hashlib

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014), elementwise on uint64."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def seed_keys(lo, hi, count):
    """One uint64 per seed record: lo | hi << 21 | count << 42 (each below 2^21)."""
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    count = np.asarray(count, dtype=np.int64)
    if lo.size and (lo.min() < 0 or hi.min() < 0 or count.min() < 0
                    or max(lo.max(), hi.max(), count.max()) >= (1 << 21)):
        raise ValueError("seed record field outside [0, 2^21)")
    return (lo | (hi << 21) | (count << 42)).astype(np.uint64)


def seed_digest(lo, hi, count, chunk=1 << 24):
    """(number of records, order-independent hash of the record multiset as hex)."""
    n = int(np.asarray(lo).shape[0])
    acc = np.uint64(0)
    for s in range(0, n, chunk):
        h = _splitmix64(seed_keys(lo[s:s + chunk], hi[s:s + chunk], count[s:s + chunk]))
        with np.errstate(over="ignore"):
            acc = np.uint64(acc + np.sum(h, dtype=np.uint64))
    return n, f"{int(acc):016x}"


def seed_digest_by_group(group, lo, hi, count, n_groups):
    """Per-group seed digests: (counts int64[n_groups], hashes as hex strings)."""
    group = np.asarray(group, dtype=np.int64)
    h = _splitmix64(seed_keys(lo, hi, count))
    order = np.argsort(group, kind="stable")
    g, h = group[order], h[order]
    starts = np.searchsorted(g, np.arange(n_groups + 1))
    counts = np.diff(starts)
    out = []
    for k in range(n_groups):
        with np.errstate(over="ignore"):
            out.append(f"{int(np.sum(h[starts[k]:starts[k + 1]], dtype=np.uint64)):016x}")
    return counts, out


def track_digest(tuples):
    """SHA-256 of (lo, hi, nhits, n_members, members...) per track, in order."""
    m = hashlib.sha256()
    for lo, hi, nhits, members in tuples:
        rec = np.asarray([lo, hi, nhits, len(members), *members], dtype=np.int64)
        m.update(rec.tobytes())
    return m.hexdigest()


def input_digest(xyz):
    return hashlib.sha256(np.ascontiguousarray(xyz, dtype=np.int32).tobytes()).hexdigest()
