"""The digests that stand in for full-size expected results (tests/golden/
fullsize.py), and the parallel drawing of the served workload's views, on the
CPU.  A digest must not depend on record order, must change when any single
field of any record changes, and must equal what the golden-value script
stores for the same oracle result."""
import os
import sys

import numpy as np
import pytest

from paper_1311_5334_gb300 import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
if GOLD not in sys.path:
    sys.path.insert(0, GOLD)
import fullsize  # noqa: E402


def _records(rng, n=5000, nmax=3000):
    lo = rng.integers(0, nmax, n)
    hi = rng.integers(0, nmax, n)
    cnt = rng.integers(2, 60, n)
    return lo, hi, cnt


def test_seed_digest_is_order_independent_and_chunked_alike():
    rng = np.random.default_rng(1)
    lo, hi, cnt = _records(rng)
    perm = rng.permutation(len(lo))
    a = fullsize.seed_digest(lo, hi, cnt)
    assert a == fullsize.seed_digest(lo[perm], hi[perm], cnt[perm])
    assert a == fullsize.seed_digest(lo, hi, cnt, chunk=7)
    assert a[0] == len(lo)


def test_seed_digest_sees_every_single_change():
    rng = np.random.default_rng(2)
    lo, hi, cnt = _records(rng, n=400)
    base = fullsize.seed_digest(lo, hi, cnt)[1]
    for k in range(0, 400, 37):
        for arr in (lo, hi, cnt):
            old = arr[k]
            arr[k] = old + 1
            assert fullsize.seed_digest(lo, hi, cnt)[1] != base
            arr[k] = old
    # a swapped pair (lo, hi) is a different record
    lo2, hi2 = lo.copy(), hi.copy()
    j = int(np.nonzero(lo != hi)[0][0])
    lo2[j], hi2[j] = hi[j], lo[j]
    assert fullsize.seed_digest(lo2, hi2, cnt)[1] != base
    # a missing and a duplicated record
    assert fullsize.seed_digest(lo[1:], hi[1:], cnt[1:])[1] != base
    assert fullsize.seed_digest(np.r_[lo, lo[:1]], np.r_[hi, hi[:1]], np.r_[cnt, cnt[:1]])[1] != base


def test_seed_digest_by_group_matches_per_group_digests():
    rng = np.random.default_rng(3)
    lo, hi, cnt = _records(rng)
    grp = rng.integers(0, 9, len(lo))
    counts, hashes = fullsize.seed_digest_by_group(grp, lo, hi, cnt, 10)
    for g in range(10):
        m = grp == g
        assert (int(counts[g]), hashes[g]) == fullsize.seed_digest(lo[m], hi[m], cnt[m])


def test_seed_digest_rejects_fields_beyond_21_bits():
    with pytest.raises(ValueError):
        fullsize.seed_digest(np.array([1 << 21]), np.array([0]), np.array([3]))


def test_track_digest_is_order_and_content_sensitive():
    t = [(3, 9, 8, (1, 3, 9, 11, 12, 14, 15, 20)), (4, 7, 8, tuple(range(30, 38)))]
    d = fullsize.track_digest(t)
    assert d == fullsize.track_digest(list(t))
    assert d != fullsize.track_digest(t[::-1])
    assert d != fullsize.track_digest([t[0], (4, 7, 8, tuple(range(31, 39)))])
    assert d != fullsize.track_digest([t[0]])


def test_golden_record_of_a_small_view_matches_the_oracle(oracle_mod):
    import importlib.util
    spec = importlib.util.spec_from_file_location("mkd", os.path.join(GOLD, "make_fullsize_digests.py"))
    mkd = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mkd)
    v = synth.make_view(5, n_fog=400, n_through=5)
    p = synth.params(v.extent)
    rec = mkd.view_record(v, p, 0)
    o = oracle_mod.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
    try:
        tr, (slo, shi, scnt) = o.find_tracks(keep_seeds=True)
    finally:
        o.close()
    assert rec["n_seeds"] == len(slo) and rec["n_tracks"] == len(tr)
    assert rec["seed_hash"] == fullsize.seed_digest(slo, shi, scnt)[1]
    assert rec["tracks_sha256"] == fullsize.track_digest(tr.as_tuples())
    assert rec["input_sha256"] == fullsize.input_digest(v.xyz)


def test_served_views_drawn_in_parallel_equal_the_batched_generator():
    import bench
    pool = bench.served_views_pool(24, seed=4)
    ref = synth.batched(n_views=24, seed=4)
    assert len(pool) == 24
    assert all(np.array_equal(a, v.xyz) for a, v in zip(pool, ref))
