"""The batched workload at full size (256 views of 300x300x50 um, seed 3) in
the launch configuration bench.py times: autotuned cells, CUDA-graph replay.

Every view's complete result is compared with the oracle's: the per-seed
table (seed_i, seed_j, count) of all 2.8e8 seeds as a multiset digest per
view, and the full track list (seed pair, nhits, members, in acceptance
order) as a SHA-256 per view, and the FP32 fit of three views with the
oracle's FP64 fit; under the two association variants (single pass, and the
grain-count cut) the complete track lists of all views as well.  The expected digests were written by
tests/golden/make_fullsize_digests.py, which calls only the oracle (Section 2,
Fig. 4 of the paper).  If the input generator draws a view differently on this
platform (its input digest differs), that view's expected values are computed
here by the oracle instead.  On a mismatch the first differing track is
reported."""
import json
import os
import sys

import numpy as np
import pytest

from paper_1311_5334_gb300 import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
if GOLD not in sys.path:
    sys.path.insert(0, GOLD)
import fullsize  # noqa: E402

pytestmark = pytest.mark.gpu


def oracle_record(oracle_mod, v, p):
    """The record make_fullsize_digests.py stores, computed now."""
    o = oracle_mod.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
    try:
        tr, (slo, shi, scnt) = o.find_tracks(keep_seeds=True)
    finally:
        o.close()
    n, sd = fullsize.seed_digest(slo, shi, scnt)
    return {"input_sha256": fullsize.input_digest(v.xyz), "n_seeds": n, "seed_hash": sd,
            "n_hits": int(scnt.astype(np.int64).sum()), "n_candidates": int(tr.n_cand),
            "n_tracks": len(tr), "tracks_sha256": fullsize.track_digest(tr.as_tuples())}


def expected_record(oracle_mod, gold, v, p):
    if gold["input_sha256"] == fullsize.input_digest(v.xyz):
        return gold
    return oracle_record(oracle_mod, v, p)


def first_difference(oracle_mod, v, p, got):
    o = oracle_mod.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
    try:
        want = o.find_tracks().as_tuples()
    finally:
        o.close()
    for k, (a, b) in enumerate(zip(got, want)):
        if a != b:
            return f"track {k}: got {a[:3]} ({len(a[3])} members), oracle {b[:3]} ({len(b[3])} members)"
    return f"{len(got)} tracks, oracle {len(want)}"


def test_full_batched_workload_all_views(oracle_mod):
    from paper_1311_5334_gb300 import et
    with open(os.path.join(GOLD, "fullsize_batched_seed3.json")) as f:
        gold = json.load(f)["views"]
    views = synth.batched(n_views=256, seed=3)
    xyz, offs = synth.concat(views)
    p = synth.params(views[0].extent)
    with et.Context(0) as ctx:
        b = et.Batch(ctx, p)
        try:
            b.load(xyz, offs)
            b.autotune()
            for _ in range(2):   # capture, then replay
                b.load(xyz, offs)
                b.find(use_graph=True)
            tracks, members, voff = b.fetch()
            st = b.stats()
            si, sj, sc = b.seed_counts()   # the same tuning, with per-seed records
        finally:
            b.close()
    assert len(voff) == 257 and voff[0] == 0 and voff[-1] == len(tracks) == st["n_tracks"]
    assert np.all(np.diff(voff) >= 0)
    for k in range(256):
        assert np.all(tracks["view"][voff[k]:voff[k + 1]] == k)
    grp = np.searchsorted(offs, si, side="right") - 1
    assert np.array_equal(grp, np.searchsorted(offs, sj, side="right") - 1), "a seed spans two views"
    base = offs[grp]
    n_seeds, seed_hash = fullsize.seed_digest_by_group(grp, si - base, sj - base, sc, 256)
    tot_seeds = tot_cand = tot_tracks = 0
    for k, v in enumerate(views):
        want = expected_record(oracle_mod, gold[k], v, p)
        assert (int(n_seeds[k]), seed_hash[k]) == (want["n_seeds"], want["seed_hash"]), \
            f"view {k} ({v.n} grains): per-seed table differs"
        got = et.track_tuples(tracks[voff[k]:voff[k + 1]], members)
        if fullsize.track_digest(got) != want["tracks_sha256"]:
            pytest.fail(f"view {k} ({v.n} grains): {first_difference(oracle_mod, v, p, got)}")
        tot_seeds += want["n_seeds"]
        tot_cand += want["n_candidates"]
        tot_tracks += want["n_tracks"]
    assert st["n_seeds"] == tot_seeds == len(si)
    assert st["n_candidates"] == tot_cand
    assert st["n_tracks"] == tot_tracks
    # the FP32 fit against the oracle's FP64 fit on the largest view and two others
    from tests.test_gpu_parity import check_fit
    sizes = np.array([v.n for v in views])
    rng = np.random.default_rng(7)
    for k in sorted({int(np.argmax(sizes))} | set(rng.choice(256, 2, replace=False).tolist())):
        v = views[k]
        o = oracle_mod.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
        try:
            want = o.find_tracks()
        finally:
            o.close()
        check_fit(tracks[voff[k]:voff[k + 1]], want)


@pytest.mark.parametrize("name", ["single_pass", "angle_cut_9_3_4"])
def test_full_batched_workload_variants(oracle_mod, name):
    """The association variants (single pass; sequential with the grain-count
    cut) on all 256 views: every view's complete track list against the
    oracle's digest in the same mode."""
    from paper_1311_5334_gb300 import et
    with open(os.path.join(GOLD, "fullsize_variants_seed3.json")) as f:
        gold = json.load(f)["variants"][name]
    views = synth.batched(n_views=256, seed=3)
    xyz, offs = synth.concat(views)
    p = synth.params(views[0].extent, flags=gold["flags"], cut=tuple(gold["cut"]))
    with et.Context(0) as ctx:
        b = et.Batch(ctx, p)
        try:
            b.load(xyz, offs)
            b.autotune()
            for _ in range(2):   # capture, then replay
                b.load(xyz, offs)
                b.find(use_graph=True)
            tracks, members, voff = b.fetch()
        finally:
            b.close()
    for k, v in enumerate(views):
        g = gold["views"][k]
        if g["input_sha256"] == fullsize.input_digest(v.xyz):
            want, n_want = g["tracks_sha256"], g["n_tracks"]
        else:
            o = oracle_mod.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"],
                                  flags=p["flags"], cut=p["cut"])
            try:
                t = o.find_tracks().as_tuples()
            finally:
                o.close()
            want, n_want = fullsize.track_digest(t), len(t)
        got = et.track_tuples(tracks[voff[k]:voff[k + 1]], members)
        assert len(got) == n_want and fullsize.track_digest(got) == want, f"{name}: view {k} ({v.n} grains)"
