"""The batched workload at full size (256 views of 300x300x50 um, seed 3) in
the launch configuration bench.py times: autotuned cells, CUDA-graph replay.
Every view's tracks are labelled with their view and the offsets are
consistent, and sampled views -- the three largest (the most seeds) and three
drawn at random -- equal the oracle's track lists exactly."""
import numpy as np
import pytest

from paper_1311_5334_gb300 import synth

pytestmark = pytest.mark.gpu


def test_full_batched_workload_sampled_views(oracle_mod):
    from paper_1311_5334_gb300 import et
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
        finally:
            b.close()
    assert len(voff) == 257 and voff[0] == 0 and voff[-1] == len(tracks) == st["n_tracks"]
    assert np.all(np.diff(voff) >= 0)
    for k in range(256):
        assert np.all(tracks["view"][voff[k]:voff[k + 1]] == k)
    sizes = np.array([v.n for v in views])
    rng = np.random.default_rng(7)
    pick = sorted(set(np.argsort(sizes)[-3:].tolist()) | set(rng.choice(256, 3, replace=False).tolist()))
    for k in pick:
        v = views[k]
        o = oracle_mod.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
        try:
            want = o.find_tracks().as_tuples()
        finally:
            o.close()
        got = et.track_tuples(tracks[voff[k]:voff[k + 1]], members)
        assert got == want, f"view {k} ({v.n} grains)"
