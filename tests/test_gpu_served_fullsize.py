"""The served configuration at its own sizes: the first 256 views of the
served stream (the batched size law, 2k-50k grains, seed 4) arrive as a
Poisson process at 2,000 views/s into a server with the 20 GB budget, and
every view's complete track list (seed pair, nhits, members, acceptance
order) must equal the oracle's.  The expected SHA-256 per view was written by
tests/golden/make_fullsize_digests.py, which calls only the oracle (Section 2,
Fig. 4); a view the generator draws differently on this platform is evaluated
by the oracle here instead."""
import json
import os
import sys
import threading
import time

import pytest

from paper_1311_5334_gb300 import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
if GOLD not in sys.path:
    sys.path.insert(0, GOLD)
import fullsize  # noqa: E402

pytestmark = pytest.mark.gpu


def expected_digest(oracle_mod, gold, v, p):
    if gold["input_sha256"] == fullsize.input_digest(v.xyz):
        return gold["tracks_sha256"], gold["n_tracks"]
    o = oracle_mod.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
    try:
        t = o.find_tracks().as_tuples()
    finally:
        o.close()
    return fullsize.track_digest(t), len(t)


def test_served_stream_matches_the_oracle(oracle_mod):
    from paper_1311_5334_gb300 import et
    with open(os.path.join(GOLD, "fullsize_served_seed4.json")) as f:
        gold = json.load(f)["views"]
    views = synth.batched(n_views=256, seed=4)
    p = synth.params(views[0].extent)
    budget = 20 << 30
    arrivals = synth.poisson_arrivals(len(views), 2000.0, seed=4)
    got = {}
    with et.Context(0) as ctx, ctx.server(p, budget, max_batch_views=256) as srv:
        t0 = time.monotonic() + 0.02
        busy = [0]

        def producer():
            for i, v in enumerate(views):
                wait = t0 + arrivals[i] - time.monotonic()
                if wait > 0:
                    time.sleep(wait)
                while srv.submit(v.xyz, tag=i) == et.BUSY:
                    busy[0] += 1
                    time.sleep(1e-4)

        th = threading.Thread(target=producer, daemon=True)
        th.start()
        deadline = time.monotonic() + 300
        while len(got) < len(views) and time.monotonic() < deadline:
            for r in srv.poll(max_results=256, timeout_us=50_000):
                assert r.status == et.OK, (r.tag, r.status)
                assert r.t_submit_ns <= r.t_admit_ns <= r.t_done_ns
                got[int(r.tag)] = srv.fetch(r.tag)
        th.join()
        st = srv.stats()
    assert sorted(got) == list(range(len(views)))
    assert 0 < st["peak_device_bytes"] <= budget and st["views_done"] == len(views)
    for k, v in enumerate(views):
        tracks, members = got[k]
        digest, n_tracks = expected_digest(oracle_mod, gold[k], v, p)
        t = et.track_tuples(tracks, members)
        assert len(t) == n_tracks and fullsize.track_digest(t) == digest, f"served view {k} ({v.n} grains)"
