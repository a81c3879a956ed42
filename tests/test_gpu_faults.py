"""Failure handling without faulting the GPU: bounded device waits that run
out, and the served loop's back-pressure and memory budget.

The tuning knob wait_polls makes every bounded device-side wait (the grid
barriers of the association, the sorts and the scans; the sorts' look-back)
give up after that many polls.  A run with wait_polls = 1 must end with ET_ERR_TIMEOUT, a status the
host reads (no trap, no hang, the context stays usable), and the next run on
the same batch with the default limit must equal the oracle.

The served loop answers ET_ERR_BUSY when its pending queue is full or a view
alone exceeds the memory budget; views it admits must still produce the
oracle's tracks, and the device memory its two micro-batches hold together
must stay within the budget."""
import numpy as np
import pytest

from paper_1311_5334_gb300 import synth

pytestmark = pytest.mark.gpu


def oracle_tuples(oracle_mod, v, p):
    o = oracle_mod.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
    try:
        return o.find_tracks().as_tuples()
    finally:
        o.close()


def timeout_then_rerun(et, v, p, cell=(0, 0, 0)):
    """Runs with wait_polls = 1 until a run times out (at most 3 tries), then
    once with the default limit on the same batch; returns (timeouts, tuples, stats)."""
    with et.Context(0) as ctx:
        b = et.Batch(ctx, p)
        try:
            timeouts = 0
            for _ in range(3):
                b.set_tuning(cell=cell, wait_polls=1)
                b.load(v.xyz, [0, v.n])
                b.find()
                try:
                    b.fetch()
                except et.EtError as e:
                    assert e.status == et.TIMEOUT, e
                    timeouts += 1
                    break
            b.set_tuning(cell=cell)
            b.load(v.xyz, [0, v.n])
            b.find()
            tracks, members, _ = b.fetch()
            st = b.stats()
        finally:
            b.close()
    return timeouts, et.track_tuples(tracks, members), st


def test_association_barrier_wait_runs_out(oracle_mod):
    """A small view on 15 x 15 x 15 cells: every sort and scan fits one tile,
    so one block does it with no wait, and the association keeps more than
    one block (over 32 candidates).  The only device wait is the grid barrier
    between association rounds."""
    from paper_1311_5334_gb300 import et
    v = synth.make_view(31, n_fog=1000, n_through=10)
    p = synth.params(v.extent)
    cell = tuple(-(-e // 15) for e in v.extent)
    timeouts, got, st = timeout_then_rerun(et, v, p, cell)
    assert v.n < 2048 and 32 < st["n_candidates"] < 2048, (v.n, st["n_candidates"])
    assert timeouts == 1
    assert got == oracle_tuples(oracle_mod, v, p)


def test_sort_lookback_wait_runs_out(oracle_mod):
    """The dense view (15 tiles in the first sort): a tile's look-back on its
    predecessor, or a grid barrier between the sort's passes, gives up after
    one poll."""
    from paper_1311_5334_gb300 import et
    v = synth.dense()
    p = synth.params(v.extent)
    timeouts, got, _ = timeout_then_rerun(et, v, p)
    assert timeouts == 1
    assert got == oracle_tuples(oracle_mod, v, p)


def _drain(et, s, n_expected):
    got = {}
    for _ in range(4000):
        for r in s.poll(max_results=64, timeout_us=100000):
            assert r.status == et.OK, r.status
            assert r.t_submit_ns <= r.t_admit_ns <= r.t_done_ns
            got[r.tag] = s.fetch(r.tag)
        if len(got) == n_expected:
            break
    return got


def test_server_budget_below_two_micro_batches(oracle_mod):
    from paper_1311_5334_gb300 import et
    views = [v for v in synth.batched(n_views=48, seed=4) if v.n < 12000][:16]
    p = synth.params(views[0].extent)
    big = max(views, key=lambda v: v.n)
    with et.Context(0) as ctx:
        # device bytes of a micro-batch holding the largest view alone
        with ctx.server(p, mem_budget_bytes=64 << 30, max_batch_views=1) as s:
            assert s.submit(big.xyz, tag=1) == et.OK
            assert len(_drain(et, s, 1)) == 1
            one = s.stats()["peak_device_bytes"]
        assert one > 0
        budget = int(1.6 * one)   # one micro-batch of that view fits; two do not
        with ctx.server(p, mem_budget_bytes=budget, max_batch_views=8) as s:
            for k, v in enumerate(views):
                assert s.submit(v.xyz, tag=100 + k) == et.OK
            got = _drain(et, s, len(views))
            st = s.stats()
    assert len(got) == len(views)
    assert 0 < st["peak_device_bytes"] <= budget, (st, budget)
    assert st["views_done"] == len(views) and st["batches"] >= 2
    for k, v in enumerate(views):
        tracks, members = got[100 + k]
        assert et.track_tuples(tracks, members) == oracle_tuples(oracle_mod, v, p)


def test_server_busy_when_full_or_too_large(oracle_mod):
    from paper_1311_5334_gb300 import et
    views = [v for v in synth.batched(n_views=40, seed=4) if v.n < 12000][:24]
    p = synth.params(views[0].extent)
    with et.Context(0) as ctx:
        with ctx.server(p, mem_budget_bytes=8 << 20, max_batch_views=8) as s:
            # a view that needs more than 8 MB of device memory on its own
            assert s.submit(views[0].xyz, tag=1) == et.BUSY
            assert s.stats()["busy_rejections"] == 1
        with ctx.server(p, mem_budget_bytes=2 << 30, max_batch_views=8) as s:
            s.set_max_pending(2)
            admitted, busy = {}, 0
            for i in range(400):   # submits come faster than the worker drains the queue
                st = s.submit(views[i % len(views)].xyz, tag=200 + i)
                if st == et.BUSY:
                    busy += 1
                    if busy >= 3:
                        break
                else:
                    assert st == et.OK
                    admitted[200 + i] = i % len(views)
            got = _drain(et, s, len(admitted))
            stats = s.stats()
    assert busy >= 1 and stats["busy_rejections"] == busy
    assert sorted(got) == sorted(admitted)
    want = {}
    for tag, k in admitted.items():
        if k not in want:
            want[k] = oracle_tuples(oracle_mod, views[k], p)
        tracks, members = got[tag]
        assert et.track_tuples(tracks, members) == want[k]
