"""GPU path vs the oracle, through the C ABI (libet.so).

Counts, candidate sets and track lists must be bit-identical; the FP32 fit is
compared with the FP64 oracle fit within the stated tolerance:
    |u32 - u64|_inf <= 1e-5,
    |c32 - c64|_inf <= 1e-5 * max(1, |c64|_inf),
    |t32 - t64|     <= 1e-5 * max(1, |t64|)   (tmin and tmax each),
for tracks whose scatter matrix is well conditioned (lambda1 >= 100 lambda2).
"""
import json
import os

import numpy as np
import pytest

from paper_1311_5334_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


@pytest.fixture(scope="module")
def et():
    from paper_1311_5334_gb300 import et as E
    E.lib()
    return E


@pytest.fixture(scope="module")
def ctx(et):
    c = et.Context(0)
    yield c
    c.close()


def run_view(et, ctx, xyz, params, cell=None, seeds=False, row_lists=0):
    v = et.View.create(ctx, xyz, params)
    try:
        if cell is not None or row_lists:
            v.set_tuning(cell if cell is not None else (0, 0, 0), row_lists=row_lists)
            v.load_host(xyz)
        v.find()
        tracks, members = v.fetch()
        st = v.stats()
        sc = v.seed_counts() if seeds else None
    finally:
        v.close()
    return tracks, members, st, sc


def oracle_run(O, xyz, params, keep_seeds=False):
    o = O.Oracle(xyz, params["extent"], params["seed_min"], params["seed_max"], params["tube_r"],
                 params["min_hits"])
    try:
        return o.find_tracks(keep_seeds=keep_seeds)
    finally:
        o.close()


def seed_table(lo, hi, cnt):
    order = np.lexsort((hi, lo))
    return np.stack([lo[order], hi[order], cnt[order]], axis=1)


def check_fit(tracks, want, tol=1e-5):
    assert len(tracks) == len(want)
    for k in range(len(want)):
        lam = want.lam[k]
        if lam[0] < 100 * max(lam[1], 1e-300):
            continue
        u32, u64 = tracks["u"][k].astype(np.float64), want.u[k]
        assert np.max(np.abs(u32 - u64)) <= tol, (k, u32, u64)
        c32, c64 = tracks["c"][k].astype(np.float64), want.c[k]
        assert np.max(np.abs(c32 - c64)) <= tol * max(1.0, np.max(np.abs(c64))), (k, c32, c64)
        for f, j in (("tmin", 0), ("tmax", 1)):
            t64 = want.t[k][j]
            assert abs(float(tracks[f][k]) - t64) <= tol * max(1.0, abs(t64)), (k, f, tracks[f][k], t64)


def assert_same(et, tracks, members, want):
    got = et.track_tuples(tracks, members)
    exp = want.as_tuples()
    assert len(got) == len(exp)
    assert got == exp


# ------------------------------------------------------------------ worked examples

def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_worked_examples(et, ctx, case):
    p = dict(extent=case["extent"], seed_min=case["seed_min"], seed_max=case["seed_max"],
             tube_r=case["tube_r"], min_hits=case["min_hits"])
    tracks, members, st, (si, sj, sc) = run_view(et, ctx, np.asarray(case["grains"]), p, seeds=True)
    want_seeds = sorted(tuple(s) for s in case["seeds"])
    assert sorted(zip(si.tolist(), sj.tolist(), sc.tolist())) == want_seeds
    got = et.track_tuples(tracks, members)
    assert got == [(a, b, n, tuple(m)) for a, b, n, m in case["tracks"]]


# ------------------------------------------------------------------ small random vs brute force

@pytest.mark.parametrize("seed", range(6))
def test_small_views_vs_brute_force(et, ctx, seed):
    from oracle import brute
    from tests.test_oracle_pins import _small_view
    rng = np.random.default_rng(100 + seed)
    extent = (1500, 1200, 400)
    xyz = _small_view(rng, extent, n_fog=60 + 20 * seed, tracks=3 + seed % 3, gap=37)
    smin, smax, r, h = [(40, 200, 6, 4), (0, 150, 10, 5), (60, 400, 3, 3), (40, 200, 0, 2),
                        (30, 250, 8, 6), (10, 120, 15, 4)][seed]
    bs, bt = brute.find(xyz, smin, smax, r, h)
    p = dict(extent=extent, seed_min=smin, seed_max=smax, tube_r=r, min_hits=h)
    for cell, rows in [(None, 0), ((97, 131, 53), 1), ((400, 400, 400), 1), ((17, 1200, 9), 1), ((1, 1, 1), 1),
                       ((97, 131, 53), 2), ((17, 1200, 9), 2), ((300, 11, 50), 2)]:
        tracks, members, st, (si, sj, sc) = run_view(et, ctx, xyz, p, cell=cell, seeds=True, row_lists=rows)
        assert {(int(a), int(b)): int(c) for a, b, c in zip(si, sj, sc)} == bs
        assert et.track_tuples(tracks, members) == bt


# ------------------------------------------------------------------ paper-shaped workloads

@pytest.mark.parametrize("workload", ["pr1", "dense"])
def test_workload_parity(et, ctx, oracle_mod, workload):
    v = synth.pr1() if workload == "pr1" else synth.dense()
    p = synth.params(v.extent)
    want, (olo, ohi, ocnt) = oracle_run(oracle_mod, v.xyz, p, keep_seeds=True)
    tracks, members, st, (si, sj, sc) = run_view(et, ctx, v.xyz, p, seeds=True)
    assert st["n_seeds"] == want.n_seeds
    assert np.array_equal(seed_table(si, sj, sc), seed_table(olo, ohi, ocnt))
    assert st["n_hits"] == int(ocnt.sum())
    assert st["n_candidates"] == want.n_cand
    assert_same(et, tracks, members, want)
    check_fit(tracks, want)


@pytest.mark.parametrize("cell,rows", [((150, 150, 150), 1), ((300, 300, 100), 1), ((600, 600, 600), 1),
                                       ((1000, 250, 125), 1), ((2000, 2000, 2000), 1), ((150, 600, 600), 2),
                                       ((1000, 250, 125), 2)])
def test_cell_size_invariance(et, ctx, oracle_mod, cell, rows):
    v = synth.dense()
    p = synth.params(v.extent)
    want = oracle_run(oracle_mod, v.xyz, p)
    tracks, members, st, _ = run_view(et, ctx, v.xyz, p, cell=cell, row_lists=rows)
    assert tuple(st["cell"]) == cell
    assert st["n_seeds"] == want.n_seeds
    assert_same(et, tracks, members, want)


def test_autotuner_keeps_results(et, ctx, oracle_mod):
    views = [v for v in synth.batched(n_views=12, seed=6) if v.n < 20000][:6]
    xyz, offs = synth.concat(views)
    p = synth.params(views[0].extent)
    b = et.Batch(ctx, p)
    try:
        b.load(xyz, offs)
        cell, ms = b.autotune(max_trials=4)
        assert all(c >= 16 for c in cell) and ms > 0
        b.find(use_graph=True)
        tracks, members, voff = b.fetch()
        assert tuple(b.stats()["cell"]) == tuple(cell)
        for k, v in enumerate(views):
            want = oracle_run(oracle_mod, v.xyz, p)
            assert et.track_tuples(tracks[voff[k]:voff[k + 1]], members) == want.as_tuples()
    finally:
        b.close()


@pytest.mark.parametrize("origins", [1, 2, 4])
def test_ticket_origins_keep_results(et, ctx, oracle_mod, origins):
    views = [v for v in synth.batched(n_views=8, seed=9) if v.n < 20000][:4] + [synth.pr1()]
    xyz, offs = synth.concat(views)
    p = synth.params(views[0].extent)
    b = et.Batch(ctx, p)
    try:
        b.set_tuning(ticket_origins=origins)
        b.load(xyz, offs)
        b.find(use_graph=True)
        tracks, members, voff = b.fetch()
        for k, v in enumerate(views):
            want = oracle_run(oracle_mod, v.xyz, p)
            assert et.track_tuples(tracks[voff[k]:voff[k + 1]], members) == want.as_tuples()
    finally:
        b.close()


def test_permutation_invariance(et, ctx):
    v = synth.pr1()
    p = synth.params(v.extent)
    rng = np.random.default_rng(4)
    perm = rng.permutation(v.n)
    t1, m1, _, _ = run_view(et, ctx, v.xyz, p)
    t2, m2, _, _ = run_view(et, ctx, v.xyz[perm], p)
    a = et.track_tuples(t1, m1)
    b = [(int(perm[i]), int(perm[j]), n, tuple(sorted(int(perm[x]) for x in mem)))
         for i, j, n, mem in et.track_tuples(t2, m2)]
    assert a == b
    assert np.array_equal(t1["u"], t2["u"]) and np.array_equal(t1["tmin"], t2["tmin"])


# ------------------------------------------------------------------ batched form

def test_batched_matches_oracle_per_view(et, ctx, oracle_mod):
    views = synth.batched(n_views=24, seed=3)
    views = [v for v in views if v.n < 20000][:16]
    xyz, offs = synth.concat(views)
    p = synth.params(views[0].extent)
    b = et.Batch(ctx, p)
    try:
        b.load(xyz, offs)
        for use_graph in (False, True, True):
            b.find(use_graph=use_graph)
            tracks, members, voff = b.fetch()
            for k, v in enumerate(views):
                want = oracle_run(oracle_mod, v.xyz, p)
                sub = tracks[voff[k]:voff[k + 1]]
                assert np.all(sub["view"] == k)
                assert et.track_tuples(sub, members) == want.as_tuples()
    finally:
        b.close()


@pytest.mark.parametrize("window", [1, 7, 64, 1000])
def test_association_windows(et, ctx, oracle_mod, window):
    # the association runs window by window over the key-sorted candidates;
    # tiny windows (many window boundaries) give the same tracks
    for v in (synth.pr1(), synth.dense()):
        p = synth.params(v.extent)
        want = oracle_run(oracle_mod, v.xyz, p)
        view = et.View.create(ctx, v.xyz, p)
        try:
            view.set_tuning((0, 0, 0), row_lists=0, assoc_window=window)
            view.load_host(v.xyz)
            view.find(use_graph=True)
            tracks, members = view.fetch()
            assert view.stats()["merge_rounds"] >= min(want.n_cand, 1000) // window
        finally:
            view.close()
        assert_same(et, tracks, members, want)


def test_graph_replay_follows_tuning_changes(et, ctx, oracle_mod):
    # a captured launch sequence must not outlive the cell grid it was captured for
    views = [v for v in synth.batched(n_views=12, seed=3) if v.n < 20000][:6]
    xyz, offs = synth.concat(views)
    p = synth.params(views[0].extent)
    want = [oracle_run(oracle_mod, v.xyz, p).as_tuples() for v in views]
    b = et.Batch(ctx, p)
    try:
        seen = set()
        for cell, rows in [((300, 300, 300), 1), ((152, 598, 598), 2), ((500, 200, 400), 1), ((300, 300, 300), 1)]:
            b.set_tuning(cell, row_lists=rows)
            b.load(xyz, offs)
            b.find(use_graph=False)
            b.sync()
            direct = b.stats()["n_tests"]   # tube tests depend on the cell grid
            b.find(use_graph=True)
            tracks, members, voff = b.fetch()
            assert b.stats()["n_tests"] == direct
            seen.add(direct)
            for k in range(len(views)):
                assert et.track_tuples(tracks[voff[k]:voff[k + 1]], members) == want[k]
        assert len(seen) == 3   # three different grids, three different test counts
    finally:
        b.close()


# ------------------------------------------------------------------ edge cases

def _p(extent=(1000, 1000, 1000), smin=10, smax=300, r=5, h=3):
    return dict(extent=extent, seed_min=smin, seed_max=smax, tube_r=r, min_hits=h)


def test_empty_and_tiny_views(et, ctx):
    for xyz in [np.zeros((0, 3)), np.array([[5, 5, 5]]), np.array([[5, 5, 5], [900, 900, 900]])]:
        tracks, members, st, _ = run_view(et, ctx, xyz, _p())
        assert len(tracks) == 0 and len(members) == 0 and st["n_seeds"] == 0
    tracks, members, st, (si, sj, sc) = run_view(et, ctx, np.array([[50, 5, 5], [5, 5, 5]]), _p(h=2), seeds=True)
    assert st["n_seeds"] == 1 and list(zip(si, sj, sc)) == [(1, 0, 2)]
    assert et.track_tuples(tracks, members) == [(1, 0, 2, (0, 1))]


def test_batch_with_empty_and_single_grain_views(et, ctx, oracle_mod):
    """Ragged batches: empty views and one-grain views between real ones, first
    and last, plain and replayed from a graph; offsets must stay consistent."""
    real = [v for v in synth.batched(n_views=12, seed=12) if v.n < 20000][:3]
    assert len(real) == 3
    one = np.array([[123, 456, 789]], dtype=np.int32)
    none = np.zeros((0, 3), dtype=np.int32)
    xyzs = [none, real[0].xyz, one, none, none, real[1].xyz, one, real[2].xyz, none]
    offs = np.concatenate([[0], np.cumsum([len(x) for x in xyzs])]).astype(np.int64)
    xyz = np.concatenate(xyzs).astype(np.int32)
    p = synth.params(real[0].extent)
    want = [oracle_run(oracle_mod, x, p).as_tuples() if len(x) > 1 else [] for x in xyzs]
    b = et.Batch(ctx, p)
    try:
        b.load(xyz, offs)
        for use_graph in (False, True, True):
            b.find(use_graph=use_graph)
            tracks, members, voff = b.fetch()
            assert len(voff) == len(xyzs) + 1 and voff[0] == 0 and voff[-1] == len(tracks)
            for k in range(len(xyzs)):
                assert et.track_tuples(tracks[voff[k]:voff[k + 1]], members) == want[k], k
    finally:
        b.close()


def test_long_collinear_line(et, ctx, oracle_mod):
    """4000 collinear grains: every seed holds all of them; one track."""
    n = 4000
    xyz = np.stack([np.arange(n) * 3 + 7, np.arange(n) * 2 + 11, np.full(n, 40)], axis=1)
    p = _p(extent=(20000, 20000, 100), smin=10, smax=60, r=0, h=5)
    tracks, members, st, _ = run_view(et, ctx, xyz, p)
    want = oracle_run(oracle_mod, xyz, p)
    assert len(want) == 1 and want.nhits[0] == n
    assert_same(et, tracks, members, want)


def test_clustered_view_forces_buffer_growth(et, ctx, oracle_mod):
    """All grains in 1 % of the volume: the uniform-density estimates of the
    seed/candidate buffers are far too small and the runtime must grow them."""
    rng = np.random.default_rng(21)
    pts = set()
    while len(pts) < 3000:
        pts.add(tuple(int(x) for x in rng.integers(0, 600, 3)))
    base = np.array(sorted(pts)) + np.array([1000, 1000, 200])
    line = np.stack([np.arange(80) * 7 + 1000, np.arange(80) * 5 + 1000, np.full(80, 500)], axis=1)
    xyz = np.unique(np.concatenate([base, line]), axis=0)
    xyz = xyz[rng.permutation(len(xyz))]
    p = _p(extent=(30000, 30000, 5000), smin=20, smax=200, r=6, h=6)
    want = oracle_run(oracle_mod, xyz, p)
    tracks, members, st, _ = run_view(et, ctx, xyz, p)
    assert st["n_seeds"] == want.n_seeds
    assert_same(et, tracks, members, want)


def test_coordinates_at_the_limit(et, ctx, oracle_mod):
    # extent 2^21 on every axis: coordinates use all 21 bits (packed grains,
    # canonical keys); seed_max 400 keeps the cross products in int32
    E = 1 << 21
    rng = np.random.default_rng(17)
    fog = rng.integers(E - 6000, E, size=(400, 3))
    lines = []
    for d in [(1, 0, 0), (0, 1, 1), (1, 1, 1), (-1, 2, 1)]:
        for k in range(12):
            lines.append([E - 1 - 150 * k * abs(c) if c else E - 1 - 3000 for c in d])
    xyz = np.unique(np.vstack([fog, np.array(lines)]), axis=0).astype(np.int32)
    p = dict(extent=(E, E, E), seed_min=100, seed_max=400, tube_r=20, min_hits=6)
    assert xyz.max() == E - 1
    # the oracle's hash with cells of 2^16 (its default paper cell would need 10^11 cells here)
    with oracle_mod.Oracle(xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"],
                           cell=(1 << 16, 1 << 16, 1 << 16)) as o:
        want = o.find_tracks()
    tracks, members, st, _ = run_view(et, ctx, xyz, p)
    assert len(want) >= 4
    assert_same(et, tracks, members, want)


def test_cell_table_limit(et, ctx):
    # the cell table is indexed with 32-bit signed arithmetic: a tuning that
    # would make 2^31 cells (16384 x 16384 x 8 cells of 128 units) is refused
    # on load, before any allocation, and an automatic grid still works
    E = 1 << 21
    xyz = np.array([[5, 5, 5], [300, 5, 5]], dtype=np.int32)
    p = dict(extent=(E, E, 1024), seed_min=100, seed_max=400, tube_r=20, min_hits=2)
    v = et.View.create(ctx, xyz, p)
    try:
        v.set_tuning((128, 128, 128), row_lists=1)
        with pytest.raises(et.EtError) as e:
            v.load_host(xyz)
        assert e.value.status == et.INVALID_ARG
        v.set_tuning((0, 0, 0), row_lists=0)
        v.load_host(xyz)
        v.find()
        tracks, members = v.fetch()
        assert len(tracks) == 1 and sorted(members.tolist()) == [0, 1]
    finally:
        v.close()


def test_input_errors(et, ctx):
    with pytest.raises(et.EtError) as e:
        v = et.View.create(ctx, np.array([[1, 2, 3], [1000, 2, 3]]), _p())
        try:
            v.find()
            v.fetch()
        finally:
            v.close()
    assert e.value.status == et.OUT_OF_RANGE
    with pytest.raises(et.EtError) as e:
        v = et.View.create(ctx, np.array([[1, 2, 3], [4, 5, 6], [1, 2, 3]]), _p())
        try:
            v.find()
            v.fetch()
        finally:
            v.close()
    assert e.value.status == et.DUPLICATE_GRAIN
    with pytest.raises(et.EtError) as e:
        et.View.create(ctx, np.zeros((1, 3)), _p(extent=(2 ** 21, 2 ** 21, 10), smax=600))
    assert e.value.status == et.PRECONDITION
    with pytest.raises(et.EtError) as e:
        et.View.create(ctx, np.zeros((1, 3)), _p(h=0))
    assert e.value.status == et.INVALID_ARG


def test_torch_allocator_same_result(et, oracle_mod):
    import torch
    v = synth.pr1()
    p = synth.params(v.extent)
    want = oracle_run(oracle_mod, v.xyz, p)
    before = torch.cuda.memory_allocated(0)
    with et.Context(0, use_torch_allocator=True) as c2:
        view = c2.view(v.xyz, p)
        assert torch.cuda.memory_allocated(0) > before
        view.find()
        tracks, members = view.fetch()
        view.close()
    assert_same(et, tracks, members, want)


# ------------------------------------------------------------------ served form

def test_server_results_match_oracle(et, ctx, oracle_mod):
    views = [v for v in synth.batched(n_views=40, seed=4) if v.n < 15000][:20]
    p = synth.params(views[0].extent)
    with ctx.server(p, mem_budget_bytes=2 << 30, max_batch_views=8) as s:
        for k, v in enumerate(views):
            assert s.submit(v.xyz, tag=1000 + k) == et.OK
        got = {}
        for _ in range(2000):
            for r in s.poll(max_results=64, timeout_us=100000):
                assert r.status == et.OK
                assert r.t_submit_ns <= r.t_admit_ns <= r.t_done_ns
                got[r.tag] = s.fetch(r.tag)
            if len(got) == len(views):
                break
    assert len(got) == len(views)
    for k, v in enumerate(views):
        tracks, members = got[1000 + k]
        assert et.track_tuples(tracks, members) == oracle_run(oracle_mod, v.xyz, p).as_tuples()
