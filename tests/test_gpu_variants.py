"""GPU variants (et_params.flags) vs the oracle and the brute force, through the C ABI.

Single-pass association and the angle-dependent grain-count cut are integer
work: the track lists (seed pair, nhits, members, order) must be identical.
"""
import numpy as np
import pytest

from paper_1311_5334_gb300 import synth
from tests.test_oracle_variants import EXT, bundle_view, planted

pytestmark = pytest.mark.gpu

SP, CUT = 1, 2


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


def gpu_tracks(et, ctx, xyz, p, cell=None, rows=0):
    v = et.View.create(ctx, xyz, p)
    try:
        if cell is not None:
            v.set_tuning(cell, row_lists=rows)
            v.load_host(xyz)
        v.find()
        tracks, members = v.fetch()
    finally:
        v.close()
    return et.track_tuples(tracks, members)


def oracle_tracks(O, xyz, p):
    o = O.Oracle(xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"],
                 flags=p.get("flags", 0), cut=p.get("cut", (0, 0, 0)))
    try:
        return o.find_tracks().as_tuples()
    finally:
        o.close()


@pytest.mark.parametrize("seed", [0, 1, 2, 5])
def test_bundles_vs_brute_force(et, ctx, seed):
    from oracle import brute
    pts = bundle_view(seed)
    for flags, cut in [(0, (0, 0, 0)), (SP, (0, 0, 0)), (CUT, (6, 1, 2)), (SP | CUT, (7, 3, 1))]:
        _, want = brute.find(pts, 100, 500, 40, 6, single_pass=bool(flags & SP),
                             cut=cut if flags & CUT else None)
        p = dict(extent=EXT, seed_min=100, seed_max=500, tube_r=40, min_hits=6, flags=flags, cut=cut)
        for cell in (None, (97, 131, 53)):
            assert gpu_tracks(et, ctx, pts, p, cell=cell, rows=1) == want


def test_angle_cut_closed_form(et, ctx):
    pts = planted([(0, 0, 100), (100, 0, 100), (60, 80, 50), (150, 0, 0)])
    ext = (20000, 20000, 2000)
    for cut, n_kept in [((6, 2, 3), 3), ((7, 2, 3), 2), ((6, 4, 1), 4), ((11, 0, 5), 0)]:
        p = dict(extent=ext, seed_min=90, seed_max=400, tube_r=5, min_hits=8, flags=CUT, cut=cut)
        assert len(gpu_tracks(et, ctx, pts, p)) == n_kept


@pytest.mark.parametrize("workload", ["pr1", "dense"])
@pytest.mark.parametrize("flags,cut", [(SP, (0, 0, 0)), (CUT, (9, 3, 4)), (SP | CUT, (8, 2, 6))])
def test_workloads(et, ctx, oracle_mod, workload, flags, cut):
    v = synth.pr1() if workload == "pr1" else synth.dense()
    p = synth.params(v.extent, flags=flags, cut=cut)
    want = oracle_tracks(oracle_mod, v.xyz, p)
    base = oracle_tracks(oracle_mod, v.xyz, synth.params(v.extent))
    if flags & CUT:
        assert 0 < len(want) < len(base) or workload == "pr1"   # the cut bites on the dense view
    assert gpu_tracks(et, ctx, v.xyz, p) == want


def test_batched_single_pass_graph(et, ctx, oracle_mod):
    views = [v for v in synth.batched(n_views=24, seed=3) if v.n < 20000][:12]
    xyz, offs = synth.concat(views)
    p = synth.params(views[0].extent, flags=SP | CUT, cut=(9, 3, 4))
    b = et.Batch(ctx, p)
    try:
        b.load(xyz, offs)
        for use_graph in (False, True, True):
            b.find(use_graph=use_graph)
            tracks, members, voff = b.fetch()
            for k, v in enumerate(views):
                sub = tracks[voff[k]:voff[k + 1]]
                assert et.track_tuples(sub, members) == oracle_tracks(oracle_mod, v.xyz, p)
    finally:
        b.close()


def test_variant_argument_errors(et, ctx):
    pts = planted([(0, 0, 100)])
    ext = (20000, 20000, 2000)
    for flags, cut in [(4, (0, 0, 0)), (CUT, (-1, 0, 0)), (CUT, (0, 1 << 21, 0)), (CUT, (0, 0, 2000))]:
        p = dict(extent=ext, seed_min=90, seed_max=400, tube_r=5, min_hits=8, flags=flags, cut=cut)
        with pytest.raises(et.EtError) as e:
            et.View.create(ctx, pts, p)
        assert e.value.status == et.INVALID_ARG
