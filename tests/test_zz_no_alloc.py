"""The allocation-free entry point (et_tube_count_noalloc) against the oracle
and against the regular, allocating path's per-seed counts.

It serves callers that cannot allocate device memory: an acquisition loop
that must not block on an allocation's device-wide synchronisation, code in a
host function enqueued on a stream, or a process whose framework owns the free
device memory.  The entry point keeps its cell list in one fixed device array
shared by all calls, so each test makes two calls in a row on the same stream
and checks both results against the CPU oracle's exact counts (and, for the
seeds of a view, against et_view_seed_counts of the regular path): the second
call must not see anything the first one left behind.  It lives in its own file,
collected last, so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

from paper_1311_5334_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc_twice(et, torch, xyz, p, pairs):
    d_xyz = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.int32)).cuda()
    d_pairs = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
    outs = []
    for _ in range(2):
        out = torch.full((len(pairs),), -7, dtype=torch.int32, device="cuda")
        et.tube_count_noalloc(d_xyz, p, d_pairs, out)     # legacy default stream, like torch's ops
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    return outs


def _expected(oracle_mod, xyz, p, pairs):
    """Oracle counts; -1 where the entry point rejects the pair (equal indices,
    coinciding grains, or seed_max or more apart along an axis)."""
    pairs = np.asarray(pairs, dtype=np.int64)
    w = xyz[pairs[:, 1]].astype(np.int64) - xyz[pairs[:, 0]].astype(np.int64)
    bad = (pairs[:, 0] == pairs[:, 1]) | np.all(w == 0, axis=1) | np.any(np.abs(w) >= p["seed_max"], axis=1)
    want = np.full(len(pairs), -1, dtype=np.int64)
    ok = np.nonzero(~bad)[0]
    o = oracle_mod.Oracle(xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
    try:
        want[ok] = o.count_pairs(pairs[ok, 0], pairs[ok, 1])
    finally:
        o.close()
    return want, bad


def test_noalloc_counts_match_oracle_on_two_calls(oracle_mod):
    import torch
    from paper_1311_5334_gb300 import et

    v = synth.pr1()
    p = synth.params(v.extent)
    o = oracle_mod.Oracle(v.xyz, v.extent, p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
    try:
        lo, hi = o.seeds()
    finally:
        o.close()
    assert len(lo) > 10000
    # every seed, plus: equal indices, and pairs across the view (far beyond
    # seed_max: rejected rather than counted with overflowing products)
    far_i = int(np.argmin(v.xyz[:, 0]))
    far_j = int(np.argmax(v.xyz[:, 0]))
    extra = np.array([[3, 3], [far_i, far_j], [far_j, far_i]], dtype=np.int64)
    pairs = np.concatenate([np.stack([lo, hi], 1), extra])
    want, bad = _expected(oracle_mod, v.xyz, p, pairs)
    assert bad[-3:].all() and not bad[:-3].any()
    # the regular, allocating path's per-seed table for the same view
    # (et_view_seed_counts after et_track_find), keyed by the seed's grain ids
    with et.Context(0) as ctx:
        view = ctx.view(v.xyz, p)
        view.find()
        view.fetch()
        si, sj, sc = view.seed_counts()
        view.close()
    n = len(v.xyz)
    order = np.argsort(si.astype(np.int64) * n + sj)
    keys = (si.astype(np.int64) * n + sj)[order]
    pos = np.searchsorted(keys, lo.astype(np.int64) * n + hi)
    assert len(si) == len(lo) and np.array_equal(keys[pos], lo.astype(np.int64) * n + hi)
    regular = sc[order][pos]
    assert np.array_equal(regular, want[:len(lo)]), "regular path differs from the oracle"
    for call, got in enumerate(_noalloc_twice(et, torch, v.xyz, p, pairs)):
        assert np.array_equal(got[:len(lo)], regular), f"call {call}: differs from et_view_seed_counts"
        assert np.array_equal(got, want), f"call {call}"


def test_noalloc_at_the_grain_and_cell_limits(oracle_mod):
    """65,536 grains (the limit) on a wide, flat extent: about one grain per
    cell would need millions of cells, so the entry point coarsens its grid
    until it fits 262,144 cells; the counts must still equal the oracle's."""
    import torch
    from paper_1311_5334_gb300 import et

    ext = (1 << 21, 1 << 20, 4)
    p = synth.params(ext, seed_min=0, seed_max=600, tube_r=40, min_hits=3)
    rng = np.random.default_rng(91)
    n = 65536
    # clusters along short random lines (many close pairs) plus uniform grains
    n_cl = 4096
    centre = rng.integers([1000, 1000, 0], [ext[0] - 1000, ext[1] - 1000, 4], size=(n_cl // 8, 3))
    d = rng.normal(size=(n_cl // 8, 2))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t = np.arange(8) * 70.0
    cl = centre[:, None, :2] + t[None, :, None] * d[:, None, :]
    cl = np.concatenate([np.rint(cl).reshape(-1, 2), np.repeat(centre[:, 2:], 8, axis=0)], axis=1)
    uni = rng.integers(0, ext, size=(n - n_cl, 3))
    xyz = np.concatenate([cl, uni]).astype(np.int64)
    xyz = np.clip(xyz, 0, np.array(ext) - 1)
    # make the coordinates distinct (the entry point does not check duplicates)
    _, first = np.unique(xyz, axis=0, return_index=True)
    keep = np.sort(first)
    while len(keep) < n:
        add = rng.integers(0, ext, size=(n - len(keep), 3))
        xyz = np.concatenate([xyz[keep], add])
        _, first = np.unique(xyz, axis=0, return_index=True)
        keep = np.sort(first)
    xyz = np.ascontiguousarray(xyz[keep][:n], dtype=np.int32)
    assert len(xyz) == n
    # pairs: neighbours inside clusters, random (mostly far apart) pairs
    pc = np.stack([np.arange(0, n_cl - 1), np.arange(1, n_cl)], 1)
    pr = rng.integers(0, n, size=(20000, 2))
    pairs = np.concatenate([pc, pr])
    want, bad = _expected(oracle_mod, xyz, p, pairs)
    assert (~bad).sum() > 3000 and bad.sum() > 10000
    assert (want[~bad] >= 2).all() and (want >= 8).sum() > 100
    for call, got in enumerate(_noalloc_twice(et, torch, xyz, p, pairs)):
        assert np.array_equal(got, want), f"call {call}"


def test_noalloc_rejects_views_beyond_the_fixed_limit():
    import torch
    from paper_1311_5334_gb300 import et

    n = 65537
    xyz = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    pairs = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = synth.params((30000, 30000, 5000))
    with pytest.raises(et.EtError) as e:
        et.tube_count_noalloc(xyz, p, pairs, out)
    assert e.value.status == et.INVALID_ARG
