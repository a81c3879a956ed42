"""Pins for the CPU oracle: what the paper and the mathematics fix, checked
without the CUDA path.

* hand-worked examples of the Section 2 definition (tests/golden);
* an independent brute-force restatement (oracle/brute.py) on tiny inputs;
* closed forms for one straight track (seed count, every count = n, one
  track, exact direction, zero residual);
* exact recovery of planted noise-free tracks, including a horizontal and a
  vertical one (Table 1: full angular acceptance);
* invariance under input permutation, axis swaps and reflections;
* the cell-hash tube cover against the all-grains definition, for several
  cell shapes;
* the FP64 fit against numpy's eigh / SVD (library routines).
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _oracle(O, xyz, extent, smin, smax, r, h, cell=None):
    kw = {} if cell is None else {"cell": cell}
    return O.Oracle(np.asarray(xyz, dtype=np.int32), extent, smin, smax, r, h, **kw)


def _seed_dict(lo, hi, cnt):
    return {(int(a), int(b)): int(c) for a, b, c in zip(lo, hi, cnt)}


# ------------------------------------------------------------------ golden

def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_worked_example(oracle_mod, case):
    args = (case["grains"], case["extent"], case["seed_min"], case["seed_max"], case["tube_r"],
            case["min_hits"])
    want_seeds = {(a, b): c for a, b, c in case["seeds"]}
    want_tracks = [(a, b, n, tuple(m)) for a, b, n, m in case["tracks"]]
    # the hand derivation agrees with the brute-force restatement ...
    bs, bt = brute.find(case["grains"], *args[2:])
    assert bs == want_seeds
    assert bt == want_tracks
    # ... and with the oracle, for the paper's cell and for tiny cells
    for cell in [None, (3, 5, 7), (1, 1, 1), (1000, 1000, 1000)]:
        with _oracle(oracle_mod, *args, cell=cell) as o:
            tr, (lo, hi, cnt) = o.find_tracks(keep_seeds=True)
            assert _seed_dict(lo, hi, cnt) == want_seeds
            assert tr.as_tuples() == want_tracks


# ------------------------------------------------------------------ brute force

def _small_view(rng, extent, n_fog, tracks, gap):
    """Fog plus straight tracks with small integer jitter, distinct points."""
    pts = set()
    out = []

    def add(p):
        p = tuple(int(min(max(v, 0), e - 1)) for v, e in zip(p, extent))
        if p not in pts:
            pts.add(p)
            out.append(p)

    for _ in range(tracks):
        start = rng.uniform(0, 1, 3) * np.asarray(extent)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        for k in range(int(rng.integers(6, 16))):
            add(np.rint(start + k * gap * d + rng.integers(-1, 2, 3)))
    for _ in range(n_fog):
        add(rng.integers(0, extent))
    xyz = np.asarray(out, dtype=np.int32)
    return xyz[rng.permutation(len(out))]


@pytest.mark.parametrize("seed", range(6))
def test_matches_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    extent = (1500, 1200, 400)
    xyz = _small_view(rng, extent, n_fog=60 + 20 * seed, tracks=3 + seed % 3, gap=37)
    smin, smax, r, h = [(40, 200, 6, 4), (0, 150, 10, 5), (60, 400, 3, 3), (40, 200, 0, 2),
                        (30, 250, 8, 6), (10, 120, 15, 4)][seed]
    bs, bt = brute.find(xyz, smin, smax, r, h)
    for cell in [None, (97, 131, 53), (400, 400, 400), (17, 1200, 9)]:
        with _oracle(oracle_mod, xyz, extent, smin, smax, r, h, cell=cell) as o:
            tr, (lo, hi, cnt) = o.find_tracks(keep_seeds=True)
            assert _seed_dict(lo, hi, cnt) == bs
            assert tr.as_tuples() == bt
            assert tr.n_cand == sum(1 for c in bs.values() if c >= h)


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n,step,direction,window", [
    (12, 1, (3, 4, 12), (30, 100)),
    (20, 2, (2, -3, 6), (20, 120)),      # |d| = 7, descending y
    (9, 5, (0, 0, 1), (4, 21)),          # vertical (theta = 0)
    (15, 3, (4, 3, 0), (14, 61)),        # horizontal (theta = 90 deg)
])
def test_single_track_closed_form(oracle_mod, n, step, direction, window):
    d = np.asarray(direction, dtype=np.int64)
    L = int(round(np.linalg.norm(d)))
    assert L * L == int(d @ d)
    g0 = np.array([500, 500, 500], dtype=np.int64)
    xyz = np.stack([g0 + k * step * d for k in range(n)]).astype(np.int32)
    extent = (2000, 2000, 2000)
    smin, smax = window
    # seeds: pairs whose gap j (in grains) puts j*step*L inside [smin, smax)
    want_seeds = sum(n - j for j in range(1, n) if smin <= j * step * L < smax)
    with _oracle(oracle_mod, xyz, extent, smin, smax, 3, n) as o:
        tr, (lo, hi, cnt) = o.find_tracks(keep_seeds=True)
    assert len(lo) == want_seeds
    assert np.all(cnt == n)
    assert len(tr) == 1 and tr.nhits[0] == n
    assert tuple(tr.member_list(0)) == tuple(range(n))
    # first candidate: all counts tie, so the lowest-ranked pair wins
    ranks = sorted(range(n), key=lambda k: tuple(xyz[k]))
    j = min(j for j in range(1, n) if smin <= j * step * L < smax)
    first = ranks[0]
    assert tr.lo[0] == first
    assert {tr.lo[0], tr.hi[0]} == {first, first + j if first == 0 else first - j}
    # fit: exact direction along lo -> hi, centroid midway, zero residual
    u_want = (xyz[tr.hi[0]] - xyz[tr.lo[0]]).astype(np.float64)
    u_want /= np.linalg.norm(u_want)
    np.testing.assert_allclose(tr.u[0], u_want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(tr.c[0], g0 + (n - 1) / 2 * step * d, rtol=0, atol=1e-9)
    half = (n - 1) / 2 * step * L
    np.testing.assert_allclose(tr.t[0], [-half, half], rtol=0, atol=1e-9)
    assert abs(tr.lam[0][1]) < 1e-6 and abs(tr.lam[0][2]) < 1e-6
    # one more grain than the track holds -> nothing passes the threshold
    with _oracle(oracle_mod, xyz, extent, smin, smax, 3, n + 1) as o:
        assert len(o.find_tracks()) == 0


def _planted(rng, extent, dirs, grains_per, margin=300):
    tracks, pts = [], []
    for d in dirs:
        d = np.asarray(d, dtype=np.int64)
        for _ in range(1000):
            g0 = rng.integers(margin, np.asarray(extent) - margin)
            line = [g0 + k * d for k in range(grains_per)]
            if all(np.all(p >= 0) and np.all(p < extent) for p in line):
                break
        tracks.append(len(pts))
        pts.extend(line)
    return np.asarray(pts, dtype=np.int32)


def test_planted_tracks_recovered_exactly(oracle_mod):
    rng = np.random.default_rng(7)
    extent = (20000, 20000, 4000)
    # horizontal, vertical and oblique lattice directions (|d| ~ 100-300 units)
    dirs = [(150, 80, 0), (0, 0, 160), (90, -120, 60), (-200, 30, 10), (40, 40, -140),
            (0, 170, 0), (120, 0, -90)]
    n_per = 14
    xyz = _planted(rng, extent, dirs, n_per)
    r, h = 20, 6
    # the construction keeps every line farther than r from other tracks' grains
    for t, d in enumerate(dirs):
        d = np.asarray(d, dtype=np.float64)
        a = xyz[t * n_per].astype(np.float64)
        others = np.delete(xyz, np.s_[t * n_per:(t + 1) * n_per], axis=0).astype(np.float64)
        dist = np.linalg.norm(np.cross(others - a, d), axis=1) / np.linalg.norm(d)
        if np.any(dist <= r):
            pytest.skip("random placement crossed another track")
    perm = rng.permutation(xyz.shape[0])   # oracle id m is grain perm[m] of xyz
    with _oracle(oracle_mod, xyz[perm], extent, 250, 1000, r, h) as o:
        tr = o.find_tracks()
    assert len(tr) == len(dirs)
    got = sorted(tuple(sorted(int(perm[m]) for m in tr.member_list(k))) for k in range(len(tr)))
    want = sorted(tuple(range(t * n_per, (t + 1) * n_per)) for t in range(len(dirs)))
    assert got == want
    for k in range(len(tr)):
        t = int(perm[tr.member_list(k)[0]]) // n_per
        d = np.asarray(dirs[t], dtype=np.float64)
        assert abs(abs(tr.u[k] @ d) / np.linalg.norm(d) - 1) < 1e-12


# ------------------------------------------------------------------ invariances

def _pr1_like(seed=11, n_fog=500, n_tracks=8):
    from paper_1311_5334_gb300 import synth
    v = synth.make_view(seed, extent=(8000, 8000, 2000), n_fog=n_fog, n_through=n_tracks,
                        n_short=2, gap_through_um=2.0)
    return v


def test_permutation_invariance(oracle_mod):
    v = _pr1_like()
    args = (v.extent, 300, 1500, 40, 5)
    rng = np.random.default_rng(3)
    perm = rng.permutation(v.n)
    with _oracle(oracle_mod, v.xyz, *args) as o:
        a = o.find_tracks()
    with _oracle(oracle_mod, v.xyz[perm], *args) as o:
        b = o.find_tracks()
    assert len(a) > 0
    mapped = [(int(perm[lo]), int(perm[hi]), n, tuple(sorted(int(perm[m]) for m in mem)))
              for lo, hi, n, mem in b.as_tuples()]
    assert mapped == a.as_tuples()
    np.testing.assert_allclose(a.u, b.u, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a.c, b.c, rtol=1e-13)
    np.testing.assert_allclose(a.t, b.t, rtol=0, atol=1e-8)


def _unordered_counts(lo, hi, cnt):
    return {frozenset((int(a), int(b))): int(c) for a, b, c in zip(lo, hi, cnt)}


@pytest.mark.parametrize("transform", ["swap_xy", "swap_xz", "reflect_x", "reflect_z"])
def test_axis_swap_and_reflection(oracle_mod, transform):
    v = _pr1_like(seed=12)
    ext = list(v.extent)
    xyz = v.xyz.copy()
    if transform == "swap_xy":
        xyz[:, [0, 1]] = xyz[:, [1, 0]]
        ext[0], ext[1] = ext[1], ext[0]
    elif transform == "swap_xz":
        xyz[:, [0, 2]] = xyz[:, [2, 0]]
        ext[0], ext[2] = ext[2], ext[0]
    elif transform == "reflect_x":
        xyz[:, 0] = ext[0] - 1 - xyz[:, 0]
    else:
        xyz[:, 2] = ext[2] - 1 - xyz[:, 2]
    with _oracle(oracle_mod, v.xyz, v.extent, 300, 1500, 40, 5) as o:
        _, s0 = o.find_tracks(keep_seeds=True)
    with _oracle(oracle_mod, xyz, ext, 300, 1500, 40, 5) as o:
        _, s1 = o.find_tracks(keep_seeds=True)
    assert _unordered_counts(*s0) == _unordered_counts(*s1)


# ------------------------------------------------------------------ cover vs definition

@pytest.mark.parametrize("cell", [(750, 750, 125), (97, 131, 53), (5000, 5000, 5000), (40, 2000, 7),
                                  (41, 41, 41)])
def test_hash_cover_equals_all_grains_pr1(oracle_mod, cell):
    from paper_1311_5334_gb300 import synth
    v = synth.pr1()
    with _oracle(oracle_mod, v.xyz, v.extent, 500, 2000, 40, 8, cell=cell) as o:
        lo, hi = o.seeds()
        a = o.count_pairs(lo, hi)
        b = o.count_pairs(lo, hi, brute=True)
    assert len(lo) > 10000
    assert np.array_equal(a, b)


def test_seeds_per_grain_matches_seed_list(oracle_mod):
    from paper_1311_5334_gb300 import synth
    v = synth.pr1()
    with _oracle(oracle_mod, v.xyz, v.extent, 500, 2000, 40, 8) as o:
        lo, hi = o.seeds()
        per = o.seeds_per_grain()
    assert per.sum() == len(lo)
    assert np.array_equal(per, np.bincount(lo, minlength=v.n))


def test_hash_cover_equals_all_grains_lattice(oracle_mod):
    """A regular lattice makes many seeds axis-aligned or diagonal, with grains
    exactly on tube walls and cell faces."""
    g = np.arange(0, 600, 60)
    xyz = np.array(list(itertools.product(g, g, g[:5])), dtype=np.int32)
    extent = (600, 600, 300)
    for cell, r in [((60, 60, 60), 0), ((59, 61, 30), 30), ((7, 7, 7), 60), ((600, 1, 13), 42)]:
        with _oracle(oracle_mod, xyz, extent, 60, 200, r, 3, cell=cell) as o:
            lo, hi = o.seeds()
            assert np.array_equal(o.count_pairs(lo, hi), o.count_pairs(lo, hi, brute=True))


# ------------------------------------------------------------------ fit

def test_jacobi_matches_numpy_eigh(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(200):
        a = rng.normal(size=(3, 3)) * rng.uniform(0.1, 1e4)
        m = a @ a.T
        lam, vec = oracle_mod.sym_eigen3(m)
        wl, wv = np.linalg.eigh(m)
        np.testing.assert_allclose(lam, wl[::-1], rtol=1e-10, atol=1e-9 * wl.max())
        # principal vector up to sign (well separated in these draws)
        if wl[2] > 1.01 * wl[1]:
            assert abs(abs(vec[0] @ wv[:, 2]) - 1) < 1e-9
        np.testing.assert_allclose(m @ vec.T, vec.T * lam, rtol=0, atol=1e-9 * wl.max())


def test_fit_matches_svd_on_noisy_tracks(oracle_mod):
    from paper_1311_5334_gb300 import synth
    v = synth.dense()
    with _oracle(oracle_mod, v.xyz[:4000], v.extent, 500, 2000, 40, 8) as o:
        rng = np.random.default_rng(9)
        for _ in range(50):
            mem = np.sort(rng.choice(4000, size=int(rng.integers(3, 60)), replace=False)).astype(np.int32)
            c, u, t, lam = o.fit(mem, mem[0], mem[-1])
            p = v.xyz[mem].astype(np.float64)
            cw = p.mean(axis=0)
            _, sv, vt = np.linalg.svd(p - cw)
            np.testing.assert_allclose(c, cw, rtol=1e-13)
            np.testing.assert_allclose(lam, sv ** 2, rtol=1e-9, atol=1e-6)
            if sv[0] > 1.01 * sv[1]:
                assert abs(abs(u @ vt[0]) - 1) < 1e-9
            proj = (p - c) @ u
            np.testing.assert_allclose(t, [proj.min(), proj.max()], rtol=1e-12, atol=1e-6)
            assert u @ (p[-1] - p[0]) >= 0


# ------------------------------------------------------------------ errors

def test_rejects_bad_input(oracle_mod):
    O = oracle_mod
    ext = (100, 100, 100)
    with pytest.raises(O.OracleError) as e:
        _oracle(O, [[0, 0, 0], [100, 0, 0]], ext, 1, 10, 1, 2)
    assert e.value.status == O.OUT_OF_RANGE
    with pytest.raises(O.OracleError) as e:
        _oracle(O, [[1, 2, 3], [4, 5, 6], [1, 2, 3]], ext, 1, 10, 1, 2)
    assert e.value.status == O.DUPLICATE
    with pytest.raises(O.OracleError) as e:
        _oracle(O, [[1, 2, 3]], ext, 10, 5, 1, 2)
    assert e.value.status == O.INVALID_ARG
    with _oracle(O, np.zeros((0, 3)), ext, 1, 10, 1, 2) as o:
        tr = o.find_tracks()
        assert len(tr) == 0 and tr.n_seeds == 0
