"""Pins for the oracle's variants (et_params.flags), without the CUDA path.

* single-pass association (the other reading of the exclusive association of
  Section 2) and the grain-count cut against background (Section 3, Fig. 9c)
  against the brute-force restatement (oracle/brute.py) on small views built
  so that the two association readings disagree;
* the cut's closed form on planted noise-free tracks whose seed vectors have
  tan theta = 0, 1, 2 and infinity, at and around the boundary;
* a single isolated track is found alike by both association readings.
"""
import numpy as np
import pytest

from oracle import brute

EXT = (3000, 3000, 1500)


def bundle_view(seed):
    """40 fog grains and 5 nearly parallel lines through one region: their tubes
    share grains, so the two association readings can disagree."""
    rng = np.random.default_rng(seed)
    pts = [tuple(p) for p in rng.integers(0, EXT, size=(40, 3))]
    c = rng.integers(1000, 2000, 3)
    for _ in range(5):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        off = rng.integers(-60, 60, 3)
        for k in range(-5, 6):
            pts.append(tuple(np.clip((c + off + d * 120 * k).astype(int), 0, np.array(EXT) - 1)))
    pts = np.array(sorted(set(pts)))
    rng.shuffle(pts)
    return pts


def run_oracle(O, pts, ext, smin, smax, r, h, flags=0, cut=(0, 0, 0)):
    o = O.Oracle(pts, ext, smin, smax, r, h, flags=flags, cut=cut)
    try:
        return o.find_tracks().as_tuples()
    finally:
        o.close()


@pytest.mark.parametrize("seed", [0, 1, 2, 5])
def test_variants_match_brute_force(oracle_mod, seed):
    pts = bundle_view(seed)
    _, greedy = brute.find(pts, 100, 500, 40, 6)
    _, single = brute.find(pts, 100, 500, 40, 6, single_pass=True)
    assert greedy != single   # these views separate the two readings
    assert run_oracle(oracle_mod, pts, EXT, 100, 500, 40, 6) == greedy
    assert run_oracle(oracle_mod, pts, EXT, 100, 500, 40, 6, flags=oracle_mod.SINGLE_PASS) == single
    for cut in [(6, 1, 2), (7, 3, 1), (9, 0, 0)]:
        for flags, sp in [(oracle_mod.ANGLE_CUT, False), (oracle_mod.ANGLE_CUT | oracle_mod.SINGLE_PASS, True)]:
            _, want = brute.find(pts, 100, 500, 40, 6, single_pass=sp, cut=cut)
            assert run_oracle(oracle_mod, pts, EXT, 100, 500, 40, 6, flags=flags, cut=cut) == want


def planted(directions, n=10, step=1):
    """Noise-free tracks of n grains at integer multiples of the given integer
    directions, far apart and at different heights (no grain lies on another
    track's line)."""
    pts, starts = [], [(2000, 2000, 200), (12000, 2000, 300), (2000, 12000, 400), (12000, 12000, 500)]
    for d, s in zip(directions, starts):
        for k in range(n):
            pts.append(tuple(s[a] + k * step * d[a] for a in range(3)))
    return np.array(pts, dtype=np.int64)


def test_angle_cut_closed_form(oracle_mod):
    # tan theta of the seed vectors: (0,0,1) -> 0, (1,0,1) -> 1, (6,8,5) -> 2, (1,0,0) -> infinite
    dirs = [(0, 0, 100), (100, 0, 100), (60, 80, 50), (150, 0, 0)]
    pts = planted(dirs)
    ext = (20000, 20000, 2000)
    base = run_oracle(oracle_mod, pts, ext, 90, 400, 5, 8)
    assert sorted(t[2] for t in base) == [10, 10, 10, 10]   # every track, all ten grains

    def kept(cut):
        got = run_oracle(oracle_mod, pts, ext, 90, 400, 5, 8, flags=oracle_mod.ANGLE_CUT, cut=cut)
        tans = []
        for lo, hi, nh, _ in got:
            w = pts[hi] - pts[lo]
            tans.append(np.inf if w[2] == 0 else round(float(np.hypot(w[0], w[1]) / abs(w[2])), 6))
        return sorted(tans)

    # 10 >= 6 + 2 * min(tan, 3): tan 0 (6), 1 (8), 2 (10: the boundary, kept); horizontal 12: dropped
    assert kept((6, 2, 3)) == [0.0, 1.0, 2.0]
    # one grain more at the base: tan 2 needs 11 now
    assert kept((7, 2, 3)) == [0.0, 1.0]
    # capped at tan 1: horizontal needs 6 + 4 = 10 -> kept, like tan 2 (also capped)
    assert kept((6, 4, 1)) == [0.0, 1.0, 2.0, np.inf]
    # slope 0: the cut is a plain count threshold
    assert kept((10, 0, 5)) == [0.0, 1.0, 2.0, np.inf]
    assert kept((11, 0, 5)) == []


def test_single_isolated_track_alike(oracle_mod):
    pts = planted([(60, 80, 50)], n=14)
    ext = (20000, 20000, 2000)
    g = run_oracle(oracle_mod, pts, ext, 90, 400, 5, 8)
    s = run_oracle(oracle_mod, pts, ext, 90, 400, 5, 8, flags=oracle_mod.SINGLE_PASS)
    assert g == s and len(g) == 1 and g[0][2] == 14


def test_variant_argument_errors(oracle_mod):
    pts = planted([(0, 0, 100)])
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Oracle(pts, (20000, 20000, 2000), 90, 400, 5, 8, flags=4)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Oracle(pts, (20000, 20000, 2000), 90, 400, 5, 8, flags=oracle_mod.ANGLE_CUT, cut=(-1, 0, 0))
