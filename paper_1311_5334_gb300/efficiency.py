"""Tracking efficiency and fake rate on synthetic views (the analogue of the
cosmic-ray study of Section 3, Fig. 8-9), using the GPU path through the
binding.

The paper measures efficiency with tracks reconstructed in the other layers
of a detector stack as references, and the fake rate by displacing one
layer's data by 1 mm so that no true counterpart exists.  Here the
references are the planted tracks of synthetic views, whose lines are known:

* efficiency: the fraction of reference tracks (planted lines with at least
  `min_grains` grains in the view) matched by a reconstructed track, in bins
  of tan theta (theta: angle to the z axis, the plate normal);
* displaced fake rate: the fraction of one view's reference tracks matched by
  a track reconstructed in a different view (no true counterpart);
* fog-only fakes: tracks reconstructed per view holding fog alone.

A reconstructed track matches a reference when its direction lies within
`max_angle` of the reference's (either orientation) and its centroid within
`max_dist_um` of the reference line.

    python -m paper_1311_5334_gb300.efficiency [--views 64] [--seed 11]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import synth

TAN_BINS = (0.0, 0.5, 1.0, 2.0, 5.0, np.inf)


def match(truth, centroids_um, directions, max_angle=0.03, max_dist_um=1.0):
    """Boolean per reference line (truth rows: point, unit direction): is there
    a track with centroid c (um) and unit direction u within the tolerances?"""
    truth = np.asarray(truth, dtype=np.float64).reshape(-1, 6)
    c = np.asarray(centroids_um, dtype=np.float64).reshape(-1, 3)
    u = np.asarray(directions, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(truth.shape[0], dtype=bool)
    if c.shape[0] == 0:
        return out
    un = u / np.linalg.norm(u, axis=1, keepdims=True)
    cos_max = np.cos(max_angle)
    for i, row in enumerate(truth):
        p, d = row[:3], row[3:] / np.linalg.norm(row[3:])
        ok = np.abs(un @ d) >= cos_max
        if not ok.any():
            continue
        rel = c[ok] - p
        dist = np.linalg.norm(rel - np.outer(rel @ d, d), axis=1)
        out[i] = bool((dist <= max_dist_um).any())
    return out


def tan_theta(directions):
    d = np.asarray(directions, dtype=np.float64).reshape(-1, 3)
    with np.errstate(divide="ignore"):
        return np.hypot(d[:, 0], d[:, 1]) / np.abs(d[:, 2])


def binned(found, tans, bins=TAN_BINS):
    """[(lo, hi, n, efficiency)] per tan theta bin."""
    rows = []
    for lo, hi in zip(bins[:-1], bins[1:]):
        sel = (tans >= lo) & ((tans < hi) | np.isinf(hi))   # the last bin holds horizontal tracks
        n = int(sel.sum())
        rows.append((lo, hi, n, float(found[sel].mean()) if n else None))
    return rows


def reference_mask(view, min_grains):
    counts = np.bincount(view.label[view.label >= 0], minlength=view.n_tracks)
    return counts >= min_grains


def run_views(et, ctx, views, params):
    """Tracks of each view through one batch: [(centroids um, directions)]."""
    xyz, offs = synth.concat(views)
    b = et.Batch(ctx, params)
    try:
        b.load(xyz, offs)
        b.find(use_graph=False)
        tracks, _, voff = b.fetch()
    finally:
        b.close()
    out = []
    for k in range(len(views)):
        t = tracks[voff[k]:voff[k + 1]]
        out.append((np.asarray(t["c"], dtype=np.float64) / synth.UM, np.asarray(t["u"], dtype=np.float64)))
    return out


def study(ctx, n_views=64, seed=11, n_fog=10000, n_tracks=100, min_grains=None, max_angle=0.03,
          max_dist_um=1.0, params=None):
    from . import et
    extent = (300 * synth.UM, 300 * synth.UM, 50 * synth.UM)
    params = params or synth.params(extent)
    min_grains = min_grains if min_grains is not None else params["min_hits"] + 2
    views = [synth.make_view([seed, k], extent=extent, n_fog=n_fog, n_through=n_tracks) for k in range(n_views)]
    reco = run_views(et, ctx, views, params)
    found, tans, disp = [], [], []
    for k, v in enumerate(views):
        ref = reference_mask(v, min_grains)
        truth = v.truth[ref]
        found.append(match(truth, *reco[k], max_angle, max_dist_um))
        tans.append(tan_theta(truth[:, 3:]))
        # displaced: the references of view k against the tracks of view k + 1
        disp.append(match(truth, *reco[(k + 1) % n_views], max_angle, max_dist_um))
    found, tans, disp = np.concatenate(found), np.concatenate(tans), np.concatenate(disp)
    fog_views = [synth.make_view([seed, 1000 + k], extent=extent, n_fog=n_fog, n_through=0)
                 for k in range(max(4, n_views // 4))]
    fog_tracks = [len(r[0]) for r in run_views(et, ctx, fog_views, params)]
    return {
        "references": int(found.size),
        "efficiency": float(found.mean()) if found.size else None,
        "efficiency_by_tan_theta": [{"tan_lo": lo, "tan_hi": (None if np.isinf(hi) else hi), "n": n,
                                     "efficiency": e} for lo, hi, n, e in binned(found, tans)],
        "displaced_fake_rate": float(disp.mean()) if disp.size else None,
        "fog_only_tracks_per_view": float(np.mean(fog_tracks)),
        "config": {"views": n_views, "seed": seed, "fog_per_view": n_fog, "tracks_per_view": n_tracks,
                   "reference_min_grains": min_grains, "max_angle_rad": max_angle, "max_dist_um": max_dist_um,
                   "fog_only_views": len(fog_views), "params": {k: params[k] for k in params}},
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--views", type=int, default=64)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--fog", default="10000,50000,90000",
                    help="fog grains per 300x300x50 um view, one report line each (90k: the stress density)")
    ap.add_argument("--tracks", type=int, default=100)
    ap.add_argument("--min-grains", type=int, default=None, help="reference tracks: grains in the view (min_hits)")
    ap.add_argument("--flags", type=int, default=0)
    ap.add_argument("--cut", default="0,0,0")
    args = ap.parse_args(argv)
    from . import et
    extent = (300 * synth.UM, 300 * synth.UM, 50 * synth.UM)
    params = synth.params(extent, flags=args.flags, cut=tuple(int(c) for c in args.cut.split(",")))
    min_grains = args.min_grains if args.min_grains is not None else params["min_hits"]
    with et.Context(0) as ctx:
        for fog in (int(f) for f in args.fog.split(",")):
            rep = study(ctx, n_views=args.views, seed=args.seed, n_fog=fog, n_tracks=args.tracks,
                        min_grains=min_grains, params=params)
            print(json.dumps(rep), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
