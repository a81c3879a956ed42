"""Writes the expected full-size results of the batched workload (256 views of
300x300x50 um, seed 3), of the first 256 views of the served workload (the
batched size law, seed 4) and of the stress workload (one 1000x1000x50 um
view, seed 5) as digests: fullsize_batched_seed3.json,
fullsize_served_seed4.json and fullsize_stress_seed5.json beside this script.

Every expected value comes from the CPU oracle (oracle/), which evaluates the
definition of Section 2 and Fig. 4 of the paper: seeds in the distance window,
exact tube counts over all grains, threshold, sequential greedy exclusive
association.  Nothing here calls the CUDA library.

  python tests/golden/make_fullsize_digests.py [batched|served|stress|variants|all] [--threads T]

"variants" writes fullsize_variants_seed3.json: the track-list digests of the
batched workload under the single-pass association (flags 1) and under the
sequential association with the grain-count cut (flags 2, cut 9, 3, 4).

Takes minutes on a multi-core host (the per-seed tube counts run on all cores).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import fullsize  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1311_5334_gb300 import synth  # noqa: E402


def view_record(v, p, threads):
    o = O.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"])
    try:
        tr, (slo, shi, scnt) = o.find_tracks(nthreads=threads, keep_seeds=True)
    finally:
        o.close()
    n_seeds, sd = fullsize.seed_digest(slo, shi, scnt)
    return {
        "n_grains": v.n,
        "input_sha256": fullsize.input_digest(v.xyz),
        "n_seeds": n_seeds,
        "seed_hash": sd,
        "n_hits": int(scnt.astype("int64").sum()),
        "n_candidates": int(tr.n_cand),
        "n_tracks": len(tr),
        "n_track_members": int(tr.moff[-1]) if len(tr) else 0,
        "tracks_sha256": fullsize.track_digest(tr.as_tuples()),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="?", default="all", choices=["batched", "served", "stress", "variants", "all"])
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    O.build()
    if a.which in ("batched", "all"):
        t0 = time.time()
        views = synth.batched(n_views=256, seed=3)
        p = synth.params(views[0].extent)
        recs = []
        for k, v in enumerate(views):
            recs.append(view_record(v, p, a.threads))
            print(f"batched view {k}: {v.n} grains, {recs[-1]['n_tracks']} tracks "
                  f"({time.time() - t0:.0f} s)", flush=True)
        out = {"workload": "batched: synth.batched(n_views=256, seed=3), synth.params",
               "source": "oracle/oracle.c via oracle.Oracle.find_tracks(keep_seeds=True)",
               "views": recs}
        with open(os.path.join(HERE, "fullsize_batched_seed3.json"), "w") as f:
            json.dump(out, f, indent=0)
    if a.which in ("served", "all"):
        t0 = time.time()
        views = synth.batched(n_views=256, seed=4)
        p = synth.params(views[0].extent)
        recs = []
        for k, v in enumerate(views):
            recs.append(view_record(v, p, a.threads))
            print(f"served view {k}: {v.n} grains, {recs[-1]['n_tracks']} tracks "
                  f"({time.time() - t0:.0f} s)", flush=True)
        out = {"workload": "served: synth.batched(n_views=256, seed=4) (the first 256 views of the served "
                           "stream), synth.params",
               "source": "oracle/oracle.c via oracle.Oracle.find_tracks(keep_seeds=True)",
               "views": recs}
        with open(os.path.join(HERE, "fullsize_served_seed4.json"), "w") as f:
            json.dump(out, f, indent=0)
    if a.which in ("variants", "all"):
        t0 = time.time()
        views = synth.batched(n_views=256, seed=3)
        out = {"workload": "batched: synth.batched(n_views=256, seed=3) under association variants",
               "source": "oracle/oracle.c via oracle.Oracle.find_tracks with flags and cut", "variants": {}}
        for name, flags, cut in (("single_pass", 1, (0, 0, 0)), ("angle_cut_9_3_4", 2, (9, 3, 4))):
            p = synth.params(views[0].extent, flags=flags, cut=cut)
            recs = []
            for k, v in enumerate(views):
                o = O.Oracle(v.xyz, p["extent"], p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"],
                             flags=flags, cut=cut)
                try:
                    tr = o.find_tracks(nthreads=a.threads)
                finally:
                    o.close()
                recs.append({"input_sha256": fullsize.input_digest(v.xyz), "n_tracks": len(tr),
                             "tracks_sha256": fullsize.track_digest(tr.as_tuples())})
            print(f"{name}: {sum(r['n_tracks'] for r in recs)} tracks ({time.time() - t0:.0f} s)", flush=True)
            out["variants"][name] = {"flags": flags, "cut": list(cut), "views": recs}
        with open(os.path.join(HERE, "fullsize_variants_seed3.json"), "w") as f:
            json.dump(out, f, indent=0)
    if a.which in ("stress", "all"):
        t0 = time.time()
        v = synth.stress()
        p = synth.params(v.extent)
        rec = view_record(v, p, a.threads)
        print(f"stress: {v.n} grains, {rec['n_seeds']} seeds, {rec['n_tracks']} tracks "
              f"({time.time() - t0:.0f} s)", flush=True)
        out = {"workload": "stress: synth.stress(seed=5), synth.params",
               "source": "oracle/oracle.c via oracle.Oracle.find_tracks(keep_seeds=True)",
               "view": rec}
        with open(os.path.join(HERE, "fullsize_stress_seed5.json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
