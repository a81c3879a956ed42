"""Benchmark of the track-finding hot path on GB300 (one JSON line on stdout).

Step = one pass of the whole path (canonical order + cell list, seeds, tube
counts, candidates + member lists, merge, fit/output) over one batch of 256
synthetic views of 300x300x50 um (lognormal grain counts, median 10k, range
2k-50k, isotropic tracks at 1 % of the grains, seed 3), run as one batched
launch sequence replayed from a CUDA graph, with the grains already resident
in device memory.  L2 is flushed (256 MiB write) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain restatement of the method)
on the machine's host cores, on a bounded sample of the same workload per step.
For N > 1 (torchrun) each rank processes its own batch (weak scaling, no
data-path collective); the timed region is bracketed by barriers and the
maximum over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1311_5334_gb300 import synth  # noqa: E402

VIEW_CM2 = 300e-4 * 300e-4          # one 300 x 300 um view in cm^2 (stress views: 1000 x 1000 um)
WORKLOAD = ("batched: 256 views 300x300x50 um, fog lognormal (median 10k, sigma 0.6, 2k-50k), "
            "isotropic through-going tracks at 1% of the fog count, gaps 3.3 um, jitter 0.05/0.3 um, "
            "int32 10 nm coords, seed window 5-20 um, tube 0.4 um, min hits 8, seed 3")
METRIC = "views/s"
# One tube-membership test: 3 IADD (offset), 6 IMUL/IMAD (int32 cross product),
# 3 IMAD.WIDE (64-bit squared norm), 2 for the 64-bit compare.
OPS_PER_TEST = 14
# One seed-window test of the seed generator: 3 IADD (offset), 3 IMAD.WIDE
# (squared distance); the two compares with the window and the rank test are
# not counted.
OPS_PER_PAIR_TEST = 6
# DRAM bytes one launch of the tube-count kernel (seed generation and tube
# counts) moves, dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture of that launch (one pass, the first timed step, the kernel as built
# now; profiles/k_tube_count_batched.md):
#   batched  613.92 MB + 45.33 MB  (256 views, cells 74x621x506, both lists, 2 origins per ticket)
# The kernel reads each view's grains and cell tables about once, so the bytes
# follow the views and the cell shape rather than the seeds.  Keyed by
# (workload, views, cell edges, cell lists, origins per ticket); a run under
# any other launch configuration reports null.
TUBE_DRAM_BYTES = {("batched", 256, (74, 621, 506), 2, 2): 613.92e6 + 45.33e6}


def tube_run_key(workload, n_views, cell, tuning, rows=1, ticket_origins=0):
    """Launch configuration of a tracking run, the key of TUBE_DRAM_BYTES:
    (workload, views, cell edges, cell lists, seed origins per ticket).
    tuning: the autotuner's choice, or None for edges fixed on the command
    line (rows 1 = x rows only, else both lists; 0 origins = the default 2)."""
    if tuning is not None:
        lists, origins = int(tuning["row_lists"]), int(tuning["ticket_origins"])
    else:
        lists, origins = (1 if rows == 1 else 2), (int(ticket_origins) or 2)
    return (workload, int(n_views), tuple(int(c) for c in cell), lists, origins)


def hbm_roofline(traffic, kernel_ms, peaks):
    """DRAM bytes of one launch over its kernel time against the measured copy
    bandwidth; None without a traffic capture for the launch configuration."""
    if traffic is None:
        return None
    peak = float(peaks.get("hbm_gbs", 6800.0))
    gbs = traffic / (kernel_ms / 1e3) / 1e9
    return {"traffic_bytes": traffic, "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak,
            "peak_src": "of measured" if "hbm_gbs" in peaks else "of fallback"}


def measured_peaks():
    """The measured peaks (MEASURED_PEAKS.json), or {} when absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}
# DRAM bytes of the front end's recognition kernel per view of raw frames
# (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of 8 views:
# 430.69 MB + 6.07 MB); a launch's traffic is scaled by its view count.
FRAMES_DRAM_BYTES_PER_VIEW = (430.692608e6 + 6.068480e6) / 8


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value, dist=None, device=None):
    """The timed region of the slowest rank (max over ranks); identity on one rank."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, n_ranks, max_ms):
    """Units processed by all ranks per second of the slowest rank's timed region."""
    return n_ranks * units_per_rank / (max_ms / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


FRAMES_VIEWS, FRAMES_DISTINCT = 64, 4
FRAMES_WORKLOAD = (f"frames: {FRAMES_VIEWS} views of raw camera frames 1280x1024x40 (300x250x50 um, 8-bit, grains "
                   f"dark), {FRAMES_DISTINCT} distinct rendered views repeated (each 10k fog grains + 100 isotropic "
                   "tracks, Gaussian PSF 1.0 px / 0.8 frame, pulse 60-110, column and pixel gain pattern, noise 3), "
                   "one camera calibration, grain threshold 25, seeds 200-203, camera seed 1")

WORKLOADS = {
    "frames": FRAMES_WORKLOAD,
    "batched": WORKLOAD,
    "dense": ("dense: one view 300x300x50 um, 20,000 fog + 200 isotropic through-going tracks (gaps 3.3 um) "
              "+ 100 short tracks (range 10-50 um, gaps 1.6 um), jitter 0.05/0.3 um, int32 10 nm coords, "
              "seed window 5-20 um, tube 0.4 um, min hits 8, seed 2"),
    "pr1": ("PR1: one view 300x300x50 um, 2,000 fog + 20 isotropic tracks (gaps 3.3 um), jitter 0.05/0.3 um, "
            "int32 10 nm coords, seed window 5-20 um, tube 0.4 um, min hits 8, seed 1"),
    "stress": ("stress: one view 1000x1000x50 um, 1,000,000 fog + 5,000 isotropic tracks (20% short-range, "
               "gaps 1.6 um; through-going gaps 3.3 um), jitter 0.05/0.3 um, int32 10 nm coords, "
               "seed window 5-20 um, tube 0.4 um, min hits 8, seed 5"),
}


def make_workload(name="batched", n_batched=256):
    if name == "dense":
        views = [synth.dense()]
    elif name == "pr1":
        views = [synth.pr1()]
    elif name == "stress":
        views = [synth.stress()]
    else:
        views = synth.batched(n_views=256, seed=3)[:n_batched]
    xyz, offs = synth.concat(views)
    return views, xyz, offs


def workload_params(views, args=None):
    """Tracking parameters of the workload, with the variant flags of the command line."""
    if args is None:
        return synth.params(views[0].extent)
    return synth.params(views[0].extent, flags=args.flags, cut=tuple(int(c) for c in args.cut.split(",")))


def oracle_views_per_s(views, budget_s, start=0, args=None, threads=0):
    """Times the oracle on views[start:] until budget_s of wall time is used
    (threads: OpenMP threads of the counting, 0 = all cores)."""
    from oracle import oracle as O
    O.build()
    p = workload_params(views, args)
    done, seeds, t_used = 0, 0, 0.0
    k = start
    names = []
    while t_used < budget_s and done < len(views):
        v = views[k % len(views)]
        t0 = time.perf_counter()
        with O.Oracle(v.xyz, v.extent, p["seed_min"], p["seed_max"], p["tube_r"], p["min_hits"],
                      flags=p["flags"], cut=p["cut"]) as o:
            tr = o.find_tracks(nthreads=threads)
        t_used += time.perf_counter() - t0
        done += 1
        seeds += tr.n_seeds
        names.append(k % len(views))
        k += 1
    return done, seeds, t_used, names


# ---------------------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "stress":   # the oracle's smallest unit of work here takes about an hour
        print(json.dumps({"impl": "reference", "unavailable": "one stress view takes the oracle about an hour "
                                                              "(3,152 s on 8 host cores)"}), flush=True)
        return 0
    views, _, _ = make_workload(args.workload)
    cores = os.cpu_count()
    per_step = max(1.0, float(os.environ.get("ET_REF_STEP_S", "4")))
    k = 0
    for _ in range(args.warmup):
        d, _, _, _ = oracle_views_per_s(views, per_step / 4, start=k, args=args)
        k += d
    tot_v, tot_s, tot_t = 0, 0, 0.0
    for _ in range(args.steps):
        d, s, t, _ = oracle_views_per_s(views, per_step, start=k, args=args)
        k += d
        tot_v += d
        tot_s += s
        tot_t += t
    value = tot_v / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload],
                                            "parallelism": "oracle on host cores"},
            "seeds_per_s": tot_s / tot_t,
            "cpu_baseline": {"value": value, "unit": "views/s", "cores": cores, "kind": "oracle",
                             "sample": f"{tot_v} views of the {len(views)}-view step, consecutive from view 0, "
                                       f"~{per_step:.0f} s per step"},
            "e2e": {"value": value, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    from paper_1311_5334_gb300 import et

    ws, rank, local = dist_env()
    # the served sweep's views are drawn by spawned processes before any CUDA call
    served_pool = None
    if not args.no_extra and args.workload == "batched" and ws == 1:   # a one-GPU measurement
        served_pool = served_views_pool(args.served_views, seed=4)
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    views, xyz_h, offs = make_workload(args.workload, args.views)
    n_views = len(views)
    params = workload_params(views, args)
    # a dedicated stream: the legacy default stream (handle 0) would mean
    # "the context's own stream" to the library
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = et.Context(local)
    info = ctx.info()
    xyz_d = torch.from_numpy(xyz_h).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    batch = et.Batch(ctx, params)
    batch.set_profiling(True)
    tuned = None
    if args.cell:
        batch.set_tuning(tuple(int(c) for c in args.cell.split(",")), row_lists=args.rows,
                         ticket_origins=args.ticket_origins, assoc_window=args.assoc_window)
    batch.load(xyz_d, offs, stream=stream)
    if not args.cell:
        cell, ms = batch.autotune(stream=stream)
        tuned = {"cell": list(cell), "row_lists": batch.tuning["row_lists"],
                 "ticket_origins": batch.tuning["ticket_origins"], "ms_per_run": ms,
                 "how": "et_batch_autotune: fastest of 11 cell shapes, each with x rows and with x+y rows, "
                        "then 1, 2 or 4 seed origins per work ticket for that shape"}

    def step():
        batch.load(xyz_d, offs, stream=stream)
        batch.find(stream=stream, use_graph=True)

    for _ in range(max(args.warmup, 1)):
        step()
        batch.sync()
        flush.zero_()
    ref_stats = batch.stats()

    # timed region: per-step CUDA events on the launching stream, L2 flushed between steps
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t_wall0 = time.perf_counter()
    step_ms, tube_ms = [], []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        batch.sync()                       # status check (device idle afterwards)
        st = batch.stats()
        step_ms.append(e0.elapsed_time(e1))
        tube_ms.append(st["stage_ms"]["tube_count"])
        assert st["n_seeds"] == ref_stats["n_seeds"] and st["n_tracks"] == ref_stats["n_tracks"]
        flush.zero_()
    barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    total_ms = reduce_max(float(np.sum(step_ms)), dist, device="cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(n_views, ws, ms_per_step)
    seeds_per_s = whole_job_rate(ref_stats["n_seeds"], ws, ms_per_step)

    # roofline of the dominant kernel (tube counts): integer ALU issue, against
    # the nominal peak and, beside it, the device's measured integer issue rates
    tube_avg_ms = float(np.mean(tube_ms))
    int_rates = ctx.int_throughput()
    ops_tube = OPS_PER_TEST * ref_stats["n_tests"]
    ops = ops_tube + OPS_PER_PAIR_TEST * ref_stats["n_pair_tests"]
    achieved = ops / (tube_avg_ms / 1e3) / 1e12
    achieved_tube = ops_tube / (tube_avg_ms / 1e3) / 1e12
    peak = info["sm_count"] * 128 * 2070e6 / 1e12
    stage_ms = ref_stats["stage_ms"]
    # DRAM bytes of one tube-count launch (an ncu capture of this launch
    # configuration) over the same in-graph kernel time, against the measured
    # copy bandwidth: how far the kernel is from being bound by HBM
    run_key = tube_run_key(args.workload, n_views, ref_stats["cell"], batch.tuning if tuned else None,
                           rows=args.rows, ticket_origins=args.ticket_origins)
    traffic = TUBE_DRAM_BYTES.get(run_key)
    hbm = hbm_roofline(traffic, tube_avg_ms, measured_peaks())

    line_extra = {}
    if args.no_extra:
        plain_views_per_s = e2e_val = None
        h2d = d2h = 0
    else:
        tuning = (tuple(ref_stats["cell"]), batch.tuning["row_lists"] if tuned else args.rows,
                  batch.tuning["ticket_origins"] if tuned else args.ticket_origins)
        plain_views_per_s, e2e_val, h2d, d2h = extras(args, ctx, params, views, xyz_h, xyz_d, offs, stream, ws,
                                                      tuning)
    line = {"metric": METRIC, "value": value, "unit": "views/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": (WORKLOADS[args.workload] if args.workload != "batched" or n_views == 256
                                    else f"first {n_views} views of " + WORKLOADS[args.workload]),
                       "views_per_step": n_views,
                       "grains_per_step": int(offs[-1]),
                       "seeds_per_step": ref_stats["n_seeds"], "tube_tests_per_step": ref_stats["n_tests"],
                       "tube_hits_per_step": ref_stats["n_hits"],
                       "seed_window_tests_per_step": ref_stats["n_pair_tests"],
                       "candidate_efficiency": (ref_stats["n_hits"] / ref_stats["n_tests"]
                                                if ref_stats["n_tests"] else None),
                       "tracks_per_step": ref_stats["n_tracks"], "candidates_per_step": ref_stats["n_candidates"],
                       "candidate_members_per_step": ref_stats["n_members"],
                       "merge_rounds": ref_stats["merge_rounds"], "cell_units": list(ref_stats["cell"]),
                       "autotune": tuned,
                       "variant": {"flags": params["flags"], "cut": list(params["cut"])},
                       "l2": "flushed between timed steps (256 MiB write); inputs resident in HBM",
                       "parallelism": f"replicas: one {n_views}-view batch per rank x {ws}"},
            "seeds_per_s": seeds_per_s,
            "cm2_per_h": value * (1e-4 if args.workload == "stress" else VIEW_CM2) * 3600,
            "plain_views_per_s": plain_views_per_s,
            "stage_ms": stage_ms,
            "wall_s": wall,
            "roofline": {"bound": "alu", "kernel": "k_tube_count", "achieved": achieved, "peak": peak,
                         "unit": "Tops/s", "frac": achieved / peak,
                         "frac_tube_tests_only": achieved_tube / peak,
                         "traffic": traffic, "hbm": hbm,
                         "basis": f"({OPS_PER_TEST} int ops per tube test x {ref_stats['n_tests']} tests + "
                                  f"{OPS_PER_PAIR_TEST} per seed-window test x {ref_stats['n_pair_tests']} "
                                  f"window tests of the seed generator) / {tube_avg_ms:.3f} ms (in-graph "
                                  f"CUDA events of the one kernel that generates the seeds and counts their "
                                  f"tubes); peak = {info['sm_count']} SMs x 128 lanes x 2070 MHz",
                         "measured_int_tops": {k: v / 1e12 for k, v in int_rates.items()},
                         "frac_of_measured_mix": achieved / (int_rates["mix"] / 1e12),
                         "measured_how": "et_probe_int_throughput: xor+add (alu), a*a+z (mad) and both (mix) "
                                         "chains, 8 per thread, 2048 threads per SM, CUDA events"},
            "e2e": {"value": e2e_val, "unit": "views/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(ref_stats["kernel_launches"]) * args.steps,
            "clocks": clk}
    if served_pool is not None:
        line["served"] = served_sweep(ctx, params, served_pool)
        line["other_workloads"] = other_workloads(ctx, stream)
    line.update(line_extra)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.no_extra and args.workload == "stress":
        # one stress view is the oracle's smallest unit of work and takes it far
        # beyond any sampling budget (3,152 s on 8 x86 host cores for counting
        # and association, measured when its expected digests were written)
        line["cpu_baseline"] = {"value": None, "unit": "views/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "not run: one stress view takes the oracle about an hour"}
    elif rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.no_extra:
        budget = float(os.environ.get("ET_CPU_BASELINE_S", "15"))
        d, s, t, names = oracle_views_per_s(views, budget, args=args)
        line["cpu_baseline"] = {"value": d / t, "unit": "views/s", "cores": os.cpu_count(), "kind": "oracle",
                                "seeds_per_s": s / t,
                                "sample": f"views {names[0]}..{names[-1]} ({d} of {n_views}) of the step, "
                                          f"{t:.1f} s; counting parallel over all cores (OpenMP), "
                                          "merge and fit single-threaded"}
        # one host thread: the paper's CPU comparison basis (Section 3, Table 2)
        d1, s1, t1, names1 = oracle_views_per_s(views, budget / 2, args=args, threads=1)
        line["cpu_baseline_1thread"] = {"value": d1 / t1, "unit": "views/s", "cores": 1, "kind": "oracle",
                                        "seeds_per_s": s1 / t1,
                                        "views_per_s_at_the_step_mean": (s1 / t1) / (ref_stats["n_seeds"] / n_views),
                                        "sample": f"views {names1[0]}..{names1[-1]} ({d1} of {n_views}) "
                                                  f"of the step, {t1:.1f} s, one thread"}
    batch.close()
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


SERVED_RATES = (100, 200, 500, 1000, 2000, 5000)


def _served_view(arg):
    seed, i, n_fog = arg
    return synth.batched_view(seed, i, n_fog).xyz


def served_views_pool(n_views=10000, seed=4):
    """The served workload's views: n_views distinct views with the batched
    size law (seed 4), drawn in parallel by spawned worker processes (no CUDA
    state is inherited)."""
    import multiprocessing as mp
    sizes = synth.batched_sizes(n_views, seed)
    args = [(seed, i, int(nf)) for i, nf in enumerate(sizes)]
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        return pool.map(_served_view, args, chunksize=64)


def served_sweep(ctx, params, pool, budget_bytes=20 << 30):
    """The served configuration: len(pool) views arriving as a Poisson
    process at each rate of SERVED_RATES, under a device-memory budget."""
    out = {"views_per_rate": len(pool), "budget_bytes": budget_bytes,
           "pool": f"{len(pool)} distinct views, batched size law (lognormal, median 10k), seed 4", "rates": []}
    for rate in SERVED_RATES:
        out["rates"].append(served_run(ctx, params, pool, rate, len(pool), budget_bytes=budget_bytes))
    return out


def served_run(ctx, params, pool, rate, n_views, budget_bytes=20 << 30, max_batch=256, seed=4):
    """Poisson arrivals at `rate` views/s through et_server_submit / et_server_poll.
    pool: views (objects with .xyz) or int32 (n, 3) arrays, cycled.

    Latency of a view = result ready - its scheduled arrival (CLOCK_MONOTONIC on
    both sides), so a producer that falls behind does not hide queueing."""
    from paper_1311_5334_gb300 import et
    arrivals = synth.poisson_arrivals(n_views, rate, seed=seed)
    done = {}
    with ctx.server(params, budget_bytes, max_batch_views=max_batch) as srv:
        t0 = time.monotonic_ns() + 20_000_000
        sched = t0 + (arrivals * 1e9).astype(np.int64)
        busy = [0]

        def producer():
            for i in range(n_views):
                wait = int(sched[i]) - time.monotonic_ns()
                if wait > 0:
                    time.sleep(wait / 1e9)
                v = pool[i % len(pool)]
                while srv.submit(getattr(v, "xyz", v), tag=i) == et.BUSY:
                    busy[0] += 1
                    time.sleep(1e-4)

        th = threading.Thread(target=producer, daemon=True)
        th.start()
        while len(done) < n_views:
            for r in srv.poll(max_results=1024, timeout_us=50_000):
                if r.status != et.OK:
                    raise RuntimeError(f"served view {r.tag} failed with status {r.status}")
                done[int(r.tag)] = int(r.t_done_ns)
        th.join()
        sst = srv.stats()
    lat = np.array([(done[i] - sched[i]) / 1e6 for i in range(n_views)])
    span = (max(done.values()) - t0) / 1e9
    return {"rate_per_s": rate, "views": n_views, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "views_per_s": n_views / span, "busy_retries": busy[0],
            "micro_batches": sst["batches"], "peak_device_bytes": sst["peak_device_bytes"],
            "budget_bytes": budget_bytes}


def pinned_array(n, dtype):
    """A numpy array of n elements in page-locked host memory (through torch)."""
    import torch
    dt = np.dtype(dtype)
    buf = torch.empty(max(1, n) * dt.itemsize, dtype=torch.uint8).pin_memory()
    arr = buf.numpy().view(dt)[:n]
    pinned_array.keep.append(buf)
    return arr


pinned_array.keep = []


def other_workloads(ctx, stream, local=0):
    """The one-view workloads (PR1, dense, stress) in the same run: graph
    replay of the whole path on device-resident grains with the autotuner's
    choice for each view, CUDA events over K steps (enough for the clock
    sampler).  views/s, ms per step, stage times, ALU roofline fraction and
    the clocks seen."""
    import torch
    from paper_1311_5334_gb300 import et
    out = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for name, steps in (("pr1", 3000), ("dense", 800), ("stress", 5)):
        v = {"pr1": synth.pr1, "dense": synth.dense, "stress": synth.stress}[name]()
        p = synth.params(v.extent)
        xyz_d = torch.from_numpy(v.xyz).cuda()
        b = et.Batch(ctx, p)
        try:
            b.set_profiling(True)
            b.load(xyz_d, [0, v.n], stream=stream)
            cell, _ = b.autotune(stream=stream)
            for _ in range(3):
                b.load(xyz_d, [0, v.n], stream=stream)
                b.find(stream=stream, use_graph=True)
                b.sync()
            st = b.stats()
            clocks = ClockSampler(local)
            clocks.start()
            torch.cuda.synchronize()
            ms = 0.0
            for _ in range(steps):
                if name == "stress":
                    flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                b.load(xyz_d, [0, v.n], stream=stream)
                b.find(stream=stream, use_graph=True)
                e1.record(stream)
                if name == "stress":
                    b.sync()
                    ms += e0.elapsed_time(e1)
                else:
                    e1.synchronize()
                    ms += e0.elapsed_time(e1)
            b.sync()
            clk = clocks.stop()
            st2 = b.stats()
        finally:
            b.close()
        tube_ms = st2["stage_ms"]["tube_count"]
        ops = OPS_PER_TEST * st["n_tests"] + OPS_PER_PAIR_TEST * st["n_pair_tests"]
        peak = 152 * 128 * 2070e6
        out[name] = {"views_per_s": steps / (ms / 1e3), "ms_per_step": ms / steps, "grains": v.n,
                     "tuning": {"cell": list(cell), "row_lists": b.tuning["row_lists"],
                                "ticket_origins": b.tuning["ticket_origins"]},
                     "seeds": st["n_seeds"], "tracks": st["n_tracks"], "stage_ms": st2["stage_ms"],
                     "alu_frac": ops / (tube_ms / 1e3) / peak, "clocks": clk,
                     "l2": "flushed between steps" if name == "stress" else "view resident in L2 between steps"}
    return out


def extras(args, ctx, params, views, xyz_h, xyz_d, offs, stream, ws, tuning):
    """Plain one-view-per-launch form and the end-to-end (host buffers) form,
    both with the cell tuning of the timed batch."""
    import torch
    from paper_1311_5334_gb300 import et
    n_views = len(views)
    # plain form: one view per launch sequence, same views, device-resident
    plain = et.Batch(ctx, params)
    plain.set_tuning(tuning[0], row_lists=tuning[1], ticket_origins=tuning[2])
    plain_ms = 0.0
    n_plain = min(n_views, int(os.environ.get("ET_PLAIN_VIEWS", "256")))
    reps = max(1, min(50, 256 // n_plain))   # a short list of views is timed several times over
    for k in range(n_plain):
        o0, o1 = int(offs[k]), int(offs[k + 1])
        sub = xyz_d[o0:o1]
        # warm-up run of this view, settled by fetch: buffers grow to the view's
        # exact needs, so the timed run cannot overflow and skip work
        plain.load(sub, [0, o1 - o0], stream=stream)
        plain.find(stream=stream)
        plain.fetch()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for _ in range(reps):
            e0.record(stream)
            plain.load(sub, [0, o1 - o0], stream=stream)
            plain.find(stream=stream)
            e1.record(stream)
            plain.sync()
            plain_ms += e0.elapsed_time(e1)
    plain.close()
    plain_views_per_s = n_plain * reps / (plain_ms / 1e3)

    # e2e: host (pinned) grains in, tracks + members out, through the C ABI
    pinned = torch.from_numpy(xyz_h).pin_memory()
    host_view = pinned.numpy()
    eb = et.Batch(ctx, params)
    eb.set_tuning(tuning[0], row_lists=tuning[1], ticket_origins=tuning[2])
    eb.load(host_view, offs)
    eb.find(use_graph=True)
    tr, mem, voff = eb.fetch()
    # page-locked result buffers, reused every step as a serving client would
    out = (pinned_array(2 * len(tr) + 1024, et.TRACK_DTYPE), pinned_array(2 * len(mem) + 4096, np.int32),
           pinned_array(n_views + 1, np.int64))
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        eb.load(host_view, offs)
        eb.find(use_graph=True)
        tr, mem, voff = eb.fetch(out)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    eb.close()
    h2d = xyz_h.nbytes + offs.nbytes
    d2h = tr.nbytes + mem.nbytes + voff.nbytes + 2 * 256
    e2e_val = ws * n_views / e2e_s
    return plain_views_per_s, e2e_val, h2d, d2h



# ---------------------------------------------------------------------------- image front end

def make_frames_workload():
    """FRAMES_DISTINCT rendered views (one camera) and the shared calibration."""
    frs = [synth.frames_view(200 + k, n_fog=10000, n_through=100, camera_seed=1)[1]
           for k in range(FRAMES_DISTINCT)]
    return frs, frs[0].gain, frs[0].thr


def oracle_frames_per_s(frs, gain, thr, budget_s):
    """Times the oracle (filter + grain recognition) on the distinct views, cycled."""
    from oracle import oracle as O
    O.build()
    done, t_used, grains = 0, 0.0, 0
    while t_used < budget_s:
        fr = frs[done % len(frs)]
        t0 = time.perf_counter()
        f = O.frames_filter(fr.raw, gain, thr)
        g = O.frames_grains(f, synth.GRAIN_THRESHOLD, synth.PITCH_NUM, synth.PITCH_DEN)
        t_used += time.perf_counter() - t0
        grains += len(g[0])
        done += 1
    return done, t_used, grains


def run_frames_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    frs, gain, thr = make_frames_workload()
    per_step = max(1.0, float(os.environ.get("ET_REF_STEP_S", "4")))
    for _ in range(args.warmup):
        oracle_frames_per_s(frs, gain, thr, per_step / 4)
    tot_v, tot_t = 0, 0.0
    for _ in range(args.steps):
        d, t, _ = oracle_frames_per_s(frs, gain, thr, per_step)
        tot_v += d
        tot_t += t
    value = tot_v / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": FRAMES_WORKLOAD, "parallelism": "oracle on one host core"},
            "cpu_baseline": {"value": value, "unit": "views/s", "cores": 1, "kind": "oracle",
                             "sample": f"{tot_v} views (the {FRAMES_DISTINCT} distinct views cycled), "
                                       f"~{per_step:.0f} s per step, filter + recognition single-threaded"},
            "e2e": {"value": value, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_frames(args):
    import torch
    from paper_1311_5334_gb300 import et

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    frs, gain, thr = make_frames_workload()
    D, H, P = frs[0].raw.shape
    W = frs[0].width
    V = args.frames_views
    view_bytes = D * H * P
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = et.Context(local)
    distinct = [torch.from_numpy(fr.raw.reshape(-1)).cuda() for fr in frs]
    raw_d = torch.empty(V * view_bytes, dtype=torch.uint8, device="cuda")
    for k in range(V):
        raw_d[k * view_bytes:(k + 1) * view_bytes].copy_(distinct[k % len(distinct)])
    del distinct
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    fp = et.make_frame_params(W, H, D, synth.PITCH_NUM, synth.PITCH_DEN, synth.GRAIN_THRESHOLD, row_pitch=P)
    fr = et.Frames(ctx, fp, gain, thr)

    def step():
        fr.run(raw_d, n_views=V, stream=stream)

    for _ in range(max(args.warmup, 1)):
        step()
        fr.sync()
        flush.zero_()
    ref = fr.stats()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t_wall0 = time.perf_counter()
    step_ms, kern_ms = [], []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        fr.sync()
        st = fr.stats()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(st["kernel_ms"])
        assert st["n_grains"] == ref["n_grains"]
        flush.zero_()
    barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    total_ms = reduce_max(float(np.sum(step_ms)), dist, device="cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(V, ws, ms_per_step)

    # roofline of the recognition kernel: HBM.  Algorithmic bytes per launch:
    # the raw frames read once, the three per-pixel tables read once, and per
    # grain a sort key (8 B), an index (4 B) and a record (16 B) written.
    k_ms = float(np.mean(kern_ms))
    alg_bytes = V * view_bytes + 3 * H * W + 28 * ref["n_grains"]
    achieved = alg_bytes / (k_ms / 1e3) / 1e9
    peaks = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "of measured" if "hbm_gbs" in peaks else "of fallback"

    extra = {}
    if not args.no_extra:
        extra = frames_extras(args, ctx, fp, frs, gain, thr, raw_d, V, view_bytes, stream, ws)
    line = {"metric": METRIC, "value": value, "unit": "views/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": FRAMES_WORKLOAD.replace(f"{FRAMES_VIEWS} views", f"{V} views"),
                       "views_per_step": V, "bytes_per_step": V * view_bytes,
                       "voxels_per_step": ref["n_voxels"], "candidates_per_step": ref["n_candidates"],
                       "grains_per_step": ref["n_grains"],
                       "l2": "inputs (3.4 GB) larger than L2; also flushed between timed steps (256 MiB write)",
                       "parallelism": f"replicas: one {V}-view batch per rank x {ws}"},
            "kernel_ms": k_ms,
            "wall_s": wall,
            "roofline": {"bound": "hbm", "kernel": "k_recognize", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": FRAMES_DRAM_BYTES_PER_VIEW * V if FRAMES_DRAM_BYTES_PER_VIEW else None,
                         "basis": f"{alg_bytes / 1e9:.3f} GB per launch (raw frames once, tables once, "
                                  f"28 B per grain written) / {k_ms:.3f} ms (CUDA events); peak {peak_src} "
                                  "copy bandwidth"},
            "gpu_launches": int(ref["kernel_launches"]) * args.steps,
            "clocks": clk}
    line.update(extra)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not args.no_extra:
        budget = float(os.environ.get("ET_CPU_BASELINE_S", "15"))
        d, t, _ = oracle_frames_per_s(frs, gain, thr, budget)
        line["cpu_baseline"] = {"value": d / t, "unit": "views/s", "cores": 1, "kind": "oracle",
                                "sample": f"{d} views (the {FRAMES_DISTINCT} distinct views cycled), {t:.1f} s, "
                                          "filter + recognition single-threaded"}
    fr.close()
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def frames_extras(args, ctx, fp, frs, gain, thr, raw_d, V, view_bytes, stream, ws):
    """End to end from pinned host frames to host grains, and the chain from
    raw frames to tracks on the device."""
    import torch
    from paper_1311_5334_gb300 import et
    pinned = torch.empty(V * view_bytes, dtype=torch.uint8).pin_memory()
    pinned.copy_(raw_d.cpu())
    host = pinned.numpy()
    fr = et.Frames(ctx, fp, gain, thr)
    fr.run(host, n_views=V)
    xyz, pulse, voff = fr.fetch()
    # page-locked result buffers, reused every step as a serving client would
    n_cap = 2 * len(xyz) + 1024
    out = (pinned_array(3 * n_cap, np.int32).reshape(n_cap, 3), pinned_array(n_cap, np.int32),
           pinned_array(V + 1, np.int64))
    steps = max(3, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        fr.run(host, n_views=V)
        xyz, pulse, voff = fr.fetch(out)
    e2e_s = (time.perf_counter() - t0) / steps
    d2h = xyz.nbytes + pulse.nbytes + voff.nbytes + 64

    # frames -> grains -> tracks, device resident (one track-finding batch of V views)
    params = synth.params(synth.FRAME_EXTENT)
    b = et.Batch(ctx, params)
    b.set_tuning((150, 600, 600), row_lists=1)

    def chain():
        fr.run(raw_d, n_views=V, stream=stream)
        fr.to_batch(b, stream=stream)
        b.find(stream=stream)
        return b.fetch()

    tr, mem, toff = chain()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        tr, mem, toff = chain()
    chain_s = (time.perf_counter() - t0) / steps
    b.close()
    fr.close()
    return {"e2e": {"value": ws * V / e2e_s, "unit": "views/s", "h2d_bytes_per_step": int(V * view_bytes),
                    "d2h_bytes_per_step": int(d2h)},
            "pipeline": {"value": ws * V / chain_s, "unit": "views/s", "tracks_per_step": int(len(tr)),
                         "what": "raw frames (device) -> grains -> batched track finding -> tracks to host, "
                                 "wall clock per step"}}

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="time only the device-resident step (no plain/e2e/cpu baseline); for profilers")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="batched")
    ap.add_argument("--views", type=int, default=256,
                    help="batched workload: time only its first N views (smaller profiling captures)")
    ap.add_argument("--cell", default="", help="cell edges x,y,z in coordinate units (default: automatic)")
    ap.add_argument("--rows", type=int, default=1, help="with --cell: 1 = x-row cell list, 2 = x and y rows")
    ap.add_argument("--ticket-origins", type=int, default=0,
                    help="with --cell: seed origins per work ticket (1, 2 or 4; 0 = automatic)")
    ap.add_argument("--assoc-window", type=int, default=0,
                    help="with --cell: candidates per association window (0 = automatic)")
    ap.add_argument("--served-views", type=int, default=10000,
                    help="distinct views of the served sweep (one run per rate of 100..5000 views/s)")
    ap.add_argument("--flags", type=int, default=0,
                    help="et_params.flags: 1 single-pass association, 2 angle cut (tracking workloads)")
    ap.add_argument("--cut", default="0,0,0", help="angle cut base,slope,tan_max (with --flags 2)")
    ap.add_argument("--frames-views", type=int, default=FRAMES_VIEWS,
                    help="views per step of the frames workload (smaller for profiler captures)")
    ap.add_argument("--served-sweep", action="store_true",
                    help="only the served form: rates 100..5000 views/s over 10,000 views (seed 4)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "frames":
        return run_frames_reference(args) if args.impl == "reference" else run_frames(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.served_sweep:
        return run_served_sweep(args)
    return run_ours(args)


def run_served_sweep(args):
    """The served configuration: 10,000 views (size law of the batched views,
    seed 4) arriving as a Poisson process, rate swept 100-5,000 views/s, under a
    20 GB device-memory budget.  One JSON line per rate."""
    import torch
    from paper_1311_5334_gb300 import et
    pool = served_views_pool(args.served_views, seed=4)
    torch.cuda.set_device(0)
    params = synth.params((30000, 30000, 5000))
    with et.Context(0) as ctx:
        for rate in SERVED_RATES:
            r = served_run(ctx, params, pool, rate, len(pool))
            r.update({"metric": "served view latency", "pool": f"{len(pool)} distinct views (seed 4)"})
            print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
