"""Seeded synthetic grain clouds for one or many emulsion views.

This module only draws inputs: it holds none of the track-finding arithmetic
and is shared by the CUDA path's tests and benchmark and by the CPU oracle's
tests.  Everything is deterministic given the seed.

Geometry and physics follow Section 2 of the paper: a view is a slab of
emulsion some 300 um wide and 50 um deep, grains are 3D points (the output of
3D grain recognition), and a minimum-ionising track leaves about 42 grains per
100 um (Section 3, sensitivity measurement).  The workloads used here are:

* PR1      -- 300x300x50 um, 2,000 fog grains + 20 isotropic through-going
              tracks, grain gaps exponential with mean 3.3 um.
* dense    -- same view, 20,000 fog + 200 through-going tracks (gaps 3.3 um)
              + 100 short tracks (range U(10, 50) um starting and stopping
              inside the layer, gaps 1.6 um: heavily ionising).
* batched  -- 256 views whose fog count is lognormal (median 10k, sigma 0.6,
              redrawn until inside [2k, 50k]) with round(1 % of it) tracks.
* stress   -- one 1000x1000x50 um view, 1,000,000 fog + 5,000 tracks, 20 % of
              them short.

Coordinates are int32 in 10 nm units; the jitter is N(0, 0.05 um) in x, y and
N(0, 0.3 um) in z, applied before rounding and clamping into the view.  No two
grains share coordinates: a duplicate is redrawn (fog) or re-jittered (track).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

UM = 100  # integer units per micrometre (1 unit = 10 nm)

# Tracking parameters of all workloads, in units (seed window 5-20 um,
# tube radius 0.4 um, at least 8 grains).
SEED_MIN = 500
SEED_MAX = 2000
TUBE_R = 40
MIN_HITS = 8


@dataclasses.dataclass
class View:
    xyz: np.ndarray          # (N, 3) int32, units of 10 nm
    label: np.ndarray        # (N,) int32: track index, or -1 for fog
    extent: tuple            # (Ex, Ey, Ez) in units; coordinates lie in [0, E)
    n_tracks: int
    truth: np.ndarray = None   # (n_tracks, 6): a point (um) and the unit direction of each track's line

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


def params(extent, seed_min=SEED_MIN, seed_max=SEED_MAX, tube_r=TUBE_R, min_hits=MIN_HITS, flags=0,
           cut=(0, 0, 0)):
    return dict(extent=tuple(int(e) for e in extent), seed_min=int(seed_min),
                seed_max=int(seed_max), tube_r=int(tube_r), min_hits=int(min_hits), flags=int(flags),
                cut=tuple(int(c) for c in cut))


def _isotropic(rng, k):
    cos_t = rng.uniform(-1.0, 1.0, k)
    phi = rng.uniform(0.0, 2.0 * math.pi, k)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def _chord(p, d, e_um):
    """Parameter interval [t0, t1] over which p + t d stays inside [0, e]."""
    t0, t1 = -math.inf, math.inf
    for a in range(3):
        if abs(d[a]) < 1e-15:
            continue
        ta = (0.0 - p[a]) / d[a]
        tb = (e_um[a] - p[a]) / d[a]
        t0 = max(t0, min(ta, tb))
        t1 = min(t1, max(ta, tb))
    return t0, t1


def _track_points(rng, p, d, t_start, t_end, gap_um, first_at_start):
    ts = []
    t = t_start if first_at_start else t_start + rng.exponential(gap_um)
    while t <= t_end:
        ts.append(t)
        t += rng.exponential(gap_um)
    if not ts:
        return np.zeros((0, 3))
    ts = np.asarray(ts)
    return p[None, :] + ts[:, None] * d[None, :]


def _to_units(rng, pts_um, extent, jitter_xy_um, jitter_z_um):
    n = pts_um.shape[0]
    jit = np.empty((n, 3))
    jit[:, 0:2] = rng.normal(0.0, jitter_xy_um, (n, 2))
    jit[:, 2] = rng.normal(0.0, jitter_z_um, n)
    q = np.rint((pts_um + jit) * UM).astype(np.int64)
    hi = np.asarray(extent, dtype=np.int64) - 1
    return np.clip(q, 0, hi)


def _pack(xyz):
    x = xyz[:, 0].astype(np.int64)
    y = xyz[:, 1].astype(np.int64)
    z = xyz[:, 2].astype(np.int64)
    return (x << 42) | (y << 21) | z


def make_view(seed, extent=(300 * UM, 300 * UM, 50 * UM), n_fog=2000, n_through=20,
              n_short=0, gap_through_um=3.3, gap_short_um=1.6,
              short_range_um=(10.0, 50.0), jitter_xy_um=0.05, jitter_z_um=0.3,
              rng=None) -> View:
    """Draw one view: uniform fog plus straight isotropic tracks."""
    if rng is None:
        rng = np.random.default_rng(seed)
    extent = tuple(int(e) for e in extent)
    e_um = np.asarray(extent, dtype=np.float64) / UM
    ext64 = np.asarray(extent, dtype=np.int64)

    pieces, labels = [], []
    fog = rng.integers(0, ext64, size=(n_fog, 3), dtype=np.int64)
    pieces.append(fog)
    labels.append(np.full(n_fog, -1, dtype=np.int32))

    track_raw = []  # per track: (points in um) for re-jitter on duplicates
    truth = []      # per track: point and direction of its line (um)
    dirs = _isotropic(rng, n_through + n_short)
    for k in range(n_through):
        p = rng.uniform(0.0, 1.0, 3) * e_um
        d = dirs[k]
        t0, t1 = _chord(p, d, e_um)
        track_raw.append(_track_points(rng, p, d, t0, t1, gap_through_um, False))
        truth.append(np.concatenate([p, d]))
    for k in range(n_short):
        p = rng.uniform(0.0, 1.0, 3) * e_um
        d = dirs[n_through + k]
        rng_um = rng.uniform(*short_range_um)
        _, t1 = _chord(p, d, e_um)
        track_raw.append(_track_points(rng, p, d, 0.0, min(rng_um, t1), gap_short_um, True))
        truth.append(np.concatenate([p, d]))

    for k, pts in enumerate(track_raw):
        pieces.append(_to_units(rng, pts, extent, jitter_xy_um, jitter_z_um))
        labels.append(np.full(pts.shape[0], k, dtype=np.int32))

    xyz = np.concatenate(pieces, axis=0)
    label = np.concatenate(labels)
    raw_all = np.concatenate([np.zeros((n_fog, 3))] + track_raw, axis=0)

    # Resolve coincident coordinates: keep the first, redraw the others.
    for _ in range(1000):
        key = _pack(xyz)
        _, first = np.unique(key, return_index=True)
        dup = np.ones(xyz.shape[0], dtype=bool)
        dup[first] = False
        idx = np.nonzero(dup)[0]
        if idx.size == 0:
            break
        for i in idx:
            if label[i] < 0:
                xyz[i] = rng.integers(0, ext64, size=3, dtype=np.int64)
            else:
                xyz[i] = _to_units(rng, raw_all[i:i + 1], extent, jitter_xy_um, jitter_z_um)[0]
    else:  # pragma: no cover
        raise RuntimeError("could not resolve duplicate grains")

    perm = rng.permutation(xyz.shape[0])
    return View(xyz=np.ascontiguousarray(xyz[perm].astype(np.int32)),
                label=np.ascontiguousarray(label[perm]), extent=extent,
                n_tracks=n_through + n_short, truth=np.array(truth, dtype=np.float64).reshape(-1, 6))


# ---------------------------------------------------------------- workloads

def pr1(seed=1) -> View:
    return make_view(seed, n_fog=2000, n_through=20)


def dense(seed=2) -> View:
    return make_view(seed, n_fog=20000, n_through=200, n_short=100)


def lognormal_sizes(rng, k, median=10000, sigma=0.6, lo=2000, hi=50000):
    out = np.empty(k, dtype=np.int64)
    for i in range(k):
        while True:
            v = int(round(math.exp(rng.normal(math.log(median), sigma))))
            if lo <= v <= hi:
                out[i] = v
                break
    return out


def batched(n_views=256, seed=3, sizes=None):
    """Views with lognormal fog counts and round(1 %) isotropic tracks each."""
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = lognormal_sizes(rng, n_views)
    return [batched_view(seed, i, int(nf)) for i, nf in enumerate(sizes)]


def batched_view(seed, i, n_fog):
    """View i of batched(seed=seed), whose fog count is n_fog (drawn by the
    batch): views can be drawn independently, e.g. in parallel."""
    sub = np.random.default_rng([seed, i])
    return make_view(None, n_fog=int(n_fog), n_through=int(round(0.01 * n_fog)), rng=sub)


def batched_sizes(n_views, seed):
    """The fog counts batched(n_views, seed) draws."""
    return lognormal_sizes(np.random.default_rng(seed), n_views)


def stress(seed=5, n_fog=1_000_000, n_tracks=5000, short_frac=0.2) -> View:
    n_short = int(round(short_frac * n_tracks))
    return make_view(seed, extent=(1000 * UM, 1000 * UM, 50 * UM), n_fog=n_fog,
                     n_through=n_tracks - n_short, n_short=n_short)


def poisson_arrivals(n, rate_per_s, seed=4):
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    rng = np.random.default_rng([seed, int(rate_per_s)])
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))


def concat(views):
    """Concatenate views: (xyz (sum N, 3) int32, offsets (V+1,) int64)."""
    offs = np.zeros(len(views) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([v.n for v in views])
    xyz = np.concatenate([v.xyz for v in views], axis=0) if views else np.zeros((0, 3), np.int32)
    return np.ascontiguousarray(xyz, dtype=np.int32), offs


# ---------------------------------------------------------------- raw frames
#
# The camera digitises a view of 300 x 250 x 50 um into 1280 x 1024 pixels and
# 40 frames (Section 2).  Pixel pitch in 10 nm units, as exact fractions:
# x 30000 / 1280 = 375 / 16, y 25000 / 1024 = 3125 / 128, z 5000 / 40 = 125.
FRAME_W, FRAME_H, FRAME_D = 1280, 1024, 40
FRAME_EXTENT = (300 * UM, 250 * UM, 50 * UM)
PITCH_NUM = (375, 3125, 125)
PITCH_DEN = (16, 128, 1)
GRAIN_THRESHOLD = 25


@dataclasses.dataclass
class Frames:
    raw: np.ndarray      # uint8 [D][H][row_pitch]; grains are dark
    gain: np.ndarray     # uint8 [H][W] per-pixel gain, 128 = 1.0
    thr: np.ndarray      # uint8 [H][W] per-pixel threshold
    width: int

    @property
    def shape(self):
        return (self.raw.shape[0], self.raw.shape[1], self.width)


def render(px, py, pz, amp, shape, seed, row_pitch=None, psf_xy=1.0, psf_z=0.8, dark=55.0,
           noise=3.0, col_sigma=0.08, px_sigma=0.03, margin=10, quantum=None, camera_seed=None):
    """Raw frames of grains at voxel positions (px, py, pz) with pulse heights amp.

    Each grain is a Gaussian blob (sigma psf_xy pixels, psf_z frames).  A pixel
    of sensitivity s (column pattern: the vertical lines of a raw frame, plus a
    per-pixel term) records darkness s * (dark + signal + noise); the raw value
    is 255 minus that, rounded and clipped.  quantum rounds the darkness to
    multiples of it first (many equal neighbours).  The calibration returned
    with the frames: gain = 128 / s and a threshold at the pixel's corrected
    background plus margin.  Rows are row_pitch >= W bytes; the padding holds
    random bytes.  camera_seed (default: seed) draws the sensitivity pattern,
    so views rendered with one camera_seed share one calibration.
    """
    D, H, W = shape
    row_pitch = W if row_pitch is None else int(row_pitch)
    rng = np.random.default_rng(seed)
    cam = np.random.default_rng(seed if camera_seed is None else camera_seed)
    col = np.clip(cam.standard_normal(W), -2.5, 2.5)
    s = 1.0 + col_sigma * col[None, :] + px_sigma * np.clip(cam.standard_normal((H, W)), -3.0, 3.0)
    gain = np.clip(np.rint(128.0 / s), 0, 255).astype(np.uint8)
    thr = np.clip(np.rint(dark * s * gain / 128.0) + margin, 0, 255).astype(np.uint8)

    sig = np.zeros(D * H * W, dtype=np.float32)
    px, py, pz = (np.asarray(a, dtype=np.float64) for a in (px, py, pz))
    amp = np.asarray(amp, dtype=np.float64)
    if px.size:
        oz, oy, ox = np.meshgrid(np.arange(-2, 3), np.arange(-3, 4), np.arange(-3, 4), indexing="ij")
        ox, oy, oz = ox.ravel(), oy.ravel(), oz.ravel()
        ix = np.rint(px)[:, None].astype(np.int64) + ox[None]
        iy = np.rint(py)[:, None].astype(np.int64) + oy[None]
        iz = np.rint(pz)[:, None].astype(np.int64) + oz[None]
        wgt = amp[:, None] * np.exp(-((ix - px[:, None]) ** 2 + (iy - py[:, None]) ** 2) / (2 * psf_xy ** 2)
                                    - (iz - pz[:, None]) ** 2 / (2 * psf_z ** 2))
        ok = (ix >= 0) & (ix < W) & (iy >= 0) & (iy < H) & (iz >= 0) & (iz < D)
        np.add.at(sig, ((iz * H + iy) * W + ix)[ok], wgt[ok].astype(np.float32))
    sig = sig.reshape(D, H, W)
    sig += np.float32(noise) * rng.standard_normal((D, H, W), dtype=np.float32)
    darkness = s.astype(np.float32)[None] * (np.float32(dark) + sig)
    if quantum:
        darkness = np.float32(quantum) * np.rint(darkness / np.float32(quantum))
    img = np.clip(np.rint(255.0 - darkness), 0, 255).astype(np.uint8)
    raw = np.empty((D, H, row_pitch), dtype=np.uint8)
    raw[:, :, :W] = img
    if row_pitch > W:
        raw[:, :, W:] = rng.integers(0, 256, (D, H, row_pitch - W), dtype=np.uint8)
    return Frames(raw=raw, gain=gain, thr=thr, width=W)


def frames_view(seed, n_fog=10000, n_through=100, n_short=0, row_pitch=None, amp=(60.0, 110.0),
                camera_seed=None):
    """One full 1280 x 1024 x 40 view: the grains of make_view on the camera's
    300 x 250 x 50 um volume, rendered into raw frames.  Returns (View, Frames)."""
    v = make_view(seed, extent=FRAME_EXTENT, n_fog=n_fog, n_through=n_through, n_short=n_short)
    rng = np.random.default_rng([seed, 7])
    xyz = v.xyz.astype(np.float64)
    px = xyz[:, 0] * PITCH_DEN[0] / PITCH_NUM[0]
    py = xyz[:, 1] * PITCH_DEN[1] / PITCH_NUM[1]
    pz = xyz[:, 2] * PITCH_DEN[2] / PITCH_NUM[2]
    a = rng.uniform(amp[0], amp[1], v.n)
    fr = render(px, py, pz, a, (FRAME_D, FRAME_H, FRAME_W), seed=[seed, 8], row_pitch=row_pitch,
                camera_seed=camera_seed)
    return v, fr


def random_blobs(shape, n, seed, row_pitch=None, amp=(40.0, 120.0), **kw):
    """n grains at uniform random voxel positions of a stack of the given shape."""
    D, H, W = shape
    rng = np.random.default_rng(seed)
    px = rng.uniform(-0.5, W - 0.5, n)
    py = rng.uniform(-0.5, H - 0.5, n)
    pz = rng.uniform(-0.5, D - 0.5, n)
    a = rng.uniform(amp[0], amp[1], n)
    return render(px, py, pz, a, shape, seed=[seed, 1], row_pitch=row_pitch, **kw)
