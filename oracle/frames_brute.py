"""Whole-array restatement of the image front end (numpy), for pinning the C oracle.

TEST INFRASTRUCTURE ONLY.  It re-derives the filtering and the 3D grain
recognition of Section 2 of the paper as whole-array operations on a padded
stack instead of the per-voxel loops of frames.c, and shares nothing with it:

* filtering: f = max(0, min(255, floor(((255 - raw) g + 64) / 128)) - t) per
  pixel gain g (128 = 1.0) and threshold t, the same for every frame;
* a voxel p with f(p) > T defines a grain iff, over its 26 neighbours q inside
  the stack, f(q) < f(p) for q before p in raster order (z, y, x) and
  f(q) <= f(p) for q after it;
* the grain lies at the pulse-height weighted centroid of the 3 x 3 x 3
  neighbourhood, voxel i of axis k at i * num[k] / den[k] units, rounded half
  up (exact rational arithmetic with Python integers).
"""
from __future__ import annotations

from fractions import Fraction
import math

import numpy as np


def filter_stack(raw, gain, thr):
    """raw uint8 [D][H][W] (no row padding), gain / thr uint8 [H][W]."""
    inv = 255 - raw.astype(np.int64)
    v = (inv * gain.astype(np.int64)[None] + 64) // 128
    v = np.minimum(v, 255) - thr.astype(np.int64)[None]
    return np.maximum(v, 0).astype(np.uint8)


def grains(f, threshold, num, den):
    """(xyz int64 [n][3], pulse int64 [n], voxel int64 [n]) in raster order."""
    f = np.asarray(f, dtype=np.int64)
    D, H, W = f.shape
    # absent voxels are -1: never above a candidate (f > T >= 0), weight 0 below
    pad = np.full((D + 2, H + 2, W + 2), -1, dtype=np.int64)
    pad[1:-1, 1:-1, 1:-1] = f
    is_max = f > threshold
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz == dy == dx == 0:
                    continue
                q = pad[1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
                earlier = (dz, dy, dx) < (0, 0, 0)
                is_max &= (q < f) if earlier else (q <= f)
    zs, ys, xs = np.nonzero(is_max)   # C order = raster order (z, y, x)
    w = np.maximum(pad, 0)
    out_xyz, out_pulse, out_vox = [], [], []
    for z, y, x in zip(zs.tolist(), ys.tolist(), xs.tolist()):
        box = w[z:z + 3, y:y + 3, x:x + 3]   # padded indices z..z+2 = voxels z-1..z+1
        s = int(box.sum())
        sz = sum(int(box[k].sum()) * (z - 1 + k) for k in range(3))
        sy = sum(int(box[:, k].sum()) * (y - 1 + k) for k in range(3))
        sx = sum(int(box[:, :, k].sum()) * (x - 1 + k) for k in range(3))
        coord = []
        for sk, nk, dk in ((sx, num[0], den[0]), (sy, num[1], den[1]), (sz, num[2], den[2])):
            c = Fraction(sk * nk, s * dk)
            coord.append(math.floor(c + Fraction(1, 2)))
        out_xyz.append(coord)
        out_pulse.append(s)
        out_vox.append((z * H + y) * W + x)
    return (np.array(out_xyz, dtype=np.int64).reshape(-1, 3), np.array(out_pulse, dtype=np.int64),
            np.array(out_vox, dtype=np.int64))
