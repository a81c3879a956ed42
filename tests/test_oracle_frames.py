"""Pins for the CPU oracle of the image front end (filtering and 3D grain
recognition, Section 2 of the paper), checked without the CUDA path.

* hand-worked examples (tests/golden/frames_worked.json);
* an independent whole-array restatement (oracle/frames_brute.py) on small
  stacks, with many equal neighbours, row padding and grains on the faces;
* closed forms of the filter (pure inversion, zero gain, saturation) and its
  monotonicity in the raw value for every gain;
* an isolated symmetric blob sits exactly at its centre voxel; single-voxel
  grains at known positions are recovered exactly;
* translation by whole pitch periods shifts the grain coordinates exactly;
* a tie between two equal neighbours yields one grain, the earlier voxel.
"""
import json
import os

import numpy as np
import pytest

from oracle import frames_brute as FB
from paper_1311_5334_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "frames_worked.json")
NUM, DEN = synth.PITCH_NUM, synth.PITCH_DEN


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_golden_filter(oracle_mod):
    g = _golden()["filter"]
    raw = np.array(g["raw"], dtype=np.uint8).reshape(1, 1, -1)
    gain = np.array(g["gain"], dtype=np.uint8).reshape(1, -1)
    thr = np.array(g["thr"], dtype=np.uint8).reshape(1, -1)
    f = oracle_mod.frames_filter(raw, gain, thr)
    assert f.ravel().tolist() == g["expected"]


def test_golden_grains(oracle_mod):
    g = _golden()["grains"]
    D, H, W = g["shape_dhw"]
    f = np.zeros((D, H, W), dtype=np.uint8)
    for e in g["nonzero"]:
        x, y, z = e["xyz"]
        f[z, y, x] = e["f"]
    xyz, pulse, vox = oracle_mod.frames_grains(f, g["threshold"], g["pitch_num"], g["pitch_den"])
    got = [{"voxel": int(v), "xyz": [int(c) for c in p], "pulse": int(s)} for p, s, v in zip(xyz, pulse, vox)]
    assert got == g["expected"]


@pytest.mark.parametrize("case", range(6))
def test_restatement_agrees(oracle_mod, case):
    shapes = [(6, 30, 40), (1, 25, 33), (2, 17, 64), (9, 40, 23), (5, 64, 48), (3, 8, 16)]
    D, H, W = shapes[case]
    pitch = W + (0 if case % 2 else 16 - W % 16 if W % 16 else 16)
    quantum = 16 if case in (2, 4) else None   # coarse levels: many equal neighbours
    fr = synth.random_blobs((D, H, W), n=max(4, D * H * W // 400), seed=100 + case, row_pitch=pitch,
                            quantum=quantum)
    f = oracle_mod.frames_filter(fr.raw, fr.gain, fr.thr)
    assert np.array_equal(f, FB.filter_stack(np.ascontiguousarray(fr.raw[:, :, :W]), fr.gain, fr.thr))
    for T in (0, 12, 25):
        a = oracle_mod.frames_grains(f, T, NUM, DEN)
        b = FB.grains(f, T, NUM, DEN)
        assert len(a[0]) == len(b[0])
        for u, v in zip(a, b):
            assert np.array_equal(u.astype(np.int64), v)


def test_filter_closed_forms(oracle_mod):
    raw = np.arange(256, dtype=np.uint8).reshape(1, 1, 256)
    one = np.full((1, 256), 128, dtype=np.uint8)
    zero = np.zeros((1, 256), dtype=np.uint8)
    # gain 1.0, no threshold: the filter is the inversion 255 - raw
    assert np.array_equal(oracle_mod.frames_filter(raw, one, zero).ravel(), 255 - np.arange(256))
    # gain 0: nothing survives
    assert not oracle_mod.frames_filter(raw, zero, zero).any()
    # gain 255 (1.99): saturates at 255 for raw <= 127 ((128 * 255 + 64) / 128 = 255.5);
    # raw 128 gives (127 * 255 + 64) / 128 = 253.5 -> 253
    f = oracle_mod.frames_filter(raw, np.full((1, 256), 255, np.uint8), zero).ravel().astype(int)
    assert (f[:128] == 255).all() and f[128] == 253 and f[255] == 0


def test_filter_monotone_in_raw(oracle_mod):
    # every gain, a few thresholds: f never increases with the raw value
    raw = np.tile(np.arange(256, dtype=np.uint8), (256, 1)).reshape(1, 256, 256)
    gain = np.tile(np.arange(256, dtype=np.uint8)[:, None], (1, 256))
    for t in (0, 7, 200):
        f = oracle_mod.frames_filter(raw, gain, np.full((256, 256), t, np.uint8))[0].astype(int)
        assert (np.diff(f, axis=1) <= 0).all()


def _blob(shape, centre, profile):
    f = np.zeros(shape, dtype=np.uint8)
    z, y, x = centre
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                f[z + dz, y + dy, x + dx] = profile[abs(dz) + abs(dy) + abs(dx)]
    return f


def test_symmetric_blob_at_centre(oracle_mod):
    # a blob symmetric about its peak has its centre of mass on the peak
    f = _blob((5, 9, 11), (2, 4, 5), [90, 40, 20, 5])
    xyz, pulse, vox = oracle_mod.frames_grains(f, 25, NUM, DEN)
    assert len(xyz) == 1
    exact = [5 * NUM[0] / DEN[0], 4 * NUM[1] / DEN[1], 2 * NUM[2] / DEN[2]]
    assert xyz[0].tolist() == [int(np.floor(e + 0.5)) for e in exact]
    assert pulse[0] == 90 + 6 * 40 + 12 * 20 + 8 * 5
    assert vox[0] == (2 * 9 + 4) * 11 + 5


def test_single_voxel_grains(oracle_mod):
    rng = np.random.default_rng(5)
    D, H, W = 7, 40, 48
    f = np.zeros((D, H, W), dtype=np.uint8)
    pts = set()
    while len(pts) < 30:
        p = (int(rng.integers(D)), int(rng.integers(H)), int(rng.integers(W)))
        if all(max(abs(p[0] - q[0]), abs(p[1] - q[1]), abs(p[2] - q[2])) > 1 for q in pts):
            pts.add(p)
    for p in pts:
        f[p] = 200
    xyz, pulse, vox = oracle_mod.frames_grains(f, 25, NUM, DEN)
    want = sorted(pts)   # raster order = (z, y, x) order
    assert [(int(v) // (W * H), (int(v) // W) % H, int(v) % W) for v in vox] == want
    for (z, y, x), c in zip(want, xyz):
        # exact voxel position, rounded half up
        assert c.tolist() == [(2 * x * NUM[0] + DEN[0]) // (2 * DEN[0]), (2 * y * NUM[1] + DEN[1]) // (2 * DEN[1]),
                              (2 * z * NUM[2] + DEN[2]) // (2 * DEN[2])]
    assert (pulse == 200).all()


def test_translation_by_pitch_periods(oracle_mod):
    # shifting the stack by (16, 128, 1) voxels shifts every grain by exactly
    # (375, 3125, 125) units, the pitch being 375/16, 3125/128 and 125
    fr = synth.random_blobs((6, 40, 60), n=25, seed=9)
    f = oracle_mod.frames_filter(fr.raw, fr.gain, fr.thr)
    big = np.zeros((6 + 1, 40 + 128, 60 + 16), dtype=np.uint8)
    big[1:, 128:, 16:] = f
    a = oracle_mod.frames_grains(f, 25, NUM, DEN)
    b = oracle_mod.frames_grains(big, 25, NUM, DEN)
    # grains touching the original faces see absent neighbours there and zeros in the
    # shifted copy; with zero weight both give the same result
    assert len(a[0]) == len(b[0])
    assert np.array_equal(b[0], a[0] + np.array([375, 3125, 125], dtype=np.int32))
    assert np.array_equal(a[1], b[1])


def test_tie_takes_the_earlier_voxel(oracle_mod):
    # two equal neighbours along z, y or x: only the first in raster order is a grain
    for axis in range(3):
        f = np.zeros((4, 4, 4), dtype=np.uint8)
        p, q = [1, 1, 1], [1, 1, 1]
        q[axis] = 2
        f[tuple(p)] = 77
        f[tuple(q)] = 77
        xyz, pulse, vox = oracle_mod.frames_grains(f, 25, NUM, DEN)
        assert len(vox) == 1 and vox[0] == (p[0] * 4 + p[1]) * 4 + p[2]
        assert pulse[0] == 154


def test_full_view_counts(oracle_mod):
    # a full 1280 x 1024 x 40 view: most planted grains are found, none twice
    v, fr = synth.frames_view(3, n_fog=4000, n_through=40)
    f = oracle_mod.frames_filter(fr.raw, fr.gain, fr.thr)
    xyz, pulse, vox = oracle_mod.frames_grains(f, synth.GRAIN_THRESHOLD, NUM, DEN)
    assert 0.85 * v.n < len(xyz) <= 1.05 * v.n
    assert (np.diff(vox) > 0).all()
    ext = np.array(synth.FRAME_EXTENT)
    assert (xyz >= 0).all() and (xyz < ext).all()
