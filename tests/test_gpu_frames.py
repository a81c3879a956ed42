"""GPU image front end vs the oracle, through the C ABI (libet.so).

Filtering and 3D grain recognition (Section 2) are exact integer work: the
grains of every view -- coordinates, pulse sums, order and per-view offsets --
must equal the oracle's bit for bit.  Cases span several tiles with ragged
edges, row padding, many equal neighbours, one- and two-frame stacks, full
1280 x 1024 x 40 views, empty and saturated stacks, an output overflow that
forces the buffer to grow, host and device input, and the chain from raw
frames to tracks.
"""
import numpy as np
import pytest

from paper_1311_5334_gb300 import synth

pytestmark = pytest.mark.gpu

NUM, DEN, T = synth.PITCH_NUM, synth.PITCH_DEN, synth.GRAIN_THRESHOLD


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


def oracle_grains(O, frames, threshold=T, num=NUM, den=DEN):
    f = O.frames_filter(frames.raw, frames.gain, frames.thr)
    return O.frames_grains(f, threshold, num, den)


def run_gpu(et, ctx, frames_list, threshold=T, num=NUM, den=DEN, device=False):
    D, H, P = frames_list[0].raw.shape
    W = frames_list[0].width
    fp = et.make_frame_params(W, H, D, num, den, threshold, row_pitch=P)
    raw = np.concatenate([f.raw.reshape(-1) for f in frames_list])
    fr = et.Frames(ctx, fp, frames_list[0].gain, frames_list[0].thr)
    try:
        if device:
            import torch
            fr.run(torch.from_numpy(raw).cuda(), n_views=len(frames_list))
        else:
            fr.run(raw, n_views=len(frames_list))
        out = fr.fetch()
        st = fr.stats()
    finally:
        fr.close()
    return out, st


def same_calibration(frames_list):
    # the views of one run share the camera's calibration
    base = frames_list[0]
    return [synth.Frames(raw=f.raw, gain=base.gain, thr=base.thr, width=f.width) for f in frames_list]


def check(O, frames_list, out, threshold=T, num=NUM, den=DEN):
    xyz, pulse, voff = out
    assert voff[0] == 0 and voff[-1] == len(xyz)
    for v, fr in enumerate(frames_list):
        wx, wp, _ = oracle_grains(O, fr, threshold, num, den)
        a, b = voff[v], voff[v + 1]
        assert b - a == len(wx), f"view {v}: {b - a} grains, oracle {len(wx)}"
        assert np.array_equal(xyz[a:b], wx), f"view {v}: coordinates differ"
        assert np.array_equal(pulse[a:b], wp), f"view {v}: pulse sums differ"


@pytest.mark.parametrize("shape,pitch,n,quantum", [
    ((6, 45, 200), 208, 60, None),     # 2 x 2 tiles, ragged in x and y, padded rows
    ((5, 70, 130), 144, 80, 16),       # coarse levels: many equal neighbours
    ((1, 33, 129), 144, 30, None),     # one frame; one column past a tile edge
    ((2, 32, 128), 128, 40, 8),        # exactly one tile, two frames
    ((9, 7, 13), 16, 6, None),         # narrower than a tile, tiny
])
def test_small_stacks(et, ctx, oracle_mod, shape, pitch, n, quantum):
    views = same_calibration([synth.random_blobs(shape, n=n, seed=s, row_pitch=pitch, quantum=quantum)
                              for s in (11, 12, 13)])
    out, st = run_gpu(et, ctx, views)
    check(oracle_mod, views, out)
    assert st["n_views"] == 3 and st["n_grains"] == len(out[0])


@pytest.mark.parametrize("threshold", [0, 12, 80])
def test_thresholds(et, ctx, oracle_mod, threshold):
    views = same_calibration([synth.random_blobs((7, 60, 150), n=120, seed=s, row_pitch=160, quantum=4)
                              for s in (21, 22)])
    out, _ = run_gpu(et, ctx, views, threshold=threshold)
    check(oracle_mod, views, out, threshold=threshold)


def test_other_pitches(et, ctx, oracle_mod):
    views = [synth.random_blobs((4, 50, 64), n=50, seed=31)]
    num, den = (7, 65535, 3), (3, 1, 65535)
    out, _ = run_gpu(et, ctx, views, num=num, den=den)
    check(oracle_mod, views, out, num=num, den=den)


def test_full_size_views(et, ctx, oracle_mod):
    # two full 1280 x 1024 x 40 views in one run (grid of 10 x 32 tiles per view)
    pairs = [synth.frames_view(s, n_fog=10000, n_through=100) for s in (41, 42)]
    views = same_calibration([fr for _, fr in pairs])
    out, st = run_gpu(et, ctx, views)
    check(oracle_mod, views, out)
    assert st["n_voxels"] == 2 * 1280 * 1024 * 40
    assert st["n_candidates"] > st["n_grains"] > 15000


def test_device_input_matches_host_input(et, ctx, oracle_mod):
    pytest.importorskip("torch")
    views = same_calibration([synth.random_blobs((5, 64, 256), n=90, seed=s) for s in (51, 52)])
    a, _ = run_gpu(et, ctx, views)
    b, _ = run_gpu(et, ctx, views, device=True)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    check(oracle_mod, views, b)


def test_empty_and_saturated(et, ctx, oracle_mod):
    D, H, W = 4, 40, 160
    gain = np.full((H, W), 128, np.uint8)
    thr = np.full((H, W), 20, np.uint8)
    bright = synth.Frames(raw=np.full((D, H, W), 255, np.uint8), gain=gain, thr=thr, width=W)
    dark = synth.Frames(raw=np.zeros((D, H, W), np.uint8), gain=gain, thr=thr, width=W)
    out, st = run_gpu(et, ctx, [bright, dark, bright])
    check(oracle_mod, [bright, dark, bright], out)
    # a constant stack is one plateau: only its first voxel has no earlier equal neighbour
    assert list(out[2]) == [0, 0, 1, 1]
    assert st["n_candidates"] == D * H * W


@pytest.mark.parametrize("shape", [(3, 64, 4096), (2, 4096, 300), (1024, 16, 32)])
def test_geometry_limits(et, ctx, oracle_mod, shape):
    # widest frames (16 tiles across), tallest (256 tiles down), deepest stack
    # (1024 frames through the stage ring)
    D, H, W = shape
    views = [synth.random_blobs(shape, n=max(8, D * H * W // 2000), seed=71, row_pitch=(W + 15) // 16 * 16)]
    out, st = run_gpu(et, ctx, views)
    check(oracle_mod, views, out)
    assert st["n_voxels"] == D * H * W


def test_output_overflow_grows(et, ctx, oracle_mod):
    # isolated maxima every second voxel along each axis: far more grains than
    # the first buffer guess (max(65536, voxels / 2000)) -- the run is repeated
    D, H, W = 12, 256, 512
    raw = np.full((D, H, W), 200, np.uint8)
    raw[::2, ::2, ::2] = 10
    gain = np.full((H, W), 128, np.uint8)
    thr = np.full((H, W), 30, np.uint8)
    fr = synth.Frames(raw=raw, gain=gain, thr=thr, width=W)
    out, st = run_gpu(et, ctx, [fr])
    assert len(out[0]) == (D // 2) * (H // 2) * (W // 2) > 65536
    check(oracle_mod, [fr], out)


def test_frames_to_tracks(et, ctx, oracle_mod):
    # raw frames -> grains -> tracks on the device equals the oracle chain
    v, fr = synth.frames_view(61, n_fog=6000, n_through=60)
    fp = et.make_frame_params(fr.width, fr.raw.shape[1], fr.raw.shape[0], NUM, DEN, T, row_pitch=fr.raw.shape[2])
    params = synth.params(synth.FRAME_EXTENT)
    with et.Frames(ctx, fp, fr.gain, fr.thr) as f, et.Batch(ctx, params) as b:
        f.run(fr.raw)
        f.to_batch(b)
        b.find()
        tracks, members, voff = b.fetch()
    gx, _, _ = oracle_grains(oracle_mod, fr)
    o = oracle_mod.Oracle(gx, params["extent"], params["seed_min"], params["seed_max"], params["tube_r"],
                          params["min_hits"])
    try:
        want = o.find_tracks()
    finally:
        o.close()
    assert len(want) > 20
    assert et.track_tuples(tracks, members) == want.as_tuples()


def test_input_errors(et, ctx):
    gain = np.full((8, 20), 128, np.uint8)
    with pytest.raises(et.EtError) as e:
        et.Frames(ctx, et.make_frame_params(20, 8, 3, NUM, DEN, T, row_pitch=20), gain, gain)
    assert e.value.status == et.INVALID_ARG
    with pytest.raises(et.EtError) as e:
        et.Frames(ctx, et.make_frame_params(20, 8, 3, NUM, DEN, 255, row_pitch=32), gain, gain)
    assert e.value.status == et.INVALID_ARG
    with pytest.raises(et.EtError) as e:
        et.Frames(ctx, et.make_frame_params(20, 8, 3, (0, 1, 1), DEN, T, row_pitch=32), gain, gain)
    assert e.value.status == et.INVALID_ARG
    torch = pytest.importorskip("torch")
    with et.Frames(ctx, et.make_frame_params(20, 8, 3, NUM, DEN, T, row_pitch=32), gain, gain) as f:
        buf = torch.zeros(3 * 8 * 32 + 16, dtype=torch.uint8, device="cuda")
        with pytest.raises(et.EtError) as e:
            f.run(buf[1:1 + 3 * 8 * 32], n_views=1)   # not 16-byte aligned
        assert e.value.status == et.INVALID_ARG
