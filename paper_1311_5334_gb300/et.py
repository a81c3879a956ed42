"""Python binding of libet (include/et.h): argument marshalling only.

Every step of the track-finding path runs in the CUDA library; this module
only converts arrays and structures.  If libet.so is missing or cannot be
loaded, importing the binding's entry points raises: there is no CPU path.

The names mirror the C ABI:

    ctx = Context(0)
    view = ctx.view(xyz, params)          # et_view_create (host grains)
    view.find()                           # et_track_find (async)
    tracks, members = view.fetch()        # et_track_fetch

and of the image front end (include/et_frames.h):

    fr = ctx.frames(frame_params, gain, thr)   # et_frames_create
    fr.run(raw)                                # et_frames_run (async)
    xyz, pulse, offsets = fr.fetch()           # et_frames_fetch
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libet.so")

OK = 0
INVALID_ARG, OUT_OF_RANGE, DUPLICATE_GRAIN, PRECONDITION, CAPACITY = -1, -2, -3, -4, -5
OOM, BUSY, TIMEOUT, CUDA, NOT_READY = -6, -7, -8, -9, -10


class EtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libet status {status}: {msg}")
        self.status = status


FLAG_SINGLE_PASS, FLAG_ANGLE_CUT = 1, 2


class Params(C.Structure):
    _fields_ = [("extent", C.c_int32 * 3), ("seed_min", C.c_int32), ("seed_max", C.c_int32),
                ("tube_r", C.c_int32), ("min_hits", C.c_int32), ("flags", C.c_uint32),
                ("cut_base", C.c_int32), ("cut_slope", C.c_int32), ("cut_tan_max", C.c_int32),
                ("reserved", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("cell", C.c_int32 * 3), ("ticket_origins", C.c_int32), ("row_lists", C.c_int32),
                ("assoc_window", C.c_int32), ("wait_polls", C.c_int32), ("reserved", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_grains", C.c_int64), ("n_seeds", C.c_int64), ("n_tests", C.c_int64),
                ("n_hits", C.c_int64), ("n_candidates", C.c_int64), ("n_members", C.c_int64),
                ("n_tracks", C.c_int64), ("n_track_members", C.c_int64), ("merge_rounds", C.c_int32),
                ("cell", C.c_int32 * 3), ("kernel_launches", C.c_int32), ("profiled", C.c_int32),
                ("stage_ms", C.c_float * 6), ("n_pair_tests", C.c_int64)]

    STAGES = ("cells", "seeds", "tube_count", "members", "merge", "output")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("cell", "stage_ms")}
        d["cell"] = tuple(self.cell)
        d["stage_ms"] = dict(zip(self.STAGES, (float(x) for x in self.stage_ms))) if self.profiled else None
        return d


class ServerStats(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("device_bytes", C.c_uint64), ("peak_device_bytes", C.c_uint64),
                ("views_done", C.c_int64), ("batches", C.c_int64), ("busy_rejections", C.c_int64),
                ("pending", C.c_int64)]


class Result(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("n_tracks", C.c_int32),
                ("n_members", C.c_int64), ("n_grains", C.c_int64), ("t_submit_ns", C.c_int64),
                ("t_admit_ns", C.c_int64), ("t_done_ns", C.c_int64)]


class FrameParams(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("depth", C.c_int32), ("row_pitch", C.c_int32),
                ("pitch_num", C.c_int32 * 3), ("pitch_den", C.c_int32 * 3), ("grain_threshold", C.c_int32),
                ("flags", C.c_uint32)]


class FramesStats(C.Structure):
    _fields_ = [("n_views", C.c_int64), ("n_voxels", C.c_int64), ("n_candidates", C.c_int64),
                ("n_grains", C.c_int64), ("kernel_ms", C.c_float), ("run_ms", C.c_float),
                ("kernel_launches", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TRACK_DTYPE = np.dtype([("seed_i", "<i4"), ("seed_j", "<i4"), ("nhits", "<i4"), ("view", "<i4"),
                        ("member_offset", "<i8"), ("c", "<f4", (3,)), ("u", "<f4", (3,)),
                        ("tmin", "<f4"), ("tmax", "<f4"), ("count", "<i4"), ("reserved", "<i4")])
assert TRACK_DTYPE.itemsize == 64

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None

_SIGS = {
    "et_abi_version": (C.c_int32, []),
    "et_last_error": (C.c_char_p, []),
    "et_status_string": (C.c_char_p, [C.c_int32]),
    "et_ctx_create": (C.c_int32, [C.c_int, C.POINTER(C.c_void_p)]),
    "et_ctx_destroy": (C.c_int32, [C.c_void_p]),
    "et_ctx_set_allocator": (C.c_int32, [C.c_void_p, ALLOC_FN, FREE_FN, C.c_void_p]),
    "et_ctx_info": (C.c_int32, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32)]),
    "et_view_create": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(Params),
                                   C.POINTER(C.c_void_p)]),
    "et_view_create_device": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(Params),
                                          C.POINTER(C.c_void_p)]),
    "et_view_load": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "et_view_destroy": (C.c_int32, [C.c_void_p]),
    "et_track_find": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "et_track_fetch": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64),
                                   C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "et_view_seed_counts": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                        C.POINTER(C.c_int64)]),
    "et_batch_create": (C.c_int32, [C.c_void_p, C.POINTER(Params), C.POINTER(C.c_void_p)]),
    "et_batch_load": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    "et_batch_set_tuning": (C.c_int32, [C.c_void_p, C.POINTER(Tuning)]),
    "et_batch_find": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32]),
    "et_batch_autotune": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(Tuning),
                                      C.POINTER(C.c_float)]),
    "et_batch_fetch": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64),
                                   C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "et_batch_stats": (C.c_int32, [C.c_void_p, C.POINTER(Stats)]),
    "et_batch_sync": (C.c_int32, [C.c_void_p]),
    "et_batch_set_profiling": (C.c_int32, [C.c_void_p, C.c_int32]),
    "et_batch_destroy": (C.c_int32, [C.c_void_p]),
    "et_server_create": (C.c_int32, [C.c_void_p, C.POINTER(Params), C.c_uint64, C.c_int32,
                                     C.POINTER(C.c_void_p)]),
    "et_server_submit": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64]),
    "et_server_poll": (C.c_int32, [C.c_void_p, C.POINTER(Result), C.c_int32, C.POINTER(C.c_int32),
                                   C.c_int32]),
    "et_server_fetch": (C.c_int32, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int64, C.POINTER(C.c_int64),
                                    C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "et_server_destroy": (C.c_int32, [C.c_void_p]),
    "et_server_set_max_pending": (C.c_int32, [C.c_void_p, C.c_int64]),
    "et_server_get_stats": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "et_tube_count_noalloc": (C.c_int32, [C.c_void_p, C.c_int64, C.POINTER(Params), C.c_void_p, C.c_int64,
                                          C.c_void_p, C.c_void_p]),
    "et_probe_int_throughput": (C.c_int32, [C.c_void_p, C.POINTER(C.c_double * 3)]),
    "et_frames_create": (C.c_int32, [C.c_void_p, C.POINTER(FrameParams), C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_void_p)]),
    "et_frames_set_calibration": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "et_frames_run": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    "et_frames_sync": (C.c_int32, [C.c_void_p]),
    "et_frames_fetch": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                    C.POINTER(C.c_int64)]),
    "et_frames_to_batch": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "et_frames_stats_get": (C.c_int32, [C.c_void_p, C.POINTER(FramesStats)]),
    "et_frames_destroy": (C.c_int32, [C.c_void_p]),
}


def lib():
    """Loads libet.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                              "(python -m paper_1311_5334_gb300.build)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        L = lib()
        raise EtError(status, L.et_last_error().decode(errors="replace"))
    return status


def make_params(extent, seed_min, seed_max, tube_r, min_hits, flags=0, cut=(0, 0, 0)) -> Params:
    p = Params()
    for k in range(3):
        p.extent[k] = int(extent[k])
    p.seed_min, p.seed_max, p.tube_r, p.min_hits, p.flags = (int(seed_min), int(seed_max), int(tube_r),
                                                             int(min_hits), int(flags))
    p.cut_base, p.cut_slope, p.cut_tan_max = (int(c) for c in cut)
    return p


def _params(pp) -> Params:
    if isinstance(pp, Params):
        return pp
    return make_params(pp["extent"], pp["seed_min"], pp["seed_max"], pp["tube_r"], pp["min_hits"],
                       pp.get("flags", 0), pp.get("cut", (0, 0, 0)))


def _host_grains(xyz):
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.int32).reshape(-1, 3))
    return a


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a.size else None


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


class Context:
    """et_ctx: one CUDA device.  use_torch_allocator routes device memory
    through PyTorch's caching allocator."""

    def __init__(self, device=0, use_torch_allocator=False):
        L = lib()
        h = C.c_void_p()
        _check(L.et_ctx_create(int(device), C.byref(h)))
        self._h = h
        self.device = int(device)
        self._hooks = None
        if use_torch_allocator:
            self._install_torch_allocator()

    def _install_torch_allocator(self):
        import torch
        dev = self.device

        def _alloc(nbytes, _user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
            except Exception:
                return None

        def _free(ptr, _user):
            torch.cuda.caching_allocator_delete(ptr)

        self._hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
        _check(lib().et_ctx_set_allocator(self._h, self._hooks[0], self._hooks[1], None))

    def info(self):
        sm, ma, mi = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().et_ctx_info(self._h, C.byref(sm), C.byref(ma), C.byref(mi)))
        return {"sm_count": sm.value, "cc": (ma.value, mi.value)}

    def int_throughput(self):
        """Measured 32-bit integer issue rates of the device, ops/s (et_probe.h):
        {"alu": xor + add, "mad": multiply-add, "mix": both in the tube test's ratio}."""
        out = (C.c_double * 3)()
        _check(lib().et_probe_int_throughput(self._h, C.byref(out)))
        return {"alu": out[0], "mad": out[1], "mix": out[2]}

    def close(self):
        if getattr(self, "_h", None):
            lib().et_ctx_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def view(self, xyz, params):
        return View.create(self, xyz, params)

    def batch(self, params):
        return Batch(self, params)

    def frames(self, frame_params, gain, thr):
        return Frames(self, frame_params, gain, thr)

    def server(self, params, mem_budget_bytes, max_batch_views=256):
        return Server(self, params, mem_budget_bytes, max_batch_views)


def _fetch(fn, h, with_view_offsets=False, n_views=1, out=None):
    """Tracks and members; `out` = (tracks, members[, view_offsets]) arrays to
    fill when large enough (reused buffers, e.g. page-locked), else new ones."""
    nt, nm = C.c_int64(), C.c_int64()
    st = fn(h, None, None, 0, C.byref(nt), None, 0, C.byref(nm)) if with_view_offsets else \
        fn(h, None, 0, C.byref(nt), None, 0, C.byref(nm))
    if st not in (OK, CAPACITY):
        _check(st)
    ot, om = (out[0], out[1]) if out is not None else (None, None)
    tracks = ot if ot is not None and ot.dtype == TRACK_DTYPE and ot.shape[0] >= nt.value \
        else np.zeros(nt.value, dtype=TRACK_DTYPE)
    members = om if om is not None and om.dtype == np.int32 and om.shape[0] >= nm.value \
        else np.zeros(nm.value, dtype=np.int32)
    if with_view_offsets:
        ov = out[2] if out is not None and len(out) > 2 else None
        voff = ov if ov is not None and ov.dtype == np.int64 and ov.shape[0] >= n_views + 1 \
            else np.zeros(n_views + 1, dtype=np.int64)
        _check(fn(h, _ptr(voff), _ptr(tracks), nt.value, C.byref(nt), _ptr(members), nm.value, C.byref(nm)))
        return tracks[:nt.value], members[:nm.value], voff[:n_views + 1]
    _check(fn(h, _ptr(tracks), nt.value, C.byref(nt), _ptr(members), nm.value, C.byref(nm)))
    return tracks[:nt.value], members[:nm.value]


class Batch:
    """et_batch: many views with one et_params."""

    def __init__(self, ctx: Context, params):
        self.ctx = ctx
        self._params = _params(params)
        h = C.c_void_p()
        _check(lib().et_batch_create(ctx._h, C.byref(self._params), C.byref(h)))
        self._h = h
        self._keep = None
        self.n_views = 0

    def set_tuning(self, cell=(0, 0, 0), row_lists=0, assoc_window=0, wait_polls=0, ticket_origins=0):
        t = Tuning()
        t.ticket_origins = int(ticket_origins)
        for k in range(3):
            t.cell[k] = int(cell[k])
        t.row_lists = int(row_lists)
        t.assoc_window = int(assoc_window)
        t.wait_polls = int(wait_polls)
        _check(lib().et_batch_set_tuning(self._h, C.byref(t)))

    def load(self, xyz, offsets, stream=None):
        """xyz: host array (total, 3) int32 or a CUDA torch tensor; offsets: (V+1,) ints."""
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        on_dev = 0
        if hasattr(xyz, "is_cuda") and xyz.is_cuda:
            t = xyz.contiguous()
            ptr, on_dev, keep = C.c_void_p(t.data_ptr()), 1, t
        else:
            keep = _host_grains(xyz)
            ptr = _ptr(keep)
        self._keep = (keep, offs)
        self.n_views = offs.shape[0] - 1
        _check(lib().et_batch_load(self._h, ptr, _ptr(offs), self.n_views, on_dev, _stream_ptr(stream)))

    def find(self, stream=None, use_graph=False):
        _check(lib().et_batch_find(self._h, _stream_ptr(stream), 1 if use_graph else 0))

    def autotune(self, stream=None, max_trials=0):
        """Times the path for candidate cell shapes; keeps and returns the fastest
        as (cell, ms per run)."""
        t = Tuning()
        ms = C.c_float()
        _check(lib().et_batch_autotune(self._h, _stream_ptr(stream), int(max_trials), C.byref(t), C.byref(ms)))
        self.tuning = {"cell": tuple(t.cell), "row_lists": int(t.row_lists), "ticket_origins": int(t.ticket_origins)}
        return tuple(t.cell), float(ms.value)

    def sync(self):
        _check(lib().et_batch_sync(self._h))

    def set_profiling(self, on=True):
        _check(lib().et_batch_set_profiling(self._h, 1 if on else 0))

    def fetch(self, out=None):
        """(tracks, members, view_track_offsets); out: optional arrays to reuse."""
        return _fetch(lib().et_batch_fetch, self._h, True, self.n_views, out)

    def stats(self):
        s = Stats()
        _check(lib().et_batch_stats(self._h, C.byref(s)))
        return s.as_dict()

    def seed_counts(self):
        """All seeds (seed_i, seed_j, count) of the last run, unordered; for a
        batch the indices run over all views' grains back to back."""
        L = lib()
        ns = C.c_int64()
        st = L.et_view_seed_counts(self._h, None, None, None, 0, C.byref(ns))
        if st not in (OK, CAPACITY):
            _check(st)
        a, b, c = (np.zeros(ns.value, dtype=np.int32) for _ in range(3))
        _check(L.et_view_seed_counts(self._h, _ptr(a), _ptr(b), _ptr(c), ns.value, C.byref(ns)))
        return a, b, c

    def close(self):
        if getattr(self, "_h", None):
            lib().et_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class View(Batch):
    """et_view: a batch of one view."""

    @classmethod
    def create(cls, ctx: Context, xyz, params):
        self = cls.__new__(cls)
        self.ctx = ctx
        self._params = _params(params)
        h = C.c_void_p()
        if hasattr(xyz, "is_cuda") and xyz.is_cuda:
            t = xyz.contiguous()
            _check(lib().et_view_create_device(ctx._h, C.c_void_p(t.data_ptr()), t.shape[0],
                                               C.byref(self._params), C.byref(h)))
            self._keep = t
        else:
            a = _host_grains(xyz)
            _check(lib().et_view_create(ctx._h, _ptr(a), a.shape[0], C.byref(self._params), C.byref(h)))
            self._keep = None
        self._h = h
        self.n_views = 1
        return self

    def load_host(self, xyz, stream=None):
        a = _host_grains(xyz)
        self._keep = a
        _check(lib().et_view_load(self._h, _ptr(a), a.shape[0], _stream_ptr(stream)))

    def find(self, stream=None, use_graph=False):
        if use_graph:
            super().find(stream, True)
        else:
            _check(lib().et_track_find(self._h, _stream_ptr(stream)))

    def fetch(self, out=None):
        """(tracks structured array, members int32); out: optional arrays to reuse."""
        return _fetch(lib().et_track_fetch, self._h, out=out)


class Server:
    """et_server: served loop with memory-budget admission."""

    def __init__(self, ctx: Context, params, mem_budget_bytes, max_batch_views=256):
        self.ctx = ctx
        self._params = _params(params)
        h = C.c_void_p()
        _check(lib().et_server_create(ctx._h, C.byref(self._params), int(mem_budget_bytes),
                                      int(max_batch_views), C.byref(h)))
        self._h = h

    def submit(self, xyz, tag):
        a = _host_grains(xyz)
        return lib().et_server_submit(self._h, _ptr(a), a.shape[0], int(tag))

    def poll(self, max_results=1024, timeout_us=1000):
        out = (Result * max_results)()
        n = C.c_int32()
        _check(lib().et_server_poll(self._h, out, max_results, C.byref(n), int(timeout_us)))
        return [out[i] for i in range(n.value)]

    def fetch(self, tag):
        nt, nm = C.c_int64(), C.c_int64()
        L = lib()
        st = L.et_server_fetch(self._h, int(tag), None, 0, C.byref(nt), None, 0, C.byref(nm))
        if st not in (OK, CAPACITY):
            _check(st)
        tracks = np.zeros(nt.value, dtype=TRACK_DTYPE)
        members = np.zeros(nm.value, dtype=np.int32)
        _check(L.et_server_fetch(self._h, int(tag), _ptr(tracks), nt.value, C.byref(nt), _ptr(members),
                                 nm.value, C.byref(nm)))
        return tracks, members

    def set_max_pending(self, n):
        _check(lib().et_server_set_max_pending(self._h, int(n)))

    def stats(self):
        st = ServerStats()
        _check(lib().et_server_get_stats(self._h, C.byref(st)))
        return {k: int(getattr(st, k)) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().et_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def make_frame_params(width, height, depth, pitch_num, pitch_den, grain_threshold, row_pitch=None,
                      flags=0) -> FrameParams:
    p = FrameParams()
    p.width, p.height, p.depth = int(width), int(height), int(depth)
    p.row_pitch = int(width if row_pitch is None else row_pitch)
    for k in range(3):
        p.pitch_num[k] = int(pitch_num[k])
        p.pitch_den[k] = int(pitch_den[k])
    p.grain_threshold, p.flags = int(grain_threshold), int(flags)
    return p


class Frames:
    """et_frames: the image front end of one camera (filtering and 3D grain
    recognition, Section 2).  gain / thr: uint8 [height][width]."""

    def __init__(self, ctx: Context, frame_params, gain, thr):
        self.ctx = ctx
        self.params = frame_params
        g = np.ascontiguousarray(gain, dtype=np.uint8)
        t = np.ascontiguousarray(thr, dtype=np.uint8)
        h = C.c_void_p()
        _check(lib().et_frames_create(ctx._h, C.byref(self.params), _ptr(g), _ptr(t), C.byref(h)))
        self._h = h
        self._keep = None
        self.n_views = 0

    def set_calibration(self, gain, thr):
        g = np.ascontiguousarray(gain, dtype=np.uint8)
        t = np.ascontiguousarray(thr, dtype=np.uint8)
        _check(lib().et_frames_set_calibration(self._h, _ptr(g), _ptr(t)))

    def run(self, raw, n_views=None, stream=None):
        """raw: uint8 views back to back (depth x height x row_pitch bytes each),
        a host array or a CUDA torch tensor (read in place)."""
        view_bytes = self.params.depth * self.params.height * self.params.row_pitch
        if hasattr(raw, "is_cuda") and raw.is_cuda:
            t = raw.contiguous()
            ptr, on_dev, keep, nbytes = C.c_void_p(t.data_ptr()), 1, t, t.numel() * t.element_size()
        else:
            keep = np.ascontiguousarray(raw, dtype=np.uint8)
            ptr, on_dev, nbytes = _ptr(keep), 0, keep.nbytes
        if n_views is None:
            if nbytes % view_bytes:
                raise ValueError(f"{nbytes} bytes is not a whole number of {view_bytes}-byte views")
            n_views = nbytes // view_bytes
        self._keep = keep
        self.n_views = int(n_views)
        _check(lib().et_frames_run(self._h, ptr, self.n_views, on_dev, _stream_ptr(stream)))

    def sync(self):
        _check(lib().et_frames_sync(self._h))

    def fetch(self, out=None):
        """(xyz int32 [n][3], pulse int32 [n], view_offsets int64 [V+1]) in raster
        order of each view's defining voxels; out: optional (xyz, pulse,
        view_offsets) arrays to fill when large enough."""
        n = C.c_int64()
        st = lib().et_frames_fetch(self._h, None, None, None, 0, C.byref(n))
        if st not in (OK, CAPACITY):
            _check(st)
        ox, op, ov = out if out is not None else (None, None, None)
        xyz = ox if ox is not None and ox.dtype == np.int32 and ox.shape[0] >= n.value and ox.ndim == 2 \
            else np.zeros((n.value, 3), dtype=np.int32)
        pulse = op if op is not None and op.dtype == np.int32 and op.shape[0] >= n.value \
            else np.zeros(n.value, dtype=np.int32)
        voff = ov if ov is not None and ov.dtype == np.int64 and ov.shape[0] >= self.n_views + 1 \
            else np.zeros(self.n_views + 1, dtype=np.int64)
        _check(lib().et_frames_fetch(self._h, _ptr(voff), _ptr(xyz), _ptr(pulse), n.value, C.byref(n)))
        return xyz[:n.value], pulse[:n.value], voff[:self.n_views + 1]

    def to_batch(self, batch, stream=None):
        _check(lib().et_frames_to_batch(self._h, batch._h, _stream_ptr(stream)))
        batch.n_views = self.n_views

    def stats(self):
        s = FramesStats()
        _check(lib().et_frames_stats_get(self._h, C.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().et_frames_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tube_count_noalloc(d_xyz, params, d_pairs, d_counts, stream=None):
    """et_tube_count_noalloc on CUDA tensors: d_xyz (n, 3) int32, d_pairs (m, 2)
    int32, d_counts (m,) int32 output; allocates nothing, returns immediately."""
    p = _params(params)
    for t in (d_xyz, d_pairs, d_counts):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("device tensors must be contiguous CUDA tensors")
    _check(lib().et_tube_count_noalloc(C.c_void_p(d_xyz.data_ptr()), d_xyz.shape[0], C.byref(p),
                                       C.c_void_p(d_pairs.data_ptr()), d_pairs.shape[0],
                                       C.c_void_p(d_counts.data_ptr()), _stream_ptr(stream)))


def track_tuples(tracks, members):
    """(seed_i, seed_j, nhits, tuple(members)) per track, in order."""
    out = []
    for t in tracks:
        o = int(t["member_offset"])
        out.append((int(t["seed_i"]), int(t["seed_j"]), int(t["nhits"]),
                    tuple(int(m) for m in members[o:o + int(t["nhits"])])))
    return out
