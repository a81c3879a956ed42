"""ctypes wrapper around the C oracle (oracle.c, frames.c).

TEST INFRASTRUCTURE ONLY: used by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py.  The product path (the CUDA library and its
binding) never imports this module.

The oracle is the plain definition of Section 2 of the paper (seeds = grain
pairs within a distance window, count of grains along each seed line,
threshold, exclusive grain association) evaluated on the CPU with exact
integer arithmetic, plus an FP64 orthogonal least-squares fit; and the image
front end of the same section (pixel filtering and 3D grain recognition,
frames.c), also in exact integer arithmetic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "frames.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

# The paper's hash cell: 32 x 32 pixels x 1 frame of a 1280 x 1024 x 40 view of
# 300 x 250 x 50 um (Section 2 and the Section 3 footnote) -> 7.5 um x 7.5 um x
# 1.25 um, in 10 nm units.
PAPER_CELL = (750, 750, 125)

OK, INVALID_ARG, OUT_OF_RANGE, DUPLICATE, OOM = 0, -1, -2, -3, -6


class OracleError(RuntimeError):
    def __init__(self, status, what=""):
        super().__init__(f"oracle status {status} {what}")
        self.status = status


SINGLE_PASS, ANGLE_CUT = 1, 2


class _Params(C.Structure):
    _fields_ = [("extent", C.c_int32 * 3), ("seed_min", C.c_int32), ("seed_max", C.c_int32),
                ("tube_r", C.c_int32), ("min_hits", C.c_int32), ("flags", C.c_uint32),
                ("cut_base", C.c_int32), ("cut_slope", C.c_int32), ("cut_tan_max", C.c_int32),
                ("reserved", C.c_int32)]


class _Tracks(C.Structure):
    _fields_ = [("n_seeds", C.c_int64), ("n_cand", C.c_int64), ("n_tracks", C.c_int64),
                ("tests", C.c_int64),
                ("lo", C.POINTER(C.c_int32)), ("hi", C.POINTER(C.c_int32)),
                ("nhits", C.POINTER(C.c_int32)), ("moff", C.POINTER(C.c_int64)),
                ("members", C.POINTER(C.c_int32)),
                ("c", C.POINTER(C.c_double)), ("u", C.POINTER(C.c_double)),
                ("t", C.POINTER(C.c_double)), ("lam", C.POINTER(C.c_double))]


_lib = None
_lock = threading.Lock()


def build(force=False, quiet=True):
    """Compile oracle.c and frames.c with gcc (-O2, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-Wno-unused-parameter", *_SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, capture_output=quiet)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P32, P64, PD = C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double)
            L.or_create.restype = C.c_void_p
            L.or_create.argtypes = [P32, C.c_int64, C.POINTER(_Params), P32, P32]
            L.or_destroy.argtypes = [C.c_void_p]
            L.or_rank.restype = C.c_int32
            L.or_rank.argtypes = [C.c_void_p, C.c_int32]
            L.or_seed_total.restype = C.c_int64
            L.or_seed_total.argtypes = [C.c_void_p]
            L.or_seeds_per_grain.restype = C.c_int64
            L.or_seeds_per_grain.argtypes = [C.c_void_p, P64]
            L.or_list_seeds.restype = C.c_int64
            L.or_list_seeds.argtypes = [C.c_void_p, P32, P32, C.c_int64]
            L.or_count_pairs.argtypes = [C.c_void_p, P32, P32, C.c_int64, P32, C.c_int]
            L.or_count_pairs_brute.argtypes = [C.c_void_p, P32, P32, C.c_int64, P32, C.c_int]
            L.or_tube_members.restype = C.c_int64
            L.or_tube_members.argtypes = [C.c_void_p, C.c_int32, C.c_int32, P32, C.c_int64]
            L.or_find_tracks.restype = C.c_int
            L.or_find_tracks.argtypes = [C.c_void_p, C.c_int, C.POINTER(_Tracks), C.c_int,
                                         C.POINTER(P32), C.POINTER(P32), C.POINTER(P32)]
            L.or_tracks_free.argtypes = [C.POINTER(_Tracks)]
            L.or_sym_eigen3.argtypes = [PD, PD, PD]
            L.or_fit.argtypes = [C.c_void_p, P32, C.c_int64, C.c_int32, C.c_int32, PD, PD, PD, PD]
            PU8 = C.POINTER(C.c_uint8)
            L.or_frames_filter.restype = C.c_int
            L.or_frames_filter.argtypes = [PU8, C.c_int64, C.c_int32, C.c_int32, C.c_int32, PU8, PU8, PU8]
            L.or_frames_grains.restype = C.c_int64
            L.or_frames_grains.argtypes = [PU8, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P32, P32,
                                           P32, P32, P64, C.c_int64]
            _lib = L
    return _lib


def _p32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(extent, seed_min, seed_max, tube_r, min_hits, flags=0, cut=(0, 0, 0)):
    p = _Params()
    for k in range(3):
        p.extent[k] = int(extent[k])
    p.seed_min, p.seed_max, p.tube_r, p.min_hits, p.flags = (int(seed_min), int(seed_max),
                                                             int(tube_r), int(min_hits), int(flags))
    p.cut_base, p.cut_slope, p.cut_tan_max = (int(c) for c in cut)
    return p


class Tracks:
    """Accepted tracks in acceptance order (input grain ids)."""

    def __init__(self, lo, hi, nhits, moff, members, c, u, t, lam, n_seeds, n_cand, tests):
        self.lo, self.hi, self.nhits, self.moff, self.members = lo, hi, nhits, moff, members
        self.c, self.u, self.t, self.lam = c, u, t, lam
        self.n_seeds, self.n_cand, self.tests = n_seeds, n_cand, tests

    def __len__(self):
        return int(self.lo.shape[0])

    def member_list(self, k):
        return self.members[self.moff[k]:self.moff[k + 1]]

    def as_tuples(self):
        """(lo, hi, nhits, tuple(members)) per track, in acceptance order."""
        return [(int(self.lo[k]), int(self.hi[k]), int(self.nhits[k]),
                 tuple(int(m) for m in self.member_list(k))) for k in range(len(self))]


class Oracle:
    """One view prepared for the oracle: grains, canonical ranks, cell hash."""

    def __init__(self, xyz, extent, seed_min, seed_max, tube_r, min_hits, flags=0, cell=PAPER_CELL,
                 cut=(0, 0, 0)):
        L = lib()
        self.xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.int32).reshape(-1, 3))
        self.params = make_params(extent, seed_min, seed_max, tube_r, min_hits, flags, cut)
        cell_arr = np.ascontiguousarray(np.asarray(cell, dtype=np.int32))
        st = np.zeros(1, dtype=np.int32)
        self._h = L.or_create(_p32(self.xyz), self.xyz.shape[0], C.byref(self.params), _p32(cell_arr),
                              _p32(st))
        if not self._h:
            raise OracleError(int(st[0]), "or_create")
        self.n = self.xyz.shape[0]

    def close(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
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

    def ranks(self):
        L = lib()
        return np.array([L.or_rank(self._h, i) for i in range(self.n)], dtype=np.int64)

    def seeds_per_grain(self):
        """Seeds per lo grain (input ids), int64 array of length n."""
        out = np.zeros(max(self.n, 1), dtype=np.int64)
        lib().or_seeds_per_grain(self._h, out.ctypes.data_as(C.POINTER(C.c_int64)))
        return out[:self.n]

    def seeds(self):
        """All seeds (lo, hi) as input ids, lo = lower rank, ordered by (rank lo, rank hi)."""
        L = lib()
        total = L.or_seed_total(self._h)
        lo = np.zeros(max(total, 1), dtype=np.int32)
        hi = np.zeros(max(total, 1), dtype=np.int32)
        got = L.or_list_seeds(self._h, _p32(lo), _p32(hi), total)
        if got < 0:
            raise OracleError(OOM, "or_list_seeds")
        return lo[:total], hi[:total]

    def count_pairs(self, lo, hi, nthreads=0, brute=False):
        lo = np.ascontiguousarray(lo, dtype=np.int32)
        hi = np.ascontiguousarray(hi, dtype=np.int32)
        out = np.zeros(max(lo.shape[0], 1), dtype=np.int32)
        fn = lib().or_count_pairs_brute if brute else lib().or_count_pairs
        fn(self._h, _p32(lo), _p32(hi), lo.shape[0], _p32(out), int(nthreads))
        return out[:lo.shape[0]]

    def tube_members(self, a, b):
        L = lib()
        m = L.or_tube_members(self._h, int(a), int(b), None, 0)
        out = np.zeros(max(m, 1), dtype=np.int32)
        L.or_tube_members(self._h, int(a), int(b), _p32(out), m)
        return out[:m]

    def find_tracks(self, nthreads=0, keep_seeds=False):
        """Run the whole method.  Returns Tracks, or (Tracks, (lo, hi, count)) with keep_seeds."""
        L = lib()
        t = _Tracks()
        slo, shi, scnt = C.POINTER(C.c_int32)(), C.POINTER(C.c_int32)(), C.POINTER(C.c_int32)()
        st = L.or_find_tracks(self._h, int(nthreads), C.byref(t), 1 if keep_seeds else 0,
                              C.byref(slo), C.byref(shi), C.byref(scnt))
        if st != OK:
            raise OracleError(st, "or_find_tracks")
        nt = t.n_tracks

        def arr(ptr, n, dt):
            if n == 0:
                return np.zeros(0, dtype=dt)
            return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt, copy=True)

        moff = arr(t.moff, nt + 1, np.int64)
        res = Tracks(lo=arr(t.lo, nt, np.int32), hi=arr(t.hi, nt, np.int32),
                     nhits=arr(t.nhits, nt, np.int32), moff=moff,
                     members=arr(t.members, int(moff[-1]) if nt else 0, np.int32),
                     c=arr(t.c, 3 * nt, np.float64).reshape(nt, 3),
                     u=arr(t.u, 3 * nt, np.float64).reshape(nt, 3),
                     t=arr(t.t, 2 * nt, np.float64).reshape(nt, 2),
                     lam=arr(t.lam, 3 * nt, np.float64).reshape(nt, 3),
                     n_seeds=int(t.n_seeds), n_cand=int(t.n_cand), tests=int(t.tests))
        L.or_tracks_free(C.byref(t))
        if keep_seeds:
            ns = res.n_seeds
            seeds = (arr(slo, ns, np.int32), arr(shi, ns, np.int32), arr(scnt, ns, np.int32))
            libc = C.CDLL(None)
            libc.free.argtypes = [C.c_void_p]
            for p in (slo, shi, scnt):
                libc.free(C.cast(p, C.c_void_p))
            return res, seeds
        return res

    def fit(self, members, lo, hi):
        mem = np.ascontiguousarray(members, dtype=np.int32)
        c, u, t, lam = np.zeros(3), np.zeros(3), np.zeros(2), np.zeros(3)
        lib().or_fit(self._h, _p32(mem), mem.shape[0], int(lo), int(hi), _pd(c), _pd(u), _pd(t), _pd(lam))
        return c, u, t, lam


def sym_eigen3(m):
    """Eigenvalues (descending) and eigenvectors (rows) of a symmetric 3x3 by the oracle's Jacobi."""
    m = np.ascontiguousarray(np.asarray(m, dtype=np.float64).reshape(9))
    lam, vec = np.zeros(3), np.zeros(9)
    lib().or_sym_eigen3(_pd(m), _pd(lam), _pd(vec))
    return lam, vec.reshape(3, 3)


# ---------------------------------------------------------------- image front end


def _pu8(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def frames_filter(raw, gain, thr):
    """Filtered pulse heights (uint8 [D][H][W]) of one view's raw frames.

    raw: uint8 [D][H][P] with P >= W row pitch (only the first W columns are
    pixels); gain, thr: uint8 [H][W] per-pixel gain (128 = 1.0) and threshold.
    """
    raw = np.ascontiguousarray(raw, dtype=np.uint8)
    gain = np.ascontiguousarray(gain, dtype=np.uint8)
    thr = np.ascontiguousarray(thr, dtype=np.uint8)
    D, H, P = raw.shape
    W = gain.shape[1]
    if gain.shape != (H, W) or thr.shape != (H, W) or P < W:
        raise OracleError(INVALID_ARG, "frames_filter shapes")
    out = np.zeros((D, H, W), dtype=np.uint8)
    st = lib().or_frames_filter(_pu8(raw), P, W, H, D, _pu8(gain), _pu8(thr), _pu8(out))
    if st != OK:
        raise OracleError(st, "or_frames_filter")
    return out


def frames_grains(filt, threshold, num, den):
    """Grains of one filtered view (uint8 [D][H][W]) in raster order of their
    defining voxel: (xyz int32 [n][3], pulse int32 [n], voxel int64 [n])."""
    filt = np.ascontiguousarray(filt, dtype=np.uint8)
    D, H, W = filt.shape
    num = np.ascontiguousarray(num, dtype=np.int32)
    den = np.ascontiguousarray(den, dtype=np.int32)
    L = lib()
    n = L.or_frames_grains(_pu8(filt), W, H, D, int(threshold), _p32(num), _p32(den), None, None, None, 0)
    if n < 0:
        raise OracleError(int(n), "or_frames_grains")
    xyz = np.zeros((max(n, 1), 3), dtype=np.int32)
    pulse = np.zeros(max(n, 1), dtype=np.int32)
    voxel = np.zeros(max(n, 1), dtype=np.int64)
    got = L.or_frames_grains(_pu8(filt), W, H, D, int(threshold), _p32(num), _p32(den), _p32(xyz),
                             _p32(pulse), voxel.ctypes.data_as(C.POINTER(C.c_int64)), n)
    assert got == n
    return xyz[:n], pulse[:n], voxel[:n]
