"""The C ABI without a GPU: libet.so builds, loads, exports every function
that the headers in include/ declare, and refuses to run without a CUDA
device (no CPU fallback).  No compute call is made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


@pytest.fixture(scope="module")
def libet():
    from paper_1311_5334_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(et_[a-z0-9_]+)\s*\(", text)) - {"et_alloc_fn", "et_free_fn"})


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["et_view_create", "et_track_find", "et_track_fetch", "et_server_submit",
                     "et_server_poll", "et_batch_find", "et_last_error", "et_frames_run", "et_frames_fetch",
                     "et_frames_to_batch"]:
        assert required in names


def test_every_declared_symbol_is_exported(libet):
    missing = [n for n in declared_functions() if not hasattr(libet, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1311_5334_gb300 import et
    assert set(declared_functions()) <= set(et._SIGS)


def test_abi_version_and_status_strings(libet):
    libet.et_abi_version.restype = C.c_int32
    assert libet.et_abi_version() == 3
    libet.et_status_string.restype = C.c_char_p
    libet.et_status_string.argtypes = [C.c_int32]
    assert libet.et_status_string(-3) == b"duplicate grain"


def test_track_layout_matches_header():
    from paper_1311_5334_gb300 import et
    assert et.TRACK_DTYPE.itemsize == 64
    assert C.sizeof(et.Params) == 48
    assert C.sizeof(et.Stats) == 8 * 8 + 4 * 4 + 4 * 2 + 4 * 6 + 8
    assert C.sizeof(et.FrameParams) == 4 * 4 + 4 * 3 + 4 * 3 + 4 + 4
    assert C.sizeof(et.FramesStats) == 8 * 4 + 4 * 4


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_no_gpu_means_an_error_not_a_fallback(libet):
    from paper_1311_5334_gb300 import et
    h = C.c_void_p()
    st = et.lib().et_ctx_create(0, C.byref(h))
    assert st == et.CUDA
    assert b"CUDA" in et.lib().et_last_error() or b"device" in et.lib().et_last_error()
