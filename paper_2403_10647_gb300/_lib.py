"""ctypes declarations of the C ABI in include/grid.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LIB_PATH = _build.LIB_PATH

GRID_OK = 0
GRID_EINVAL = -1
GRID_ENOMEM = -2
GRID_EOVERFLOW = -3
GRID_EAGAIN = -4
GRID_ETIMEOUT = -5
GRID_ECUDA = -6
GRID_ENOSPC = -7
GRID_ENOTREADY = -8
GRID_ELIMIT = -9

# cudaStreamLegacy: the handle of the legacy default stream (grid_ctx_set_stream)
CUDA_STREAM_LEGACY = 1
GRID_RES_MAX = 65535
GRID_PAIRS_FUSED = 0
GRID_PAIRS_EMIT = 1
GRID_PAIRS_PER_OBJECT = 2
GRID_PAIRS_REGEN = 3

c_int32, c_int64, c_float, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p
P = ctypes.POINTER


class GridInfo(ctypes.Structure):
    _fields_ = [
        ("lo", c_float * 3),
        ("hi", c_float * 3),
        ("scale", c_float * 3),
        ("res", c_int32 * 3),
        ("key_bits", c_int32),
        ("ncells", c_int64),
        ("nrefs", c_int64),
        ("n", c_int64),
    ]


class GridBuf(ctypes.Structure):
    _fields_ = [("ptr", c_void_p), ("count", c_int64), ("bytes", ctypes.c_size_t)]


class GridMesh(ctypes.Structure):
    _fields_ = [("verts", c_void_p), ("nverts", c_int64), ("tris", c_void_p), ("n", c_int64),
                ("lam", c_float), ("reserved", c_int32)]


class GridKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class GridOpts(ctypes.Structure):
    _fields_ = [("radix_bits", c_int32), ("pair_gen", c_int32), ("cull", c_int32), ("tile_shape", c_int32),
                ("local_bits", c_int32), ("reserved", c_int32 * 3)]


class GridServeOpts(ctypes.Structure):
    _fields_ = [("nworkers", c_int32), ("max_batch", c_int32), ("batch_pairs", c_int64),
                ("hbm_budget", c_int64), ("radix_bits", c_int32), ("arrival_order", c_int32),
                ("small_workers", c_int32), ("tune_meshes", c_int32), ("reserved", c_int32 * 2)]


class GridServeStats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("failed", c_int64), ("refused", c_int64),
                ("batches", c_int64), ("batched_requests", c_int64), ("queued", c_int64),
                ("reserved_bytes", c_int64), ("peak_reserved_bytes", c_int64), ("budget_bytes", c_int64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("p50_service_us", ctypes.c_double),
                ("builds_per_s", ctypes.c_double), ("elapsed_s", ctypes.c_double)]


# name -> (restype, argtypes); one entry per function declared in include/grid.h
SIGNATURES = {
    "grid_ctx_create": (c_int32, [ctypes.c_int, P(GridOpts), P(c_void_p)]),
    "grid_ctx_destroy": (None, [c_void_p]),
    "grid_ctx_set_stream": (c_int32, [c_void_p, c_void_p]),
    "grid_ctx_get_opts": (c_int32, [c_void_p, P(GridOpts)]),
    "grid_ctx_set_opts": (c_int32, [c_void_p, P(GridOpts)]),
    "grid_ctx_mem_in_use": (c_int32, [c_void_p, P(c_int64)]),
    "grid_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "grid_version": (ctypes.c_char_p, []),
    "grid_ctx_profile": (c_int32, [c_void_p, ctypes.c_int]),
    "grid_ctx_counters": (c_int32, [c_void_p, P(c_int64), P(c_int64)]),
    "grid_ctx_sort_plan": (c_int32, [c_void_p, c_int32, c_int64, c_int64, P(c_int32), P(c_int32)]),
    "grid_ctx_autotune": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_float, c_int32, P(GridOpts),
                                    P(ctypes.c_double)]),
    "grid_ctx_autotune_batched": (c_int32, [c_void_p, P(GridMesh), c_int32, c_int32, P(GridOpts),
                                            P(ctypes.c_double)]),
    "grid_ctx_kernel_stats": (c_int32, [c_void_p, c_void_p, ctypes.c_int, P(ctypes.c_int)]),
    "grid_build": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_float, P(GridBuf), P(GridBuf),
                             P(GridInfo)]),
    "grid_build_host": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_float, c_void_p, c_int64,
                                  c_void_p, c_int64, P(GridInfo)]),
    "grid_build_batched": (c_int32, [c_void_p, P(GridMesh), c_int32, P(GridBuf), P(GridBuf), P(GridInfo),
                                     P(c_int64), P(c_int64)]),
    "grid_buf_free": (None, [c_void_p, P(GridBuf)]),
    "grid_bounds": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, P(c_float), P(c_float)]),
    "grid_plan": (c_int32, [P(c_float), P(c_float), c_int64, c_float, P(GridInfo)]),
    "grid_count_scan": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, P(GridInfo), c_void_p,
                                  P(c_int64)]),
    "grid_emit_pairs": (c_int32, [c_void_p, c_void_p, c_int64, c_int64, P(GridInfo), c_void_p, c_void_p]),
    "grid_cull_pairs": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, P(GridInfo), c_void_p, c_int64,
                                  c_void_p, c_void_p, P(c_int64)]),
    "grid_emit_pairs_per_object": (c_int32, [c_void_p, c_void_p, c_int64, c_int64, P(GridInfo), c_void_p,
                                             c_void_p]),
    "grid_sort_pairs": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p]),
    "grid_extract_ranges": (c_int32, [c_void_p, c_void_p, c_int64, c_int64, c_void_p]),
    "grid_extract_ranges_noalloc": (c_int32, [c_void_p, c_int64, c_int64, c_void_p, c_void_p]),
    "grid_selftest_wait_timeout": (c_int32, [c_void_p, P(ctypes.c_double)]),
    "grid_jitter": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_float, ctypes.c_uint64]),
    "grid_serve_create": (c_int32, [ctypes.c_int, P(GridServeOpts), P(c_void_p)]),
    "grid_serve_destroy": (None, [c_void_p]),
    "grid_serve_register": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_float, P(c_int32)]),
    "grid_serve_submit": (c_int32, [c_void_p, c_int32, c_void_p, c_float, ctypes.c_uint64, P(ctypes.c_uint64)]),
    "grid_serve_poll": (c_int32, [c_void_p, ctypes.c_uint64, P(GridBuf), P(GridBuf), P(GridInfo)]),
    "grid_serve_wait": (c_int32, [c_void_p, ctypes.c_uint64, c_int64, P(GridBuf), P(GridBuf), P(GridInfo)]),
    "grid_serve_release": (c_int32, [c_void_p, ctypes.c_uint64]),
    "grid_serve_get_stats": (c_int32, [c_void_p, P(GridServeStats), ctypes.c_int]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Loads the compiled library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA grid library not built ({LIB_PATH} missing); run __graft_entry__.build() "
                "or python -m paper_2403_10647_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class GridError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = load().grid_strerror(code).decode()
        super().__init__(f"{what}: {msg} (code {code})" if what else f"{msg} (code {code})")
        self.code = code


def check(code: int, what: str = "") -> None:
    if code != GRID_OK:
        raise GridError(code, what)
