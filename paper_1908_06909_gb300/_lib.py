"""ctypes declarations of libtetproj.so (include/tetproj.h); marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtetproj.so")

# status codes (include/tetproj.h)
OK = 0
ERR_ARG = 1
ERR_INDEX = 2
ERR_DEGENERATE_TET = 3
ERR_NONMANIFOLD = 4
ERR_NONCONVEX = 5
ERR_CUDA = 6
ERR_OOM = 7
ERR_RAY_LIMIT = 8
ERR_TIMEOUT = 9
ERR_SOURCE_INSIDE = 10
ERR_TOO_LARGE = 11

FILTERED = 0
PLAIN_FP64 = 1
ORDER_ROW = 0
ORDER_MORTON = 1
SCATTER_ATOMIC = 0
SCATTER_WARP = 1
SCATTER_SORT = 2
FLAG_RSTAR_ENTRY = 1
FLAG_ACC64 = 2
FLAG_ACC32 = 4

c_vp = ctypes.c_void_p
c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_dbl = ctypes.c_double


class Options(ctypes.Structure):
    _fields_ = [("precision", c_i32), ("channels", c_i32), ("tile_u", c_i32), ("tile_v", c_i32),
                ("order", c_i32), ("scatter", c_i32), ("max_steps", c_i32), ("flags", c_i32)]


class Stats(ctypes.Structure):
    _fields_ = [("rays", c_i64), ("hits", c_i64), ("segments", c_i64), ("fp64_filter", c_i64),
                ("exact", c_i64), ("sos", c_i64), ("bvh_nodes", c_i64), ("bvh_faces", c_i64),
                ("deferred", c_i64), ("error", c_i32), ("error_count", c_i32), ("grazing", c_i64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RStarInfo(ctypes.Structure):
    _fields_ = [("nodes", c_i64), ("leaves", c_i64), ("entries", c_i64), ("depth", c_i32),
                ("min_fill", c_i32), ("max_fill", c_i32), ("ok", c_i32)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("nt", c_i64), ("nv", c_i64), ("nboundary", c_i64), ("nbvh_nodes", c_i64),
                ("nflipped", c_i64), ("device_bytes", c_i64), ("bbox", c_dbl * 6)]


# name -> (restype, argtypes); mirrors include/tetproj.h
SIGNATURES = {
    "tetproj_version": (c_i32, []),
    "tetproj_launch_count": (c_i64, []),
    "tetproj_default_options": (None, [ctypes.POINTER(Options)]),
    "tetproj_status_string": (ctypes.c_char_p, [c_i32]),
    "tetproj_mesh_create": (c_i32, [c_vp, c_i64, c_vp, c_i64, ctypes.POINTER(c_vp)]),
    "tetproj_mesh_destroy": (c_i32, [c_vp]),
    "tetproj_mesh_get_info": (c_i32, [c_vp, ctypes.POINTER(MeshInfo)]),
    "tetproj_mesh_reserve": (c_i32, [c_vp, c_i32, c_i32]),
    "tetproj_mesh_topology_host": (c_i32, [c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "tetproj_mesh_stats_reset": (c_i32, [c_vp, c_vp]),
    "tetproj_mesh_stats_read": (c_i32, [c_vp, c_vp, ctypes.POINTER(Stats)]),
    "tetproj_geometry_create": (c_i32, [c_dbl, c_dbl, c_i32, c_i32, c_dbl, c_dbl, c_vp, c_i32,
                                        ctypes.POINTER(c_vp)]),
    "tetproj_geometry_destroy": (c_i32, [c_vp]),
    "tetproj_geometry_rays": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "tetproj_forward": (c_i32, [c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(Options), c_vp]),
    "tetproj_backward": (c_i32, [c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(Options), c_vp]),
    "tetproj_backward_noalloc": (c_i32, [c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(Options), c_vp]),
    "tetproj_forward_rays": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, c_vp,
                                     ctypes.POINTER(Options), c_vp]),
    "tetproj_backward_rays": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, c_vp,
                                      ctypes.POINTER(Options), c_vp]),
    "tetproj_trace_rays": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp,
                                   ctypes.POINTER(Options), c_vp]),
    "tetproj_batch_create": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, ctypes.POINTER(c_vp)]),
    "tetproj_batch_bind": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "tetproj_batch_forward": (c_i32, [c_vp, c_vp]),
    "tetproj_batch_backward": (c_i32, [c_vp, c_vp]),
    "tetproj_batch_set_wait": (c_i32, [c_vp, c_i32, c_i32]),
    "tetproj_batch_destroy": (c_i32, [c_vp]),
    "tetproj_forward_mt": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "tetproj_forward_rays_mt": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "tetproj_entry": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "tetproj_rstar_build_host": (c_i32, [c_vp, c_i64, c_vp, c_i64, c_vp]),
    "tetproj_fma64_probe": (c_i32, [c_i64, c_vp, ctypes.POINTER(ctypes.c_double), c_vp]),
    "tetproj_side_host": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_vp]),
    "tetproj_side_device": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp]),
}

_lib = None


class TetprojError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = load().tetproj_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} (status {code})")


def load():
    """Load libtetproj.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
            f"g.build()'` (there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(code: int, what: str):
    if code != OK:
        raise TetprojError(code, what)
