"""ctypes view of include/ligen.h and the loader of libligen.so.

The library must be present (built by `__graft_entry__.build()` or
`python -m paper_2303_06150_gb300.build`); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libligen.so")

LIGEN_OK = 0
LIGEN_ERR_INVALID_ARG = -1
LIGEN_ERR_UNSUPPORTED = -2
LIGEN_ERR_OOM = -3
LIGEN_ERR_CUDA = -4
LIGEN_ERR_TIMEOUT = -5
LIGEN_ERR_BAD_LIGAND = -6
LIGEN_N_STAGES = 5
LIGEN_BATCH_PLAIN = 0
LIGEN_BATCH_BUCKETS = 1
LIGEN_BATCH_BUCKETS_STATIC = 2
LIGEN_BATCH_QUEUE = 3
LIGEN_N_BUCKETS = 44
LIGEN_GRID_F32 = 0
LIGEN_GRID_F16 = 1
LIGEN_GRID_BF16 = 2
STAGE_NAMES = ("h2d", "grid_prep", "pack", "dock", "topk_d2h")

P = C.c_void_p


class LigandsT(C.Structure):
    _fields_ = [("n_ligands", C.c_int32), ("reserved", C.c_int32), ("h_atom_off", P), ("h_rot_off", P),
                ("atom_off", P), ("xyz", P), ("type", P), ("bonds", P), ("rot_off", P), ("rot_edge", P)]


class GridT(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nc", C.c_int32),
                ("origin", C.c_float * 3), ("spacing", C.c_float), ("dtype", C.c_int32),
                ("reserved", C.c_int32), ("data", P)]


class ParamsT(C.Structure):
    _fields_ = [("restarts", C.c_int32), ("n_rigid", C.c_int32), ("torsion_step_deg", C.c_int32),
                ("passes", C.c_int32), ("top_k", C.c_int32), ("mode", C.c_int32), ("seed", C.c_uint64),
                ("jitter", C.c_float), ("out_penalty", C.c_float), ("stream", P), ("status", P),
                ("trace", P), ("top_restart", P), ("stage_ms", P), ("batching", C.c_int32),
                ("grid_format", C.c_int32), ("rescore_fp64", C.c_int32), ("reserved3", C.c_int32),
                ("scores_f64", P), ("samples", P), ("coords", P)]


# Every function include/ligen.h declares, with its ctypes signature.
SIGNATURES = {
    "ligen_dock_batch": (C.c_int, [P, P, P, P, P]),
    "ligen_dock_batch_static": (C.c_int, [P, P, P, P, P]),
    "ligen_dock_sites": (C.c_int, [P, P, C.c_int32, P, P, P]),
    "ligen_score_poses": (C.c_int, [P, P, C.c_int32, P, C.c_float, P, P]),
    "ligen_pose_grad": (C.c_int, [P, P, C.c_int32, P, C.c_float, P, P, P]),
    "ligen_refine_poses": (C.c_int, [P, P, C.c_int32, P, C.c_float, C.c_int32, C.c_float, C.c_float, C.c_float,
                                     P, P, P]),
    "ligen_pack_ligands": (C.c_int, [P, C.c_int32, P, P, P, P, P]),
    "ligen_bucket_size": (C.c_int64, [C.c_int32, P, P, P, P]),
    "ligen_probe_gather": (C.c_int, [P, C.c_int64, C.c_int32, C.c_int32, P, P, P, P]),
    "ligen_tune_set": (C.c_int, [C.c_int32, C.c_int32, C.c_int32]),
    "ligen_tune_get": (C.c_int, [C.c_int32, P, P]),
    "ligen_autotune": (C.c_int, [P, P, P, C.c_int32, P, P, P]),
    "ligen_release_workspaces": (C.c_int, []),
    "ligen_last_error": (C.c_char_p, []),
    "ligen_probe_stream": (C.c_int, [P, C.c_int64, C.c_int32, P, P, P, P]),
    "ligen_set_workspace_limit": (C.c_int, [C.c_int64]),
    "ligen_pack_touch": (C.c_int, [P, C.c_int32, P, P]),
    "ligen_abi_version": (C.c_int, []),
    "ligen_prepare_scoring": (C.c_int, [P, P, P, P]),
    "ligen_score_prepared": (C.c_int, [P, C.c_int32, P, C.c_float, P, P]),
    "ligen_release_prepared": (C.c_int, [P]),
}

_lock = threading.Lock()
_lib = None


class LigenError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ligen error {code}: {msg}")
        self.code = code


def load(path: str | None = None):
    """Load libligen.so once; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"{p} is missing: build it with `python -m paper_2303_06150_gb300.build`")
            lib = C.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def check(rc: int) -> int:
    if rc < 0:
        raise LigenError(rc, load().ligen_last_error().decode())
    return rc
