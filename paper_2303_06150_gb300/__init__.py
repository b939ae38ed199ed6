"""GB300 docking pose search behind a C ABI (include/ligen.h).

libligen.so is loaded on first use (or by `load()`); every call raises
ImportError when it has not been built. There is no fallback path.
"""
from . import _abi
from ._abi import LigenError, load
from .api import (DockResult, Ligands, PocketGrid, abi_version, bucket_size, dock_batch, dock_batch_static,
                  last_error,
                  pack_ligands, pose_offsets, probe_gather, release_workspaces, score_poses)

__all__ = ["DockResult", "Ligands", "LigenError", "PocketGrid", "abi_version", "bucket_size", "dock_batch",
           "dock_batch_static",
           "last_error", "load", "pack_ligands", "pose_offsets", "probe_gather", "release_workspaces",
           "score_poses"]
