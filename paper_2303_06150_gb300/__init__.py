"""GB300 docking pose search behind a C ABI (include/ligen.h).

libligen.so is loaded on first use (or by `load()`); every call raises
ImportError when it has not been built. There is no fallback path.
"""
from . import _abi
from ._abi import LigenError, load
from .api import (BATCHING, DockResult, Ligands, PocketGrid, abi_version, autotune, bucket_size, dock_batch,
                  dock_batch_static, dock_sites, last_error, load_tuning, pack_ligands, pack_touch, pose_grad,
                  pose_offsets, pose_score, prepare_scoring, PreparedScoring, probe_gather, probe_stream,
                  refine_poses, release_workspaces,
                  save_tuning, score_poses, set_workspace_limit, tune_get, tune_set)

__all__ = ["BATCHING", "DockResult", "Ligands", "LigenError", "PocketGrid", "abi_version", "autotune",
           "bucket_size", "dock_batch", "dock_batch_static", "dock_sites", "last_error", "load", "load_tuning",
           "pack_ligands", "pack_touch", "pose_grad", "pose_offsets", "pose_score", "prepare_scoring",
           "PreparedScoring", "probe_gather",
           "probe_stream", "refine_poses", "release_workspaces", "save_tuning", "score_poses",
           "set_workspace_limit", "tune_get", "tune_set"]
