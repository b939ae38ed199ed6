"""Python binding of the docking library: same calls as include/ligen.h.

Argument marshalling only. PyTorch provides the memory (device tensors, or
pinned host tensors for the end-to-end path) and the current CUDA stream;
every step of the search runs in libligen.so's kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi
from ._abi import GridT, LigandsT, ParamsT, check


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# torch's current raw stream of a device without building a Stream object
# (measured: 2.3 us per call through torch.cuda.current_stream); the public
# call where this binding is absent
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream_handle(device: torch.device):
    if device.type == "cuda":
        if _raw_stream is not None:
            return C.c_void_p(_raw_stream(device.index if device.index is not None else torch.cuda.current_device()))
        return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    if torch.cuda.is_available():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return None


class Ligands:
    """A ligand library in CSR form, resident in one memory space.

    Tensors: atom_off int32 [L+1], xyz float32 [sum N, 3], type uint8 [sum N],
    bonds int32 [sum N - L, 2] (local atom ids), rot_off int32 [L+1],
    rot_edge int32 [sum n] (local bond rows). Host copies of the offsets are
    kept for the library's sizing.
    """

    def __init__(self, atom_off, xyz, type_, bonds, rot_off, rot_edge):
        self.atom_off, self.xyz, self.type = atom_off, xyz, type_
        self.bonds, self.rot_off, self.rot_edge = bonds, rot_off, rot_edge
        self.h_atom_off = np.ascontiguousarray(atom_off.cpu().numpy(), np.int32)
        self.h_rot_off = np.ascontiguousarray(rot_off.cpu().numpy(), np.int32)
        self._s = LigandsT(len(self.h_atom_off) - 1, 0, self.h_atom_off.ctypes.data,
                           self.h_rot_off.ctypes.data, atom_off.data_ptr(), xyz.data_ptr(),
                           type_.data_ptr(), bonds.data_ptr(), rot_off.data_ptr(), rot_edge.data_ptr())

    @classmethod
    def from_arrays(cls, lib, device="cuda", pin: bool = False) -> "Ligands":
        """From any object with numpy atom_off/xyz/type/bonds/rot_off/rot_edge."""
        def t(a, dtype):
            x = torch.from_numpy(np.ascontiguousarray(a, dtype))
            if str(device) == "cpu":
                return x.pin_memory() if pin else x
            return x.to(device)
        return cls(t(lib.atom_off, np.int32), t(lib.xyz, np.float32).reshape(-1, 3), t(lib.type, np.uint8),
                   t(lib.bonds, np.int32).reshape(-1, 2), t(lib.rot_off, np.int32), t(lib.rot_edge, np.int32))

    @property
    def n_ligands(self) -> int:
        return len(self.h_atom_off) - 1

    @property
    def n_rot(self) -> np.ndarray:
        return np.diff(self.h_rot_off)

    @property
    def device(self) -> torch.device:
        return self.xyz.device

    def tensors(self):
        return [self.atom_off, self.xyz, self.type, self.bonds, self.rot_off, self.rot_edge]

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in self.tensors())


class PocketGrid:
    """values [nz, ny, nx, nc] float32 (channel innermost), origin, spacing."""

    def __init__(self, values: torch.Tensor, origin, spacing: float):
        assert values.dtype == torch.float32 and values.dim() == 4 and values.is_contiguous()
        self.values = values
        self.origin = tuple(float(v) for v in origin)
        self.spacing = float(spacing)
        nz, ny, nx, nc = values.shape
        self._s = GridT(nx, ny, nz, nc, (C.c_float * 3)(*self.origin), self.spacing, 0, 0,
                        values.data_ptr())

    @classmethod
    def from_array(cls, values, origin, spacing, device="cuda", pin: bool = False) -> "PocketGrid":
        x = torch.from_numpy(np.ascontiguousarray(values, np.float32))
        x = (x.pin_memory() if pin else x) if str(device) == "cpu" else x.to(device)
        return cls(x, origin, spacing)


def _empty(shape, dtype, like: torch.device):
    if like.type == "cuda":
        return torch.empty(shape, dtype=dtype, device=like)
    return torch.empty(shape, dtype=dtype, pin_memory=torch.cuda.is_available())


def pose_offsets(rot_off: np.ndarray, K: int) -> np.ndarray:
    """Start (in floats) of each ligand's K poses: K * (7 l + rot_off[l])."""
    L = len(rot_off) - 1
    return K * (7 * np.arange(L + 1, dtype=np.int64) + np.asarray(rot_off, np.int64))


@dataclass
class DockResult:
    poses: torch.Tensor          # flat float32, see pose_offsets
    scores: torch.Tensor         # [L, K]
    status: torch.Tensor | None  # [L]
    trace: torch.Tensor | None   # flat int16
    top_restart: torch.Tensor | None
    stage_ms: np.ndarray | None
    scores_f64: torch.Tensor | None = None
    samples: int | None = None   # atom samples the search needed (count_samples=True)
    coords: torch.Tensor | None = None   # debug: final grid-unit positions per restart (coords=True)

    def ligand_poses(self, rot_off, l: int) -> torch.Tensor:
        K = self.scores.shape[1]
        off = pose_offsets(rot_off, K)
        n = int(rot_off[l + 1] - rot_off[l])
        return self.poses[off[l]:off[l + 1]].reshape(K, 7 + n)


BATCHING = {"plain": _abi.LIGEN_BATCH_PLAIN, "buckets": _abi.LIGEN_BATCH_BUCKETS,
            "buckets_static": _abi.LIGEN_BATCH_BUCKETS_STATIC, "queue": _abi.LIGEN_BATCH_QUEUE}
GRID_FORMATS = {"f32": _abi.LIGEN_GRID_F32, "f16": _abi.LIGEN_GRID_F16, "bf16": _abi.LIGEN_GRID_BF16}


def dock_batch(ligands: Ligands, grid: PocketGrid, *, restarts: int, torsion_step_deg: int, passes: int,
               top_k: int, seed: int, n_rigid: int = 24, jitter: float = 1.0, out_penalty: float = 5.0,
               status: bool = True, trace: bool = False, top_restart: bool = False,
               stage_ms: bool = False, batching: str = "plain", grid_format: str = "f32",
               rescore_fp64: bool = False, mode: str = "greedy", count_samples: bool = False,
               coords: bool = False, out: DockResult | None = None) -> DockResult:
    """ligen_dock_batch: dock every ligand, keep the top_k poses of each.

    batching: "plain" (one launch), "buckets" (paper §3 classes, one
    persistent launch per atom class, replayed from a CUDA graph),
    "buckets_static" (the same groups, one CTA per work item) or "queue"
    (one persistent launch over the whole library in bucket order).
    grid_format: "f32", "f16" or "bf16" grid records in the docking kernel.
    rescore_fp64: re-score and re-rank the kept poses in FP64 on the GPU;
    the FP64 scores are returned in `scores_f64`.
    mode: "greedy" (the search) or "exhaustive" (every combination of cube
    rotation and torsion increments per restart; small ligands only).
    count_samples: return in `samples` the atom samples the search needed
    (the call then waits for its work).
    coords: return in `coords` (debug) the docking kernel's final FP32 atom
    positions of every restart, in grid units, [3 * R * sum N] flat."""
    lib = _abi.load()
    if out is None:
        out = _dock_outputs(ligands, restarts, passes, top_k, (), status, trace, top_restart, stage_ms, rescore_fp64)
        if coords:
            out.coords = _empty((3 * restarts * int(ligands.h_atom_off[-1]),), torch.float32, ligands.device)
    p = _dock_params(ligands.device, out, restarts, torsion_step_deg, passes, top_k, seed, n_rigid, jitter,
                     out_penalty, batching, grid_format, rescore_fp64, mode)
    if out.coords is not None:
        p.coords = _ptr(out.coords)
    n_samples = C.c_int64(0)
    if count_samples:
        p.samples = C.cast(C.pointer(n_samples), C.c_void_p)
    check(lib.ligen_dock_batch(C.byref(ligands._s), C.byref(grid._s), C.byref(p), _ptr(out.poses),
                               _ptr(out.scores)))
    out.samples = int(n_samples.value) if count_samples else None
    return out


def _dock_outputs(ligands, restarts, passes, top_k, lead, status, trace, top_restart, stage_ms, rescore_fp64):
    L, dev = ligands.n_ligands, ligands.device
    n_sum = int(ligands.h_rot_off[-1])
    return DockResult(
        poses=_empty(lead + (top_k * (7 * L + n_sum),), torch.float32, dev),
        scores=_empty(lead + (L, top_k), torch.float32, dev),
        status=_empty((L,), torch.int32, dev) if status else None,
        trace=_empty(lead + (restarts * int(np.sum(1 + passes * np.diff(ligands.h_rot_off))),), torch.int16, dev)
        if trace else None,
        top_restart=_empty(lead + (L, top_k), torch.int32, dev) if top_restart else None,
        stage_ms=np.zeros(_abi.LIGEN_N_STAGES, np.float32) if stage_ms else None,
        scores_f64=_empty(lead + (L, top_k), torch.float64, dev) if rescore_fp64 else None,
    )


MODES = {"greedy": 0, "exhaustive": 1}


def _dock_params(dev, out, restarts, torsion_step_deg, passes, top_k, seed, n_rigid, jitter, out_penalty,
                 batching, grid_format, rescore_fp64, mode="greedy"):
    return ParamsT(restarts, n_rigid, torsion_step_deg, passes, top_k, MODES[mode], int(seed) & ((1 << 64) - 1),
                   float(jitter), float(out_penalty), _stream_handle(dev), _ptr(out.status), _ptr(out.trace),
                   _ptr(out.top_restart),
                   out.stage_ms.ctypes.data if out.stage_ms is not None else None, BATCHING[batching],
                   GRID_FORMATS[grid_format], int(bool(rescore_fp64)), 0,
                   _ptr(out.scores_f64) if rescore_fp64 else None)


def dock_sites(ligands: Ligands, grids: list, *, restarts: int, torsion_step_deg: int, passes: int,
               top_k: int, seed: int, n_rigid: int = 24, jitter: float = 1.0, out_penalty: float = 5.0,
               status: bool = True, trace: bool = False, top_restart: bool = False,
               stage_ms: bool = False, batching: str = "plain", grid_format: str = "f32",
               rescore_fp64: bool = False, mode: str = "greedy", out: DockResult | None = None) -> DockResult:
    """ligen_dock_sites: dock the library into every grid of `grids` (the
    docking sites). Outputs gain a leading site axis ([n_sites, L, K] scores,
    [n_sites, pose floats] poses, ...); status stays [L]. Site g's slice
    equals dock_batch(ligands, grids[g], ...) with the same settings."""
    lib = _abi.load()
    n = len(grids)
    if n < 1:
        raise ValueError("dock_sites needs at least one grid")
    if out is None:
        out = _dock_outputs(ligands, restarts, passes, top_k, (n,), status, trace, top_restart, stage_ms,
                            rescore_fp64)
    arr = (GridT * n)(*[g._s for g in grids])
    p = _dock_params(ligands.device, out, restarts, torsion_step_deg, passes, top_k, seed, n_rigid, jitter,
                     out_penalty, batching, grid_format, rescore_fp64, mode)
    check(lib.ligen_dock_sites(C.byref(ligands._s), arr, n, C.byref(p), _ptr(out.poses), _ptr(out.scores)))
    return out


def dock_batch_static(ligands: Ligands, grid: PocketGrid, *, restarts: int, torsion_step_deg: int, passes: int,
                      top_k: int, seed: int, n_rigid: int = 24, jitter: float = 1.0, out_penalty: float = 5.0,
                      status: bool = True, trace: bool = False, top_restart: bool = False,
                      batching: str = "plain", grid_format: str = "f32", rescore_fp64: bool = False,
                      mode: str = "greedy", stage_ms: bool = False, count_samples: bool = False,
                      out: DockResult | None = None) -> DockResult:
    """ligen_dock_batch_static: ligen_dock_batch with the library's fixed
    device scratch instead of an allocated workspace (device tensors only).

    Pass `out` (device tensors allocated beforehand) to make the call itself
    allocate nothing; without it the binding allocates the outputs with torch.
    Every setting is passed to the library as given: it runs the plain launch
    over FP32 records only and rejects the others (LigenError, code -2)."""
    lib = _abi.load()
    if out is None:
        out = _dock_outputs(ligands, restarts, passes, top_k, (), status, trace, top_restart, stage_ms, rescore_fp64)
    p = _dock_params(ligands.device, out, restarts, torsion_step_deg, passes, top_k, seed, n_rigid, jitter,
                     out_penalty, batching, grid_format, rescore_fp64, mode)
    n_samples = C.c_int64(0)
    if count_samples:
        p.samples = C.cast(C.pointer(n_samples), C.c_void_p)
    check(lib.ligen_dock_batch_static(C.byref(ligands._s), C.byref(grid._s), C.byref(p), _ptr(out.poses),
                                      _ptr(out.scores)))
    return out


def score_poses(ligands: Ligands, grid: PocketGrid, poses: torch.Tensor, poses_per_ligand: int,
                out_penalty: float = 5.0, out: torch.Tensor | None = None) -> torch.Tensor:
    """ligen_score_poses: scores [L, poses_per_ligand] of packed poses."""
    lib = _abi.load()
    L = ligands.n_ligands
    if out is None:
        out = _empty((L, poses_per_ligand), torch.float32, poses.device)
    check(lib.ligen_score_poses(C.byref(ligands._s), C.byref(grid._s), poses_per_ligand, _ptr(poses),
                                float(out_penalty), _ptr(out), _stream_handle(poses.device)))
    return out


class PreparedScoring:
    """ligen_prepare_scoring: grid records and packed library built once for
    many score() calls (ligen_score_prepared); release() (or garbage
    collection) frees them with ligen_release_prepared."""

    def __init__(self, ligands: Ligands, grid: PocketGrid):
        lib = _abi.load()
        h = C.c_void_p()
        check(lib.ligen_prepare_scoring(C.byref(ligands._s), C.byref(grid._s), _stream_handle(ligands.device),
                                        C.byref(h)))
        self._h = h
        self.n_ligands = ligands.n_ligands

    def score(self, poses: torch.Tensor, poses_per_ligand: int, out_penalty: float = 5.0,
              out: torch.Tensor | None = None) -> torch.Tensor:
        if self._h is None:
            raise ValueError("released")
        if out is None:
            out = _empty((self.n_ligands, poses_per_ligand), torch.float32, poses.device)
        check(_abi.load().ligen_score_prepared(self._h, poses_per_ligand, _ptr(poses), float(out_penalty),
                                               _ptr(out), _stream_handle(poses.device)))
        return out

    def release(self) -> None:
        if getattr(self, "_h", None) is not None:
            h, self._h = self._h, None
            check(_abi.load().ligen_release_prepared(h))

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def prepare_scoring(ligands: Ligands, grid: PocketGrid) -> PreparedScoring:
    """Grid records and packed library for repeated scoring (see PreparedScoring)."""
    return PreparedScoring(ligands, grid)


def pose_grad(ligands: Ligands, grid: PocketGrid, poses: torch.Tensor, poses_per_ligand: int,
              out_penalty: float = 5.0):
    """ligen_pose_grad: (scores [L, P], dS/dpose in the packing of `poses`)."""
    lib = _abi.load()
    L = ligands.n_ligands
    scores = _empty((L, poses_per_ligand), torch.float32, poses.device)
    grads = _empty(tuple(poses.shape), torch.float32, poses.device)
    check(lib.ligen_pose_grad(C.byref(ligands._s), C.byref(grid._s), poses_per_ligand, _ptr(poses),
                              float(out_penalty), _ptr(scores), _ptr(grads), _stream_handle(poses.device)))
    return scores, grads


def refine_poses(ligands: Ligands, grid: PocketGrid, poses: torch.Tensor, poses_per_ligand: int, *,
                 steps: int = 50, step_t: float = 0.1, step_q: float = 0.02, step_theta: float = 0.05,
                 out_penalty: float = 5.0, accept: bool = False, inplace: bool = False):
    """ligen_refine_poses: (refined poses, scores [L, P], accept flags or None)."""
    lib = _abi.load()
    L = ligands.n_ligands
    out = poses if inplace else poses.clone()
    scores = _empty((L, poses_per_ligand), torch.float32, poses.device)
    acc = _empty((L * poses_per_ligand, steps), torch.int8, poses.device) if accept else None
    check(lib.ligen_refine_poses(C.byref(ligands._s), C.byref(grid._s), poses_per_ligand, _ptr(out),
                                 float(out_penalty), int(steps), float(step_t), float(step_q), float(step_theta),
                                 _ptr(scores), _ptr(acc), _stream_handle(poses.device)))
    return out, scores, acc


def _pose_lengths(ligands: Ligands, poses_per_ligand: int, device) -> torch.Tensor:
    n = torch.from_numpy(np.diff(ligands.h_rot_off).astype(np.int64) + 7)
    return n.repeat_interleave(poses_per_ligand).to(device)


class PoseScore(torch.autograd.Function):
    """Differentiable pose score: forward ligen_score_poses, backward
    ligen_pose_grad (coordinates rebuilt in the backward pass)."""

    @staticmethod
    def forward(ctx, poses, ligands, grid, poses_per_ligand, out_penalty):
        ctx.save_for_backward(poses)
        ctx.args = (ligands, grid, poses_per_ligand, out_penalty)
        return score_poses(ligands, grid, poses.detach(), poses_per_ligand, out_penalty)

    @staticmethod
    def backward(ctx, grad_scores):
        (poses,) = ctx.saved_tensors
        ligands, grid, P, pen = ctx.args
        _, grads = pose_grad(ligands, grid, poses.detach().contiguous(), P, pen)
        weight = grad_scores.reshape(-1).repeat_interleave(_pose_lengths(ligands, P, poses.device))
        return grads * weight, None, None, None, None


def pose_score(poses: torch.Tensor, ligands: Ligands, grid: PocketGrid, poses_per_ligand: int,
               out_penalty: float = 5.0) -> torch.Tensor:
    """Scores [L, P] of packed poses, differentiable with respect to `poses`."""
    return PoseScore.apply(poses, ligands, grid, poses_per_ligand, out_penalty)


def pack_ligands(ligands: Ligands, n_channels: int):
    """ligen_pack_ligands: (frag_bits [sum n, 8] uint32 as int32, axis [sum n, 2], bucket [L], status [L])."""
    lib = _abi.load()
    L, dev = ligands.n_ligands, ligands.device
    n_sum = int(ligands.h_rot_off[-1])
    bits = _empty((max(n_sum, 1), 8), torch.int32, dev)
    axis = _empty((max(n_sum, 1), 2), torch.int32, dev)
    bucket = _empty((L,), torch.int32, dev)
    status = _empty((L,), torch.int32, dev)
    check(lib.ligen_pack_ligands(C.byref(ligands._s), n_channels, _ptr(bits), _ptr(axis), _ptr(bucket),
                                 _ptr(status), _stream_handle(dev)))
    return bits[:n_sum], axis[:n_sum], bucket, status


def pack_touch(ligands: Ligands, n_channels: int) -> torch.Tensor:
    """ligen_pack_touch: bond interaction masks [sum n] (uint32 bits as int64)."""
    lib = _abi.load()
    n_sum = int(ligands.h_rot_off[-1])
    out = _empty((max(n_sum, 1),), torch.int32, ligands.device)
    check(lib.ligen_pack_touch(C.byref(ligands._s), n_channels, _ptr(out), _stream_handle(ligands.device)))
    return out[:n_sum].to(torch.int64) & 0xFFFFFFFF


def bucket_size(max_atoms: int) -> dict:
    """ligen_bucket_size: paper Eq. 1 factors for the docking kernel."""
    lib = _abi.load()
    b, sm, t, ws = (C.c_int32() for _ in range(4))
    l = check(lib.ligen_bucket_size(max_atoms, C.byref(b), C.byref(sm), C.byref(t), C.byref(ws)))
    return dict(l=int(l), b=b.value, sm=sm.value, t=t.value, ws=ws.value)


def probe_gather(records: torch.Tensor, loads_per_thread: int = 256, bytes_per_load: int = 32) -> dict:
    """ligen_probe_gather: random-record load rate over `records` (device, [n, 8] float32)."""
    lib = _abi.load()
    assert records.is_cuda and records.dtype == torch.float32 and records.shape[-1] == 8
    sink = torch.zeros(1, dtype=torch.float32, device=records.device)
    ms = C.c_float()
    loads = C.c_double()
    check(lib.ligen_probe_gather(_ptr(records), records.numel() // 8, bytes_per_load, loads_per_thread,
                                 _ptr(sink), C.byref(loads), C.byref(ms), _stream_handle(records.device)))
    return dict(loads=loads.value, ms=ms.value, loads_per_s=loads.value / (ms.value * 1e-3),
                gbs=loads.value * bytes_per_load / (ms.value * 1e-3) / 1e9)


def set_workspace_limit(nbytes: int) -> None:
    """ligen_set_workspace_limit: cap every internal workspace (<= 0: no cap)."""
    check(_abi.load().ligen_set_workspace_limit(int(nbytes)))


def probe_stream(buffer: torch.Tensor, passes: int = 20) -> dict:
    """ligen_probe_stream: L2 streaming read bandwidth over `buffer` (device)."""
    lib = _abi.load()
    assert buffer.is_cuda and buffer.is_contiguous()
    nbytes = buffer.numel() * buffer.element_size() // 16 * 16
    sink = torch.zeros(1, dtype=torch.float32, device=buffer.device)
    ms = C.c_float()
    done = C.c_double()
    check(lib.ligen_probe_stream(_ptr(buffer), nbytes, int(passes), _ptr(sink), C.byref(done), C.byref(ms),
                                 _stream_handle(buffer.device)))
    return dict(bytes=done.value, ms=ms.value, gbs=done.value / (ms.value * 1e-3) / 1e9)


def tune_get() -> list:
    """ligen_tune_get for every bucket: [(lanes, restarts_per_cta)] * 44."""
    lib = _abi.load()
    out = []
    for b in range(_abi.LIGEN_N_BUCKETS):
        lanes, rpc = C.c_int32(), C.c_int32()
        check(lib.ligen_tune_get(b, C.byref(lanes), C.byref(rpc)))
        out.append((lanes.value, rpc.value))
    return out


def tune_set(table) -> None:
    """ligen_tune_set from {bucket: (lanes, restarts_per_cta)} or a 44-list."""
    lib = _abi.load()
    items = table.items() if isinstance(table, dict) else enumerate(table)
    for b, (lanes, rpc) in items:
        check(lib.ligen_tune_set(int(b), int(lanes), int(rpc)))


def autotune(ligands: Ligands, grid: PocketGrid, *, restarts: int, torsion_step_deg: int, passes: int,
             top_k: int, seed: int, n_rigid: int = 24, jitter: float = 1.0, out_penalty: float = 5.0,
             sample: int = 256, grid_format: str = "f32") -> dict:
    """ligen_autotune: time the candidate shapes per bucket on (a sample of)
    this library and store the fastest; returns {bucket: (lanes, rpc, ms per ligand)}."""
    lib = _abi.load()
    p = ParamsT(restarts, n_rigid, torsion_step_deg, passes, top_k, 0, int(seed) & ((1 << 64) - 1),
                float(jitter), float(out_penalty), _stream_handle(ligands.device), None, None, None, None,
                _abi.LIGEN_BATCH_PLAIN, GRID_FORMATS[grid_format], 0, 0, None)
    lanes = np.zeros(_abi.LIGEN_N_BUCKETS, np.int32)
    rpc = np.zeros(_abi.LIGEN_N_BUCKETS, np.int32)
    ms = np.zeros(_abi.LIGEN_N_BUCKETS, np.float32)
    check(lib.ligen_autotune(C.byref(ligands._s), C.byref(grid._s), C.byref(p), int(sample),
                             lanes.ctypes.data, rpc.ctypes.data, ms.ctypes.data))
    return {b: (int(lanes[b]), int(rpc[b]), float(ms[b])) for b in range(len(lanes)) if lanes[b]}


def save_tuning(path: str) -> None:
    """Write the current device's tuning table as JSON keyed by GPU name."""
    import json
    import os
    name = torch.cuda.get_device_name()
    data = json.load(open(path)) if os.path.exists(path) else {}
    data[name] = {str(b): list(v) for b, v in enumerate(tune_get())}
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def load_tuning(path: str) -> bool:
    """Load this GPU's entry of a JSON tuning file, if present."""
    import json
    data = json.load(open(path))
    entry = data.get(torch.cuda.get_device_name())
    if not entry:
        return False
    tune_set({int(b): tuple(v) for b, v in entry.items()})
    return True


def release_workspaces() -> None:
    check(_abi.load().ligen_release_workspaces())


def last_error() -> str:
    return _abi.load().ligen_last_error().decode()


def abi_version() -> int:
    return int(_abi.load().ligen_abi_version())
