"""Python view of the FP64 docking oracle (ligen_oracle.cpp).

TEST INFRASTRUCTURE. Only the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg may import this package. It shares no code with
the CUDA library and never imports it.

The oracle is single-threaded per call; `dock_library` fans ligands out over
threads (ctypes releases the GIL during each call).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ligen_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (g++, C++17, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Ligand(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("n_rot", C.c_int32), ("xyz", C.c_void_p),
                ("type", C.c_void_p), ("bonds", C.c_void_p), ("rot_edge", C.c_void_p)]


class GridS(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nc", C.c_int32),
                ("origin", C.c_double * 3), ("spacing", C.c_double), ("v", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("restarts", C.c_int32), ("n_rigid", C.c_int32), ("step_deg", C.c_int32),
                ("passes", C.c_int32), ("top_k", C.c_int32), ("reserved", C.c_int32),
                ("seed", C.c_uint64), ("jitter", C.c_double), ("penalty", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # LIGEN_ORACLE_LIB: a deliberately broken build of this oracle,
            # loaded by the mutation tests to show that the pins catch it.
            path = os.environ.get("LIGEN_ORACLE_LIB") or build()
            L = C.CDLL(path)
            P = C.c_void_p
            sig = {
                "or_splitmix64": (C.c_uint64, [C.c_uint64]),
                "or_uniform": (C.c_double, [C.c_uint64, C.c_int64, C.c_int64, C.c_int32]),
                "or_shoemake": (None, [P, P]),
                "or_quat_mul": (None, [P, P, P]),
                "or_quat_to_mat": (None, [P, P]),
                "or_octahedral": (None, [C.c_int32, P]),
                "or_rodrigues": (None, [P, P, P, C.c_double, P]),
                "or_validate": (C.c_int32, [P, C.c_int32]),
                "or_fragments": (C.c_int32, [P, P, P]),
                "or_atom_class": (C.c_int32, [C.c_int32]),
                "or_rot_class": (C.c_int32, [C.c_int32]),
                "or_bucket_id": (C.c_int32, [C.c_int32, C.c_int32]),
                "or_eq1_bucket_size": (C.c_int64, [C.c_int64] * 4),
                "or_trilinear": (C.c_double, [P, C.c_int32, P, P]),
                "or_trilinear_grad": (C.c_double, [P, C.c_int32, P, P, P]),
                "or_score_coords": (C.c_double, [P, P, P, C.c_double, P, P, P]),
                "or_pose_coords": (None, [P, P, P, P, P]),
                "or_score_pose": (C.c_double, [P, P, P, P, P, C.c_double, P, P, P]),
                "or_pose_grad": (C.c_double, [P, P, P, P, P, C.c_double, P]),
                "or_refine_pose": (C.c_double, [P, P, P, P, P, C.c_double, C.c_int32, C.c_double, C.c_double,
                                                C.c_double, P, P]),
                "or_torsion_angle": (C.c_double, [C.c_int32, C.c_int32]),
                "or_restart_init": (None, [P, P, C.c_int64, C.c_int64, P, P]),
                "or_dock_ligand": (C.c_int32, [P, P, P, C.c_int64, C.c_int32, C.c_int32, P, P, P, P, P, P]),
                "or_dock_exhaustive": (C.c_int32, [P, P, P, C.c_int64, C.c_int32, C.c_int32, P, P]),
                "or_top_k": (None, [C.c_int32, P, C.c_int32, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OLigand:
    """One ligand held as contiguous arrays plus its ctypes view."""

    def __init__(self, xyz, type_, bonds, rot_edge):
        self.xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        self.type = np.ascontiguousarray(type_, np.uint8)
        self.bonds = np.ascontiguousarray(bonds, np.int32).reshape(-1, 2)
        self.rot_edge = np.ascontiguousarray(rot_edge, np.int32)
        self.s = Ligand(len(self.xyz), len(self.rot_edge), _ptr(self.xyz).value,
                        _ptr(self.type).value, _ptr(self.bonds).value, _ptr(self.rot_edge).value)

    @classmethod
    def from_library(cls, lib_, l: int) -> "OLigand":
        g = lib_.ligand(l)
        return cls(g["xyz"], g["type"], g["bonds"], g["rot_edge"])

    @property
    def n_atoms(self):
        return len(self.xyz)

    @property
    def n_rot(self):
        return len(self.rot_edge)


class OGrid:
    def __init__(self, values, origin, spacing):
        self.values = np.ascontiguousarray(values, np.float64)
        nz, ny, nx, nc = self.values.shape
        self.s = GridS(nx, ny, nz, nc, (C.c_double * 3)(*origin), float(spacing), _ptr(self.values).value)

    @classmethod
    def from_grid(cls, g) -> "OGrid":
        return cls(g.values, g.origin, g.spacing)


def make_params(search: dict) -> Params:
    return Params(int(search["restarts"]), int(search.get("n_rigid", 24)),
                  int(search["torsion_step_deg"]), int(search["passes"]), int(search["top_k"]), 0,
                  int(search["seed"]) & ((1 << 64) - 1), float(search.get("jitter", 1.0)),
                  float(search.get("out_penalty", 5.0)))


# ------------------------------------------------------------- wrappers --

def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(x & ((1 << 64) - 1)))


def uniform(seed: int, lig: int, restart: int, k: int) -> float:
    return float(lib().or_uniform(seed & ((1 << 64) - 1), lig, restart, k))


def shoemake(u) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float64)
    q = np.zeros(4)
    lib().or_shoemake(_ptr(u), _ptr(q))
    return q


def quat_mul(a, b) -> np.ndarray:
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    o = np.zeros(4)
    lib().or_quat_mul(_ptr(a), _ptr(b), _ptr(o))
    return o


def quat_to_mat(q) -> np.ndarray:
    q = np.ascontiguousarray(q, np.float64)
    m = np.zeros(9)
    lib().or_quat_to_mat(_ptr(q), _ptr(m))
    return m.reshape(3, 3)


def octahedral(k: int) -> np.ndarray:
    q = np.zeros(4)
    lib().or_octahedral(k, _ptr(q))
    return q


def rodrigues(p, a, d, theta) -> np.ndarray:
    p, a, d = (np.ascontiguousarray(v, np.float64) for v in (p, a, d))
    o = np.zeros(3)
    lib().or_rodrigues(_ptr(p), _ptr(a), _ptr(d), float(theta), _ptr(o))
    return o


def validate(lig: OLigand, n_channels: int = 256) -> int:
    return int(lib().or_validate(C.byref(lig.s), n_channels))


def fragments(lig: OLigand):
    """(status, mask [n, N] bool, axis [n, 2] (u fixed, v moving))."""
    n, N = lig.n_rot, lig.n_atoms
    mask = np.zeros((max(n, 1), N), np.uint8)
    axis = np.zeros((max(n, 1), 2), np.int32)
    st = lib().or_fragments(C.byref(lig.s), _ptr(mask), _ptr(axis))
    return int(st), mask[:n].astype(bool), axis[:n]


def atom_class(n_atoms: int) -> int:
    return int(lib().or_atom_class(n_atoms))


def rot_class(n_rot: int) -> int:
    return int(lib().or_rot_class(n_rot))


def bucket_id(n_atoms: int, n_rot: int) -> int:
    return int(lib().or_bucket_id(n_atoms, n_rot))


def eq1_bucket_size(b: int, sm: int, t: int, ws: int) -> int:
    return int(lib().or_eq1_bucket_size(b, sm, t, ws))


def trilinear(grid: OGrid, c: int, x):
    """(value, inbox) of channel c at point x."""
    x = np.ascontiguousarray(x, np.float64)
    inb = C.c_int32(0)
    v = lib().or_trilinear(C.byref(grid.s), c, _ptr(x), C.byref(inb))
    return float(v), bool(inb.value)


def trilinear_grad(grid: OGrid, c: int, x):
    """(value, gradient [3] per Angstrom, inbox) of channel c at point x."""
    x = np.ascontiguousarray(x, np.float64)
    g = np.zeros(3)
    inb = C.c_int32(0)
    v = lib().or_trilinear_grad(C.byref(grid.s), c, _ptr(x), _ptr(g), C.byref(inb))
    return float(v), g, bool(inb.value)


def _frag_arrays(lig: OLigand):
    st, mask, axis = fragments(lig)
    if st:
        raise ValueError("invalid ligand")
    return (np.ascontiguousarray(mask.astype(np.uint8).reshape(-1)) if lig.n_rot else np.zeros(1, np.uint8),
            np.ascontiguousarray(axis.reshape(-1)) if lig.n_rot else np.zeros(2, np.int32))


def pose_coords(lig: OLigand, pose) -> np.ndarray:
    mask, axis = _frag_arrays(lig)
    pose = np.ascontiguousarray(pose, np.float64)
    out = np.zeros((lig.n_atoms, 3))
    lib().or_pose_coords(C.byref(lig.s), _ptr(mask), _ptr(axis), _ptr(pose), _ptr(out))
    return out


def score_coords(lig: OLigand, grid: OGrid, xyz, penalty: float = 5.0, sensitivity: bool = False):
    """(S, D, E[N]) for explicit atom positions; adds Gs when sensitivity=True."""
    xyz = np.ascontiguousarray(xyz, np.float64)
    D, G = C.c_double(0), C.c_double(0)
    E = np.zeros(lig.n_atoms)
    s = lib().or_score_coords(C.byref(lig.s), C.byref(grid.s), _ptr(xyz), penalty, C.byref(D), _ptr(E),
                              C.byref(G))
    return (float(s), float(D.value), E, float(G.value)) if sensitivity else (float(s), float(D.value), E)


def score_pose(lig: OLigand, grid: OGrid, pose, penalty: float = 5.0, sensitivity: bool = False):
    """(S, D, E[N]) of pose (t[3], q[4], theta[n]); adds Gs when sensitivity=True."""
    mask, axis = _frag_arrays(lig)
    pose = np.ascontiguousarray(pose, np.float64)
    D, G = C.c_double(0), C.c_double(0)
    E = np.zeros(lig.n_atoms)
    s = lib().or_score_pose(C.byref(lig.s), C.byref(grid.s), _ptr(mask), _ptr(axis), _ptr(pose),
                            penalty, C.byref(D), _ptr(E), C.byref(G))
    return (float(s), float(D.value), E, float(G.value)) if sensitivity else (float(s), float(D.value), E)


def pose_grad(lig: OLigand, grid: OGrid, pose, penalty: float = 5.0):
    """(S, dS/dpose [7 + n]) of pose (t[3], q[4], theta[n]) in FP64."""
    mask, axis = _frag_arrays(lig)
    pose = np.ascontiguousarray(pose, np.float64)
    g = np.zeros(7 + lig.n_rot)
    S = lib().or_pose_grad(C.byref(lig.s), C.byref(grid.s), _ptr(mask), _ptr(axis), _ptr(pose), penalty,
                           _ptr(g))
    return float(S), g


def refine_pose(lig: OLigand, grid: OGrid, pose, steps: int = 50, step_t: float = 0.1, step_q: float = 0.02,
                step_theta: float = 0.05, penalty: float = 5.0):
    """FP64 gradient refinement: (final pose, final S, accept [steps], gap [steps])."""
    mask, axis = _frag_arrays(lig)
    pose = np.array(pose, np.float64)
    acc = np.zeros(steps, np.int8)
    gap = np.zeros(steps)
    S = lib().or_refine_pose(C.byref(lig.s), C.byref(grid.s), _ptr(mask), _ptr(axis), _ptr(pose), penalty,
                             steps, step_t, step_q, step_theta, _ptr(acc), _ptr(gap))
    return pose, float(S), acc, gap


def torsion_angle(count: int, step_deg: int) -> float:
    return float(lib().or_torsion_angle(count, step_deg))


def restart_init(grid: OGrid, search: dict, lig_index: int, restart: int):
    p = make_params(search)
    q = np.zeros(4)
    t = np.zeros(3)
    lib().or_restart_init(C.byref(grid.s), C.byref(p), lig_index, restart, _ptr(q), _ptr(t))
    return q, t


def dock_ligand(lig: OLigand, grid: OGrid, search: dict, lig_index: int, restarts=None) -> dict:
    """Greedy search of one ligand over `restarts` (a range; default all)."""
    p = make_params(search)
    r0, r1 = (0, p.restarts) if restarts is None else (restarts.start, restarts.stop)
    R = r1 - r0
    n = lig.n_rot
    dlen = 1 + p.passes * n
    out = dict(score=np.zeros(R), pose=np.zeros((R, 7 + n)), trace=np.zeros((R, dlen), np.int16),
               gap=np.zeros((R, dlen)), dnorm=np.zeros((R, dlen)), gsens=np.zeros((R, dlen)))
    st = lib().or_dock_ligand(C.byref(lig.s), C.byref(grid.s), C.byref(p), lig_index, r0, r1,
                              _ptr(out["score"]), _ptr(out["pose"]), _ptr(out["trace"]),
                              _ptr(out["gap"]), _ptr(out["dnorm"]), _ptr(out["gsens"]))
    out["status"] = int(st)
    out["restarts"] = np.arange(r0, r1)
    return out


def dock_exhaustive(lig: OLigand, grid: OGrid, search: dict, lig_index: int, restarts=None) -> dict:
    p = make_params(search)
    r0, r1 = (0, p.restarts) if restarts is None else (restarts.start, restarts.stop)
    R = r1 - r0
    out = dict(score=np.zeros(R), pose=np.zeros((R, 7 + lig.n_rot)))
    st = lib().or_dock_exhaustive(C.byref(lig.s), C.byref(grid.s), C.byref(p), lig_index, r0, r1,
                                  _ptr(out["score"]), _ptr(out["pose"]))
    out["status"] = int(st)
    return out


def top_k(scores, K: int) -> np.ndarray:
    s = np.ascontiguousarray(scores, np.float64)
    out = np.zeros(K, np.int32)
    lib().or_top_k(len(s), _ptr(s), K, _ptr(out))
    return out


def dock_library(library, grid, search: dict, ligands=None, threads: int | None = None,
                 restarts=None) -> list[dict]:
    """Greedy search of the selected ligands (default all), one thread per core.

    Each result adds the ligand's top-K (`top_restart`, `top_score`,
    `top_pose`) when all restarts ran.
    """
    og = grid if isinstance(grid, OGrid) else OGrid.from_grid(grid)
    idx = list(range(library.n_ligands)) if ligands is None else [int(l) for l in ligands]
    K = int(search["top_k"])

    def one(l):
        lig = OLigand.from_library(library, l)
        r = dock_ligand(lig, og, search, l, restarts)
        r["ligand"] = l
        if restarts is None and r["status"] == 0:
            top = top_k(r["score"], K)
            r["top_restart"] = top
            r["top_score"] = r["score"][top]
            r["top_pose"] = r["pose"][top]
        return r

    n = threads or os.cpu_count() or 1
    if n == 1 or len(idx) == 1:
        return [one(l) for l in idx]
    with ThreadPoolExecutor(max_workers=n) as ex:
        return list(ex.map(one, idx))
