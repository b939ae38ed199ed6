"""The C ABI library loads, exports every declared symbol and rejects bad
arguments on the host before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_2303_06150_gb300 import build
    build.build()
    from paper_2303_06150_gb300 import _abi
    return _abi


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(ligen_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(abi):
    lib = abi.load()
    declared = _declared()
    assert {"ligen_dock_batch", "ligen_score_poses", "ligen_last_error"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(abi.SIGNATURES) == declared
    assert lib.ligen_abi_version() == 5


def _lig_struct(abi, arrays):
    return abi.LigandsT(arrays["L"], 0, arrays["atom_off"].ctypes.data, arrays["rot_off"].ctypes.data,
                        arrays["atom_off"].ctypes.data, arrays["xyz"].ctypes.data, arrays["type"].ctypes.data,
                        arrays["bonds"].ctypes.data, arrays["rot_off"].ctypes.data,
                        arrays["rot_edge"].ctypes.data)


def _arrays(N=4, n=1):
    return dict(L=1, atom_off=np.array([0, N], np.int32), rot_off=np.array([0, n], np.int32),
                xyz=np.zeros((N, 3), np.float32), type=np.zeros(N, np.uint8),
                bonds=np.array([[i, i + 1] for i in range(N - 1)], np.int32).reshape(-1, 2),
                rot_edge=np.zeros(max(n, 1), np.int32))


def _grid(abi, values):
    nz, ny, nx, nc = values.shape
    return abi.GridT(nx, ny, nz, nc, (C.c_float * 3)(0, 0, 0), 0.5, 0, 0, values.ctypes.data)


def _params(abi, **kw):
    d = dict(restarts=8, n_rigid=24, torsion_step_deg=30, passes=2, top_k=4, mode=0, seed=0, jitter=1.0,
             out_penalty=5.0, stream=None, status=None, trace=None, top_restart=None, stage_ms=None)
    d.update(kw)
    return abi.ParamsT(**d)


@pytest.mark.parametrize("bad, code", [
    (dict(torsion_step_deg=7), -1), (dict(torsion_step_deg=1), -1), (dict(top_k=9), -1),
    (dict(restarts=0), -1), (dict(n_rigid=25), -1), (dict(passes=-1), -1), (dict(mode=2), -1), (dict(mode=1, trace=C.c_void_p(8)), -1),
    (dict(jitter=float("nan")), -1), (dict(batching=4), -1), (dict(grid_format=3), -1),
    (dict(mode=1, coords=C.c_void_p(8)), -1),
    (dict(rescore_fp64=2), -1),
])
def test_bad_params_rejected_on_host(abi, bad, code):
    lib = abi.load()
    a = _arrays()
    vals = np.zeros((4, 4, 4, 2), np.float32)
    out = np.zeros(64, np.float32)
    rc = lib.ligen_dock_batch(C.byref(_lig_struct(abi, a)), C.byref(_grid(abi, vals)),
                              C.byref(_params(abi, **bad)), out.ctypes.data, out.ctypes.data)
    assert rc == code
    assert lib.ligen_last_error()


@pytest.mark.parametrize("case, code", [("too_many_atoms", -2), ("too_many_rot", -2), ("empty_ligand", -1),
                                        ("grid_1pt", -1), ("grid_channels", -2), ("null_out", -1)])
def test_bad_shapes_rejected_on_host(abi, case, code):
    lib = abi.load()
    a = _arrays(300, 1) if case == "too_many_atoms" else _arrays(40, 33) if case == "too_many_rot" else _arrays()
    if case == "empty_ligand":
        a["atom_off"] = np.array([0, 0], np.int32)
    vals = np.zeros((4, 4, 4, 2), np.float32)
    if case == "grid_1pt":
        vals = np.zeros((1, 4, 4, 2), np.float32)
    if case == "grid_channels":
        vals = np.zeros((2, 2, 2, 65), np.float32)
    out = np.zeros(64, np.float32)
    outp = None if case == "null_out" else out.ctypes.data
    rc = lib.ligen_dock_batch(C.byref(_lig_struct(abi, a)), C.byref(_grid(abi, vals)), C.byref(_params(abi)),
                              outp, outp)
    assert rc == code, abi.load().ligen_last_error()


def test_empty_library_needs_no_outputs(abi):
    lib = abi.load()
    a = _arrays()
    a["L"] = 0
    vals = np.zeros((4, 4, 4, 2), np.float32)
    rc = lib.ligen_dock_batch(C.byref(_lig_struct(abi, a)), C.byref(_grid(abi, vals)), C.byref(_params(abi)),
                              None, None)
    assert rc == 0


@pytest.mark.parametrize("case", ["no_sites", "null_grids", "mixed_channels"])
def test_bad_sites_rejected_on_host(abi, case):
    lib = abi.load()
    a = _arrays()
    vals = [np.zeros((4, 4, 4, 2), np.float32),
            np.zeros((4, 4, 4, 3 if case == "mixed_channels" else 2), np.float32)]
    g2 = (abi.GridT * 2)(*[_grid(abi, v) for v in vals])
    n = 0 if case == "no_sites" else 2
    out = np.zeros(64, np.float32)
    rc = lib.ligen_dock_sites(C.byref(_lig_struct(abi, a)), None if case == "null_grids" else g2, n,
                              C.byref(_params(abi)), out.ctypes.data, out.ctypes.data)
    assert rc == -1 and lib.ligen_last_error()


def test_null_structs_rejected(abi):
    lib = abi.load()
    assert lib.ligen_dock_batch(None, None, None, None, None) == -1
    assert lib.ligen_score_poses(None, None, 1, None, 5.0, None, None) == -1
    assert lib.ligen_pack_ligands(None, 4, None, None, None, None, None) == -1
    assert lib.ligen_bucket_size(0, None, None, None, None) == -1
    assert lib.ligen_tune_set(44, 8, 16) == -1 and lib.ligen_tune_set(0, 3, 16) == -1
    assert lib.ligen_tune_set(0, 8, 10) == -1 and lib.ligen_tune_set(0, 4, 64) == -1
    assert lib.ligen_autotune(None, None, None, 1, None, None, None) == -1
    assert lib.ligen_probe_stream(None, 16, 1, None, None, None, None) == -1
    assert lib.ligen_set_workspace_limit(1 << 20) == 0 and lib.ligen_set_workspace_limit(0) == 0
    h = C.c_void_p()
    assert lib.ligen_prepare_scoring(None, None, None, None) == -1           # no output handle
    assert lib.ligen_prepare_scoring(None, None, None, C.byref(h)) == -1 and h.value is None
    assert lib.ligen_score_prepared(None, 30, None, 5.0, None, None) == -1
    assert lib.ligen_release_prepared(None) == 0
    # shapes beyond 128 threads, off the warp's restart multiple or of an unsupported width
    assert lib.ligen_tune_set(0, 32, 8) == -1 and lib.ligen_tune_set(0, 16, 9) == -1
    assert lib.ligen_tune_set(0, 64, 2) == -1


def test_package_refuses_to_load_without_library(tmp_path):
    from paper_2303_06150_gb300 import _abi
    with pytest.raises(ImportError):
        _abi._lib, saved = None, _abi._lib
        try:
            _abi.load(str(tmp_path / "missing.so"))
        finally:
            _abi._lib = saved
