"""Pins of bucketing (paper §3, Eq. 1, Table 1) and of the input generators (no GPU)."""
import os

import numpy as np

import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [list(map(int, line.split())) for line in f if line.strip() and not line.startswith("#")]


def test_eq1_reproduces_table1(oracle_lib):
    # Table 1's CUDA "active blocks" are Eq. 1 bucket sizes on an A100 (108 SMs)
    # with t = ws = 32; the blocks-per-SM b must come out integral.
    for max_atoms, _regs, active, _sregs, _sactive in _rows("table1_active_blocks.txt"):
        b, rem = divmod(active, 108)
        assert rem == 0 and b in (16, 20)
        assert oracle_lib.eq1_bucket_size(b, 108, 32, 32) == active
    # t counts threads per block; two warps per block double the bucket
    assert oracle_lib.eq1_bucket_size(16, 108, 64, 32) == 3456


def test_atom_classes_follow_section3_example(oracle_lib):
    for n, cls in _rows("atom_classes.txt"):
        assert oracle_lib.atom_class(n) == cls
    assert oracle_lib.atom_class(128) == 2 and oracle_lib.atom_class(129) == 3


def test_rotamer_classes_uneven_and_finer_at_low_counts(oracle_lib):
    cls = [oracle_lib.rot_class(n) for n in range(0, 40)]
    assert cls[0] == 0 and all(b >= a for a, b in zip(cls, cls[1:]))
    widths = np.bincount(cls[:33])
    assert widths[0] == 1 and all(b >= a for a, b in zip(widths, widths[1:]))
    assert oracle_lib.bucket_id(33, 5) == 1 * 11 + 5


def test_library_is_deterministic_and_in_range():
    w = gen.WORKLOADS["small32"]
    a, b = gen.make_library(w["library"]), gen.make_library(w["library"])
    for f in ("atom_off", "xyz", "type", "bonds", "rot_off", "rot_edge"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert a.n_ligands == 32
    assert a.n_atoms.min() >= 12 and a.n_atoms.max() <= 24
    assert a.n_rot.min() >= 1 and a.n_rot.max() <= 3
    assert a.type.max() < 4


def test_library_geometry_and_rotatable_edges(oracle_lib, screen_sample):
    _, lib, _ = screen_sample
    assert lib.n_atoms.min() >= 8 and lib.n_atoms.max() <= 100 and lib.n_rot.max() <= 24
    for l in range(lib.n_ligands):
        g = lib.ligand(l)
        lig = oracle_lib.OLigand(g["xyz"], g["type"], g["bonds"], g["rot_edge"])
        assert oracle_lib.validate(lig, 8) == 0
        x, b = g["xyz"], g["bonds"]
        np.testing.assert_allclose(np.linalg.norm(x[b[:, 0]] - x[b[:, 1]], axis=1), 1.5, atol=1e-12)
        deg = np.bincount(b.ravel(), minlength=len(x))
        assert deg.max() <= 4
        e = g["rot_edge"]
        assert np.all(deg[b[e, 0]] >= 2) and np.all(deg[b[e, 1]] >= 2)
        assert len(np.unique(e)) == len(e)


def test_chunked_generation_is_prefix_stable():
    w = gen.scaled("screen20k", 5000)
    big = gen.make_library(w["library"])
    small = gen.make_library(gen.scaled("screen20k", 4096)["library"])
    assert np.array_equal(big.atom_off[:4097], small.atom_off)
    assert np.array_equal(big.xyz[:small.xyz.shape[0]], small.xyz)


def test_grid_nodes_match_direct_sum():
    w = gen.WORKLOADS["small32"]
    g = gen.make_grid(w["grid"])
    rng = np.random.default_rng(0)
    nx, ny, nz, nc = g.dims
    for _ in range(100):
        i, j, k = rng.integers(0, nx), rng.integers(0, ny), rng.integers(0, nz)
        p = np.asarray(g.origin) + g.spacing * np.array([i, j, k])
        d2 = [float(((p - c) ** 2).sum()) for c in g.centers]
        ref = [sum(wt[c] * np.exp(-d / (2 * 1.2 ** 2)) for wt, d in zip(g.weights, d2)) for c in range(nc)]
        if min(d2) < 2.5 ** 2:
            ref = [5.0] * nc
        np.testing.assert_allclose(g.values[k, j, i], ref, rtol=1e-12, atol=1e-14)
    r = np.linalg.norm(g.centers - g.center, axis=1)
    assert r.min() >= 7 and r.max() <= 11
