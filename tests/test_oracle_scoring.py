"""Pins of the oracle's grid sampling and pose scores (no GPU)."""
import numpy as np

import indep


def _grid(values, origin=(0.0, 0.0, 0.0), spacing=0.5):
    import oracle
    return oracle.OGrid(values, origin, spacing)


def test_trilinear_exact_on_linear_fields(oracle_lib):
    rng = np.random.default_rng(1)
    nz, ny, nx, nc = 7, 9, 11, 3
    origin, h = (-1.0, 2.0, 0.5), 0.4
    coef = rng.normal(size=(nc, 4))
    zz, yy, xx = np.meshgrid(*(origin[2 - a] + h * np.arange(n) for a, n in enumerate((nz, ny, nx))),
                             indexing="ij")
    vals = np.stack([c[0] + c[1] * xx + c[2] * yy + c[3] * zz for c in coef], -1)
    g = _grid(vals, origin, h)
    lo = np.array(origin)
    hi = lo + h * (np.array([nx, ny, nz]) - 1)
    for _ in range(500):
        p = rng.uniform(lo, hi)
        c = rng.integers(nc)
        v, inb = oracle_lib.trilinear(g, c, p)
        assert inb
        ref = coef[c, 0] + coef[c, 1:] @ p
        assert abs(v - ref) <= 1e-12 * max(1.0, abs(ref))


def test_trilinear_matches_scipy_and_nodes(oracle_lib, small32):
    _, _, grid = small32
    g = _grid(grid.values, grid.origin, grid.spacing)
    samp = indep.trilinear_sampler(grid.values, grid.origin, grid.spacing)
    rng = np.random.default_rng(2)
    nx, ny, nz, nc = grid.dims
    pts = rng.uniform(-1, grid.spacing * nx + 1, (400, 3))
    for c in range(nc):
        ref, rin = samp(c, pts)
        for p, r, ri in zip(pts, ref, rin):
            v, inb = oracle_lib.trilinear(g, c, p)
            assert inb == ri
            if inb:
                assert abs(v - r) < 1e-12
    # at grid nodes the sample is the node value (the analytic sum of Gaussians,
    # or the clash plateau)
    for _ in range(200):
        i, j, k, c = rng.integers(0, nx), rng.integers(0, ny), rng.integers(0, nz), rng.integers(0, nc)
        p = np.asarray(grid.origin) + grid.spacing * np.array([i, j, k])
        v, inb = oracle_lib.trilinear(g, c, p)
        assert inb and abs(v - grid.values[k, j, i, c]) < 1e-13


def test_trilinear_box_edges_and_continuity(oracle_lib, small32):
    _, _, grid = small32
    g = _grid(grid.values, grid.origin, grid.spacing)
    nx, ny, nz, nc = grid.dims
    h = grid.spacing
    top = np.array([nx - 1, ny - 1, nz - 1]) * h
    v, inb = oracle_lib.trilinear(g, 1, top)
    assert inb and abs(v - grid.values[-1, -1, -1, 1]) < 1e-13
    for d in ([1e-9, 0, 0], [0, 1e-9, 0], [0, 0, 1e-9]):
        assert not oracle_lib.trilinear(g, 1, top + np.array(d))[1]
    assert not oracle_lib.trilinear(g, 0, [-1e-9, 1.0, 1.0])[1]
    assert oracle_lib.trilinear(g, 0, [0.0, 1.0, 1.0])[1]
    rng = np.random.default_rng(3)
    for _ in range(100):
        p = rng.uniform(h, top - h)
        p[rng.integers(3)] = h * rng.integers(1, 10)        # on a cell face
        for c in range(nc):
            a = oracle_lib.trilinear(g, c, p - 1e-10)[0]
            b = oracle_lib.trilinear(g, c, p + 1e-10)[0]
            assert abs(a - b) < 1e-7


def test_score_pose_matches_independent_scorer(oracle_lib, small32, screen_sample):
    import oracle
    rng = np.random.default_rng(4)
    for w, lib, grid in (small32, screen_sample):
        og = oracle.OGrid.from_grid(grid)
        samp = indep.trilinear_sampler(grid.values, grid.origin, grid.spacing)
        for l in range(0, lib.n_ligands, 4):
            lig = oracle.OLigand.from_library(lib, l)
            pose = np.concatenate([grid.center + rng.uniform(-3, 3, 3), rng.normal(size=4),
                                   rng.uniform(-np.pi, np.pi, lig.n_rot)])
            S, D, E = oracle_lib.score_pose(lig, og, pose, 5.0)
            pts = indep.pose_coords(lig.xyz, lig.bonds, lig.rot_edge, pose)
            S2, D2, E2 = indep.score_coords(samp, lig.type, pts, 5.0)
            np.testing.assert_allclose(E, E2, atol=1e-11)
            assert abs(S - S2) <= 1e-11 * D2 and abs(D - D2) <= 1e-11 * D2
            assert abs(S + E.sum()) < 1e-12 * D
            assert abs(D - max(abs(S), np.abs(E).sum())) <= 1e-14 * D


def test_out_of_box_atoms_take_the_penalty(oracle_lib, small32):
    import oracle
    _, lib, grid = small32
    og = oracle.OGrid.from_grid(grid)
    lig = oracle.OLigand.from_library(lib, 0)
    pose = np.concatenate([[1e3, 0, 0], [1, 0, 0, 0], np.zeros(lig.n_rot)])
    S, D, E = oracle_lib.score_pose(lig, og, pose, 7.5)
    assert np.all(E == 7.5) and S == -7.5 * lig.n_atoms
