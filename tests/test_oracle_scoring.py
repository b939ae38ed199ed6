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
    import oracle
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
    # the value-and-gradient sampler (the one the score uses) has the same box:
    # nodes on the upper faces are inside and take their node value
    vg, _, inb = oracle_lib.trilinear_grad(g, 1, top)
    assert inb and abs(vg - grid.values[-1, -1, -1, 1]) < 1e-13
    for d in ([1e-9, 0, 0], [0, 1e-9, 0], [0, 0, 1e-9]):
        assert not oracle_lib.trilinear_grad(g, 1, top + np.array(d))[2]
    one = oracle.OLigand(np.zeros((1, 3)), [1], np.zeros((0, 2)), [])
    S, _, E = oracle_lib.score_coords(one, g, top[None, :], 5.0)
    assert S == -E[0] and abs(E[0] - grid.values[-1, -1, -1, 1]) < 1e-13
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


def test_trilinear_gradient_pins(oracle_lib, small32):
    # exact on linear fields, and the central difference elsewhere (away from faces)
    rng = np.random.default_rng(5)
    vals = np.zeros((6, 6, 6, 1))
    zz, yy, xx = np.meshgrid(*(0.5 * np.arange(6),) * 3, indexing="ij")
    b = np.array([0.3, -1.7, 2.2])
    vals[..., 0] = 1.0 + b[0] * xx + b[1] * yy + b[2] * zz
    g = _grid(vals, (0.0, 0.0, 0.0), 0.5)
    for _ in range(50):
        v, gr, inb = oracle_lib.trilinear_grad(g, 0, rng.uniform(0, 2.5, 3))
        assert inb
        np.testing.assert_allclose(gr, b, atol=1e-12)
    _, _, grid = small32
    g = _grid(grid.values, grid.origin, grid.spacing)
    h = 1e-6
    for _ in range(300):
        cell = rng.integers(2, 35, 3)
        p = grid.spacing * (cell + rng.uniform(0.05, 0.95, 3))
        c = int(rng.integers(0, 4))
        v, gr, inb = oracle_lib.trilinear_grad(g, c, p)
        assert inb and v == oracle_lib.trilinear(g, c, p)[0]
        fd = [(oracle_lib.trilinear(g, c, p + h * e)[0] - oracle_lib.trilinear(g, c, p - h * e)[0]) / (2 * h)
              for e in np.eye(3)]
        np.testing.assert_allclose(gr, fd, atol=1e-6 * (1 + np.abs(gr).max()))


def test_position_sensitivity_bounds_relative_coordinate_noise(oracle_lib, small32):
    import oracle
    _, lib, grid = small32
    og = oracle.OGrid.from_grid(grid)
    rng = np.random.default_rng(6)
    for l in range(0, 32, 4):
        lig = oracle.OLigand.from_library(lib, l)
        pose = np.concatenate([grid.center + rng.uniform(-3, 3, 3), rng.normal(size=4),
                               rng.uniform(-np.pi, np.pi, lig.n_rot)])
        x = oracle_lib.pose_coords(lig, pose)
        S, D, E, Gs = oracle_lib.score_coords(lig, og, x, 5.0, sensitivity=True)
        eps = 1e-7
        for _ in range(20):
            noisy = x * (1 + eps * rng.uniform(-1, 1, x.shape))   # origin is (0, 0, 0) here
            S2 = oracle_lib.score_coords(lig, og, noisy, 5.0)[0]
            assert abs(S2 - S) <= 1.01 * eps * Gs + 1e-12


def _face_safe(lig, og, oracle_lib, pose, a, h, spacing, origin, dims):
    """True when moving parameter a by +-h keeps every atom inside one cell
    and on the same side of the box boundary (no kink in the interval)."""
    cells = []
    for sgn in (-1, 1):
        p = pose.copy()
        p[a] += sgn * h
        u = (oracle_lib.pose_coords(lig, p) - np.asarray(origin)) / spacing
        inside = np.all((u >= 0) & (u <= np.asarray(dims) - 1), axis=1)
        cells.append((np.floor(u).astype(int), inside))
    return np.array_equal(cells[0][0], cells[1][0]) and np.array_equal(cells[0][1], cells[1][1])


def test_pose_gradient_matches_central_differences(oracle_lib, small32, screen_sample):
    import oracle
    rng = np.random.default_rng(12)
    h = 1e-4
    checked = 0
    for _, lib, grid in (small32, screen_sample):
        og = oracle.OGrid.from_grid(grid)
        nx, ny, nz, _ = grid.dims
        for l in range(0, lib.n_ligands, 2):
            lig = oracle.OLigand.from_library(lib, l)
            pose = np.concatenate([grid.center + rng.uniform(-2, 2, 3), rng.normal(size=4),
                                   rng.uniform(-np.pi, np.pi, lig.n_rot)])
            S, g = oracle_lib.pose_grad(lig, og, pose)
            assert abs(S - oracle_lib.score_pose(lig, og, pose)[0]) <= 1e-12 * max(1, abs(S))
            for a in range(7 + lig.n_rot):
                if not _face_safe(lig, og, oracle_lib, pose, a, h, grid.spacing, grid.origin, (nx, ny, nz)):
                    continue
                p1, p0 = pose.copy(), pose.copy()
                p1[a] += h
                p0[a] -= h
                fd = (oracle_lib.score_pose(lig, og, p1)[0] - oracle_lib.score_pose(lig, og, p0)[0]) / (2 * h)
                assert abs(fd - g[a]) <= 1e-5 * (1 + np.abs(g).max()), (l, a, fd, g[a])
                checked += 1
    assert checked > 300


def test_pose_gradient_invariances(oracle_lib, small32):
    # scaling q leaves the pose unchanged: dS/dq is orthogonal to q; a pure
    # translation field E = a + b.x gives dS/dt = -N_in * b
    import oracle
    _, lib, grid = small32
    og = oracle.OGrid.from_grid(grid)
    rng = np.random.default_rng(13)
    for l in range(8):
        lig = oracle.OLigand.from_library(lib, l)
        pose = np.concatenate([grid.center, rng.normal(size=4), rng.uniform(-np.pi, np.pi, lig.n_rot)])
        _, g = oracle_lib.pose_grad(lig, og, pose)
        assert abs(g[3:7] @ pose[3:7]) <= 1e-10 * (1 + np.abs(g).max())
    nz, ny, nx, nc = 30, 30, 30, 4
    zz, yy, xx = np.meshgrid(*(0.5 * np.arange(30),) * 3, indexing="ij")
    b = np.array([0.2, -0.4, 0.7])
    vals = np.repeat((1.0 + b[0] * xx + b[1] * yy + b[2] * zz)[..., None], nc, axis=3)
    lin = oracle.OGrid(vals, (0.0, 0.0, 0.0), 0.5)
    lig = oracle.OLigand.from_library(lib, 0)
    pose = np.concatenate([[7.2, 7.3, 7.4], rng.normal(size=4), rng.uniform(-np.pi, np.pi, lig.n_rot)])
    _, g = oracle_lib.pose_grad(lig, lin, pose)
    np.testing.assert_allclose(g[:3], -lig.n_atoms * b, atol=1e-10)
    # and then rotations and torsions cannot change a linear field's sum
    # except through the atom positions' moment: compare with differences
    h = 1e-5
    for a in range(3, 7 + lig.n_rot):
        p1, p0 = pose.copy(), pose.copy()
        p1[a] += h
        p0[a] -= h
        fd = (oracle_lib.score_pose(lig, lin, p1)[0] - oracle_lib.score_pose(lig, lin, p0)[0]) / (2 * h)
        assert abs(fd - g[a]) <= 1e-7 * (1 + abs(g[a]))
