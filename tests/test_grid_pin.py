"""Pins of the synthetic pocket grid against its recipe (no GPU).

The generator (gen/grid.py) builds node values with a factorised matrix
product; these tests recompute them from the pseudo-atom list one node at a
time with code of their own, and check the pseudo-atom list against the
recipe's distributions:

* pseudo-atoms lie on a 7-11 A shell around the grid centre, uniform in
  shell volume (r^3 uniform) and in direction;
* weights are N(-1, 0.3), one per (pseudo-atom, channel);
* node value V_c = sum_p w_pc exp(-d^2 / (2 * 1.2^2)), overwritten with +5 in
  every channel where some pseudo-atom is nearer than 2.5 A;
* the oracle's trilinear sample at a node is that value (the benchmark spec's
  "trilinear sampling reproduces the analytic sum-of-Gaussians at nodes").

A mutant generator (sigma, shell, weights, plateau radius or value changed
one at a time) must fail these checks.
"""
import math

import numpy as np
import pytest
from scipy import stats

import gen
import gen.grid as gg

SIGMA = 1.2
SHELL = (7.0, 11.0)
PLATEAU_R = 2.5
PLATEAU_V = 5.0
W_MU, W_SD = -1.0, 0.3


def _centre(grid):
    nx, ny, nz, _ = grid.dims
    return np.array(grid.origin) + grid.spacing * (np.array([nx, ny, nz]) - 1) / 2.0


def shell_ok(grid) -> bool:
    d = grid.centers - _centre(grid)
    r = np.sqrt((d * d).sum(1))
    if r.min() < SHELL[0] - 1e-9 or r.max() > SHELL[1] + 1e-9:
        return False
    # r^3 uniform on [r0^3, r1^3]; direction uniform: z/r uniform on [-1, 1]
    # and the azimuth uniform on [0, 2 pi)
    p_r = stats.kstest((r ** 3 - SHELL[0] ** 3) / (SHELL[1] ** 3 - SHELL[0] ** 3), "uniform").pvalue
    p_z = stats.kstest((d[:, 2] / r + 1.0) / 2.0, "uniform").pvalue
    p_phi = stats.kstest((np.arctan2(d[:, 1], d[:, 0]) % (2 * np.pi)) / (2 * np.pi), "uniform").pvalue
    return min(p_r, p_z, p_phi) > 1e-4


def weights_ok(grid) -> bool:
    w = np.asarray(grid.weights).ravel()
    n = w.size
    # mean within 5 standard errors, sd within 5 standard errors of its estimate
    if abs(w.mean() - W_MU) > 5 * W_SD / math.sqrt(n):
        return False
    if abs(w.std(ddof=1) - W_SD) > 5 * W_SD / math.sqrt(2 * (n - 1)):
        return False
    return stats.kstest((w - W_MU) / W_SD, "norm").pvalue > 1e-4


def node_value(grid, i, j, k, c) -> float:
    """V_c at node (i, j, k), one pseudo-atom at a time."""
    x = np.array(grid.origin, dtype=np.float64) + grid.spacing * np.array([i, j, k], dtype=np.float64)
    total = 0.0
    nearest = math.inf
    for p in range(len(grid.centers)):
        dx, dy, dz = (float(x[a] - grid.centers[p][a]) for a in range(3))
        d2 = dx * dx + dy * dy + dz * dz
        nearest = min(nearest, math.sqrt(d2))
        total += float(grid.weights[p][c]) * math.exp(-d2 / (2.0 * SIGMA * SIGMA))
    return PLATEAU_V if nearest < PLATEAU_R else total


def sample_nodes(grid, rng, n_random=150, n_near=150):
    """Random nodes plus nodes close to pseudo-atoms (inside, at and beyond
    the plateau radius), so both rules are exercised."""
    nx, ny, nz, nc = grid.dims
    out = [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz)), int(rng.integers(nc)))
           for _ in range(n_random)]
    h = grid.spacing
    for _ in range(n_near):
        p = grid.centers[int(rng.integers(len(grid.centers)))]
        q = p + rng.normal(size=3) * (PLATEAU_R * rng.uniform(0.5, 1.5) / math.sqrt(3))
        ijk = np.rint((q - np.array(grid.origin)) / h).astype(int)
        if np.all(ijk >= 0) and np.all(ijk < np.array([nx, ny, nz])):
            out.append((int(ijk[0]), int(ijk[1]), int(ijk[2]), int(rng.integers(nc))))
    return out


def nodes_ok(grid, nodes) -> bool:
    for i, j, k, c in nodes:
        ref = node_value(grid, i, j, k, c)
        if abs(grid.values[k, j, i, c] - ref) > 1e-12 * max(1.0, abs(ref)):
            return False
    return True


GRIDS = {
    "small32": gen.WORKLOADS["small32"]["grid"],
    "screen_grid": dict(gen.WORKLOADS["screen20k"]["grid"], points=64),   # 600 pseudo-atoms, 0.375 A
}


@pytest.mark.parametrize("name", list(GRIDS))
def test_pseudo_atoms_follow_the_recipe(name):
    grid = gen.make_grid(GRIDS[name])
    assert len(grid.centers) == GRIDS[name]["n_pseudo"]
    assert np.asarray(grid.weights).shape == (GRIDS[name]["n_pseudo"], GRIDS[name]["channels"])
    assert shell_ok(grid)
    assert weights_ok(grid)


@pytest.mark.parametrize("name", list(GRIDS))
def test_node_values_are_the_sum_of_gaussians_or_the_plateau(name):
    grid = gen.make_grid(GRIDS[name])
    rng = np.random.default_rng(5)
    nodes = sample_nodes(grid, rng)
    plateau = sum(node_value(grid, *n) == PLATEAU_V for n in nodes)
    assert 20 <= plateau <= len(nodes) - 20, plateau      # both rules exercised
    assert nodes_ok(grid, nodes)


def test_trilinear_at_nodes_reproduces_the_analytic_values(oracle_lib):
    grid = gen.make_grid(GRIDS["small32"])
    og = oracle_lib.OGrid.from_grid(grid)
    rng = np.random.default_rng(6)
    for i, j, k, c in sample_nodes(grid, rng, 100, 100):
        p = np.array(grid.origin) + grid.spacing * np.array([i, j, k])
        v, inb = oracle_lib.trilinear(og, c, p)
        assert inb
        ref = node_value(grid, i, j, k, c)
        assert abs(v - ref) <= 1e-12 * max(1.0, abs(ref)), (i, j, k, c, v, ref)


@pytest.mark.parametrize("attr,value,check", [
    ("SIGMA_A", 1.0, "nodes"),
    ("SIGMA_A", 1.3, "nodes"),
    ("CLASH_A", 2.0, "nodes"),
    ("CLASH_A", 3.0, "nodes"),
    ("CLASH_VALUE", 4.0, "nodes"),
    ("SHELL_A", (6.0, 11.0), "shell"),
    ("SHELL_A", (7.0, 12.0), "shell"),
    ("W_MU_SD", (-0.9, 0.3), "weights"),
    ("W_MU_SD", (-1.0, 0.4), "weights"),
])
def test_mutant_generators_fail_the_pins(monkeypatch, attr, value, check):
    monkeypatch.setattr(gg, attr, value)
    grid = gg.make_grid(GRIDS["small32"])
    rng = np.random.default_rng(5)
    ok = {"nodes": lambda: nodes_ok(grid, sample_nodes(grid, rng)),
          "shell": lambda: shell_ok(grid),
          "weights": lambda: weights_ok(grid)}[check]()
    assert not ok, (attr, value)
