"""Seeded synthetic pocket grids.

Input generation only. A pocket grid holds, at every node of a regular
lattice, one energy value per atom type (channel). The docking method reads
these values; it never builds them.

Recipe (shape of a pocket: attractive walls around an empty site):

* n_pseudo pseudo-atoms are placed around the grid centre
  g_c = origin + spacing * (G - 1) / 2 at radius r = cbrt(U[r0^3, r1^3])
  (uniform in shell volume, r0 = 7 A, r1 = 11 A) in a uniform direction;
* each pseudo-atom p has one weight per channel, w[p, c] ~ N(-1, 0.3);
* node value V_c(x) = sum_p w[p, c] exp(-|x - x_p|^2 / (2 * 1.2^2));
* where the nearest pseudo-atom is closer than 2.5 A, every channel is
  overwritten with +5 (a clash plateau).

Layout: values[z, y, x, c] (channel innermost), float64. The generator uses
its own stream, `numpy.random.default_rng([seed, 1])`.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SIGMA_A = 1.2
SHELL_A = (7.0, 11.0)
CLASH_A = 2.5
CLASH_VALUE = 5.0
W_MU_SD = (-1.0, 0.3)


@dataclass
class Grid:
    values: np.ndarray          # float64 [nz, ny, nx, nc]
    origin: tuple               # (x, y, z) Angstrom of node (0, 0, 0)
    spacing: float              # Angstrom between nodes, all axes
    centers: np.ndarray         # [P, 3] pseudo-atom positions
    weights: np.ndarray         # [P, nc]

    @property
    def dims(self):
        nz, ny, nx, nc = self.values.shape
        return nx, ny, nz, nc

    @property
    def center(self) -> np.ndarray:
        nx, ny, nz, _ = self.dims
        return np.asarray(self.origin) + self.spacing * (np.array([nx, ny, nz]) - 1) / 2.0


def node_positions(dims, origin, spacing, z: int) -> np.ndarray:
    nx, ny = dims[0], dims[1]
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([xx, yy, np.full_like(xx, z)], -1).reshape(-1, 3).astype(np.float64)
    return np.asarray(origin, np.float64) + spacing * pts


def make_grid(spec: dict) -> Grid:
    G = int(spec["points"])
    nc = int(spec["channels"])
    h = float(spec["spacing"])
    origin = tuple(float(v) for v in spec.get("origin", (0.0, 0.0, 0.0)))
    rng = np.random.default_rng([int(spec["seed"]), 1])
    P = int(spec["n_pseudo"])
    r0, r1 = SHELL_A
    r = np.cbrt(rng.uniform(r0 ** 3, r1 ** 3, P))
    z = rng.uniform(-1.0, 1.0, P)
    phi = rng.uniform(0.0, 2.0 * np.pi, P)
    s = np.sqrt(1.0 - z * z)
    dirs = np.stack([s * np.cos(phi), s * np.sin(phi), z], 1)
    center = np.asarray(origin) + h * (G - 1) / 2.0
    centers = center + r[:, None] * dirs
    weights = rng.normal(W_MU_SD[0], W_MU_SD[1], (P, nc))

    # The Gaussian factorises over axes, so each z-slab is one matrix product:
    # V[z, y, (x, c)] = sum_p Ez[p, z] Ey[p, y] * (Ex[p, x] w[p, c]).
    inv2s2 = 1.0 / (2.0 * SIGMA_A * SIGMA_A)
    axis = np.asarray(origin)[None, :] + h * np.arange(G)[:, None]      # [G, 3]
    E = np.exp(-((axis[None, :, :] - centers[:, None, :]) ** 2) * inv2s2)  # [P, G, 3]
    B = (E[:, :, 0, None] * weights[:, None, :]).reshape(P, G * nc)
    values = np.empty((G, G, G, nc))
    for zi in range(G):
        A = E[:, zi, 2, None] * E[:, :, 1]                                # [P, G(y)]
        values[zi] = (A.T @ B).reshape(G, G, nc)
    # Clash plateau: every node within CLASH_A of some pseudo-atom.
    reach = int(np.ceil(CLASH_A / h)) + 1
    for c in centers:
        lo = np.maximum(np.floor((c - np.asarray(origin)) / h).astype(int) - reach, 0)
        hi = np.minimum(lo + 2 * reach + 2, G)
        xs, ys, zs = (np.asarray(origin)[k] + h * np.arange(lo[k], hi[k]) for k in range(3))
        d2 = ((zs[:, None, None] - c[2]) ** 2 + (ys[None, :, None] - c[1]) ** 2
              + (xs[None, None, :] - c[0]) ** 2)
        sub = values[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[d2 < CLASH_A ** 2] = CLASH_VALUE
    return Grid(values=values, origin=origin, spacing=h, centers=centers, weights=weights)
