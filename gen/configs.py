"""Named synthetic workloads: library recipe, grid recipe and search settings.

Each workload stands in for a dataset the paper used but does not ship (its
three test ligands and a ten-million-ligand library of 20-120 atoms and 0-20
rotamers, docked into a protein's sites, §5). The shapes follow those
workloads; the molecules and grids are synthetic and seeded.
"""
from __future__ import annotations

SEARCH_DEFAULTS = dict(n_rigid=24, jitter=1.0, out_penalty=5.0)

WORKLOADS = {
    # 32 ligands of 12-24 atoms with 1-3 rotatable bonds; 40^3 x 4 grid at 0.5 A.
    "small32": dict(
        library=dict(kind="uniform", n_ligands=32, n_atoms=(12, 24), n_rot=(1, 3),
                     n_types=4, seed=0),
        grid=dict(points=40, channels=4, spacing=0.5, n_pseudo=150, seed=0),
        search=dict(SEARCH_DEFAULTS, restarts=8, torsion_step_deg=30, passes=2, top_k=4, seed=0),
    ),
    # 20,000 ligands, atoms ~ round(N(38, 14)) in [8, 100], rotatable bonds
    # ~ Poisson(6) in [0, 24]; 96^3 x 8 grid at 0.375 A from 600 pseudo-atoms.
    "screen20k": dict(
        library=dict(kind="normal", n_ligands=20000, atoms_mu_sd=(38, 14), atoms_clip=(8, 100),
                     rot_poisson=6, rot_clip=(0, 24), n_types=8, seed=1),
        grid=dict(points=96, channels=8, spacing=0.375, n_pseudo=600, seed=1),
        search=dict(SEARCH_DEFAULTS, restarts=256, torsion_step_deg=10, passes=3, top_k=30, seed=1),
    ),
    # 200,000 ligands, bimodal: 70% with 15-35 atoms and 0-8 rotatable bonds,
    # 30% with 60-120 atoms and 8-30; grid and search as screen20k.
    "bimodal200k": dict(
        library=dict(kind="bimodal", n_ligands=200000, small_frac=0.7,
                     small_atoms=(15, 35), small_rot=(0, 8),
                     large_atoms=(60, 120), large_rot=(8, 30), n_types=8, seed=2),
        grid=dict(points=96, channels=8, spacing=0.375, n_pseudo=600, seed=1),
        search=dict(SEARCH_DEFAULTS, restarts=256, torsion_step_deg=10, passes=3, top_k=30, seed=2),
    ),
}


def scaled(name: str, n_ligands: int) -> dict:
    """The named workload with its library cut to `n_ligands` (same recipe)."""
    import copy
    w = copy.deepcopy(WORKLOADS[name])
    w["library"]["n_ligands"] = int(n_ligands)
    return w


def site_grids(grid_spec: dict, n_sites: int) -> list:
    """Grid recipes of n_sites docking sites of one synthetic target (§5
    docks into twelve sites of one protein): site g keeps the channels,
    points and spacing of `grid_spec`, takes seed 1000 * seed + g, and sits
    at origin (30 g, -7 g, 11 g) Angstrom (sites are distinct boxes of one
    frame). Site 0 is `grid_spec` with its own seed and origin."""
    import copy
    out = []
    for g in range(int(n_sites)):
        s = copy.deepcopy(grid_spec)
        if g:
            s["seed"] = 1000 * int(grid_spec["seed"]) + g
            s["origin"] = (30.0 * g, -7.0 * g, 11.0 * g)
        out.append(s)
    return out
