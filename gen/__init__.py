"""Seeded synthetic inputs shared by the CUDA path and the oracle.

Holds input generation only: ligand trees, pocket grids and the named
workloads. Nothing here computes a fragment, a pose or a score.
"""
from .configs import WORKLOADS, scaled, site_grids
from .grid import Grid, make_grid
from .library import Library, from_ligands, make_library, shuffle_bonds

__all__ = ["WORKLOADS", "scaled", "site_grids", "Grid", "make_grid", "Library", "from_ligands",
           "make_library", "shuffle_bonds"]
