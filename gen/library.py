"""Seeded synthetic ligand libraries.

Input generation only: this module draws random molecular trees and writes
them in the CSR layout that both the CUDA path and the oracle read. It holds
none of the docking method's arithmetic (no fragments, no poses, no scores).

A ligand is a tree of heavy atoms (paper §3: atoms plus *rotamers*, the
rotatable subsets of atoms). Growth rule, per ligand with N atoms:

* atom 0 sits at the origin;
* atom i (i >= 1) picks a parent p uniformly among existing atoms whose
  degree is below 4, and is placed 1.5 A from p;
* atom 1 goes in a uniform random direction; every later atom makes a
  109.5 degree angle with the bond from p to p's reference neighbour
  (p's parent, or atom 1 when p is atom 0), at a uniform random azimuth
  about that bond measured from the global z axis (x axis when the bond is
  within 8 degrees of z);
* if the new atom is closer than 1.2 A to any atom other than p, the parent
  and azimuth are redrawn, up to 100 attempts; the last attempt is kept;
* atom types are uniform over the grid's channels;
* rotatable bonds are drawn without replacement among the edges whose two
  endpoints both have degree >= 2, sorted by edge index.

Edge e of a ligand joins atom e+1 to its parent (bonds row e = [parent, e+1]).
Ligands are generated in chunks of 4096 with one `numpy.random.Generator` per
chunk seeded by (seed, 0, chunk), so the library is deterministic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

CHUNK = 4096
BOND_A = 1.5
ANGLE_DEG = 109.5
MIN_NONBONDED_A = 1.2
MAX_TRIES = 100


@dataclass
class Library:
    """A ligand library in CSR form (host, numpy).

    atom_off [L+1] int32   atom range of ligand l is atom_off[l]:atom_off[l+1]
    xyz      [sum N, 3]    float64 input conformation, Angstrom
    type     [sum N]       uint8 atom type (grid channel)
    bonds    [sum N - L, 2] int32 local atom ids; ligand l's rows start at
                           atom_off[l] - l
    rot_off  [L+1] int32   rotatable-bond range of ligand l
    rot_edge [sum n] int32 local edge (bond row) ids of the rotatable bonds
    """

    atom_off: np.ndarray
    xyz: np.ndarray
    type: np.ndarray
    bonds: np.ndarray
    rot_off: np.ndarray
    rot_edge: np.ndarray

    @property
    def n_ligands(self) -> int:
        return len(self.atom_off) - 1

    @property
    def n_atoms(self) -> np.ndarray:
        return np.diff(self.atom_off)

    @property
    def n_rot(self) -> np.ndarray:
        return np.diff(self.rot_off)

    def ligand(self, l: int) -> dict:
        a0, a1 = int(self.atom_off[l]), int(self.atom_off[l + 1])
        r0, r1 = int(self.rot_off[l]), int(self.rot_off[l + 1])
        return {
            "xyz": self.xyz[a0:a1],
            "type": self.type[a0:a1],
            "bonds": self.bonds[a0 - l:a1 - l - 1],
            "rot_edge": self.rot_edge[r0:r1],
        }

    def subset(self, idx) -> "Library":
        return from_ligands([self.ligand(int(l)) for l in idx])


def from_ligands(ligs: list[dict]) -> Library:
    """Assemble a Library from per-ligand dicts (xyz, type, bonds, rot_edge)."""
    n_atoms = [len(g["xyz"]) for g in ligs]
    n_rot = [len(g["rot_edge"]) for g in ligs]
    atom_off = np.zeros(len(ligs) + 1, np.int32)
    atom_off[1:] = np.cumsum(n_atoms)
    rot_off = np.zeros(len(ligs) + 1, np.int32)
    rot_off[1:] = np.cumsum(n_rot)

    def cat(key, shape, dtype):
        parts = [np.asarray(g[key], dtype).reshape(shape) for g in ligs]
        return np.concatenate(parts) if parts else np.zeros((0,) + shape[1:], dtype)

    return Library(
        atom_off=atom_off,
        xyz=cat("xyz", (-1, 3), np.float64),
        type=cat("type", (-1,), np.uint8),
        bonds=cat("bonds", (-1, 2), np.int32),
        rot_off=rot_off,
        rot_edge=cat("rot_edge", (-1,), np.int32),
    )


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _grow_trees(rng, n_atoms: np.ndarray):
    """Grow one tree per ligand of the chunk; returns positions, parents, degrees."""
    lc = len(n_atoms)
    nmax = int(n_atoms.max())
    pos = np.zeros((lc, nmax, 3))
    parent = np.full((lc, nmax), -1, np.int64)
    deg = np.zeros((lc, nmax), np.int64)
    ca, sa = np.cos(np.radians(ANGLE_DEG)), np.sin(np.radians(ANGLE_DEG))
    for i in range(1, nmax):
        pending = np.nonzero(n_atoms > i)[0]
        for attempt in range(MAX_TRIES):
            m = len(pending)
            if m == 0:
                break
            elig = deg[pending, :i] < 4
            cnt = elig.sum(1)
            pick = np.minimum((rng.random(m) * cnt).astype(np.int64), cnt - 1)
            p = np.argmax(np.cumsum(elig, 1) > pick[:, None], axis=1)
            if i == 1:
                z = 2.0 * rng.random(m) - 1.0
                phi = 2.0 * np.pi * rng.random(m)
                s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
                d = np.stack([s * np.cos(phi), s * np.sin(phi), z], 1)
            else:
                a = np.where(p != 0, parent[pending, p], 1)
                e = _unit(pos[pending, a] - pos[pending, p])
                ref = np.zeros_like(e)
                near_z = np.abs(e[:, 2]) > np.cos(np.radians(8.0))
                ref[~near_z, 2] = 1.0
                ref[near_z, 0] = 1.0
                n1 = _unit(ref - (ref * e).sum(1, keepdims=True) * e)
                n2 = np.cross(e, n1)
                phi = 2.0 * np.pi * rng.random(m)
                d = ca * e + sa * (np.cos(phi)[:, None] * n1 + np.sin(phi)[:, None] * n2)
            newp = pos[pending, p] + BOND_A * d
            dist2 = ((pos[pending, :i] - newp[:, None, :]) ** 2).sum(-1)
            dist2[np.arange(m), p] = np.inf
            ok = (dist2 >= MIN_NONBONDED_A ** 2).all(1) | (attempt == MAX_TRIES - 1)
            acc = pending[ok]
            pos[acc, i] = newp[ok]
            parent[acc, i] = p[ok]
            deg[acc, p[ok]] += 1
            deg[acc, i] = 1
            pending = pending[~ok]
    return pos, parent, deg


def _draw_sizes(rng, kind: str, lc: int, spec: dict):
    if kind == "uniform":
        lo, hi = spec["n_atoms"]
        rlo, rhi = spec["n_rot"]
        n_atoms = rng.integers(lo, hi + 1, lc)
        n_rot = rng.integers(rlo, rhi + 1, lc)
    elif kind == "normal":
        mu, sd = spec["atoms_mu_sd"]
        lo, hi = spec["atoms_clip"]
        n_atoms = np.clip(np.round(rng.normal(mu, sd, lc)), lo, hi).astype(np.int64)
        rlo, rhi = spec["rot_clip"]
        n_rot = np.clip(rng.poisson(spec["rot_poisson"], lc), rlo, rhi)
    elif kind == "bimodal":
        small = rng.random(lc) < spec["small_frac"]
        (sa0, sa1), (sr0, sr1) = spec["small_atoms"], spec["small_rot"]
        (la0, la1), (lr0, lr1) = spec["large_atoms"], spec["large_rot"]
        n_atoms = np.where(small, rng.integers(sa0, sa1 + 1, lc), rng.integers(la0, la1 + 1, lc))
        n_rot = np.where(small, rng.integers(sr0, sr1 + 1, lc), rng.integers(lr0, lr1 + 1, lc))
    else:
        raise ValueError(f"unknown library kind {kind!r}")
    return n_atoms.astype(np.int64), n_rot.astype(np.int64)


def _chunk(seed: int, chunk: int, lc: int, spec: dict) -> list[dict]:
    rng = np.random.default_rng([seed, 0, chunk])
    n_atoms, n_rot = _draw_sizes(rng, spec["kind"], lc, spec)
    pos, parent, deg = _grow_trees(rng, n_atoms)
    nmax = pos.shape[1]
    types = rng.integers(0, spec["n_types"], (lc, nmax))
    keys = rng.random((lc, max(nmax - 1, 1)))
    out = []
    for l in range(lc):
        n = int(n_atoms[l])
        child = np.arange(1, n)
        par = parent[l, 1:n]
        bonds = np.stack([par, child], 1).astype(np.int32)
        cand = np.nonzero((deg[l, par] >= 2) & (deg[l, child] >= 2))[0]
        k = min(int(n_rot[l]), len(cand))
        chosen = cand[np.argsort(keys[l, cand], kind="stable")[:k]] if k else cand[:0]
        out.append({
            "xyz": pos[l, :n].copy(),
            "type": types[l, :n].astype(np.uint8),
            "bonds": bonds.reshape(-1, 2),
            "rot_edge": np.sort(chosen).astype(np.int32),
        })
    return out


def _chunk_args(args):
    return _chunk(*args)


def make_library(spec: dict, workers: int = 1) -> Library:
    """Generate the library described by `spec` (see gen.configs).

    workers > 1 grows the chunks in that many spawned processes (each chunk
    has its own generator, so the library is the same for any worker count;
    spawn, not fork, so a process that already holds a CUDA context may call
    it)."""
    L = int(spec["n_ligands"])
    seed = int(spec["seed"])
    jobs = [(seed, c, min(CHUNK, L - start), spec) for c, start in enumerate(range(0, L, CHUNK))]
    ligs: list[dict] = []
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(min(workers, len(jobs)), mp_context=mp.get_context("spawn")) as ex:
            for part in ex.map(_chunk_args, jobs):
                ligs.extend(part)
    else:
        for job in jobs:
            ligs.extend(_chunk(*job))
    return from_ligands(ligs)


def shuffle_bonds(lib: Library, seed: int) -> Library:
    """Same molecules with bond rows permuted and endpoints swapped at random.

    Rotatable-bond ids are remapped so that rotatable bond b still names the
    same chemical bond (the list keeps its order); the result describes the
    identical molecules in a different encoding.
    """
    rng = np.random.default_rng([seed, 7])
    ligs = []
    for l in range(lib.n_ligands):
        g = lib.ligand(l)
        b = g["bonds"].copy()
        perm = rng.permutation(len(b))
        flip = rng.random(len(b)) < 0.5
        nb = b[perm]
        nb[flip] = nb[flip][:, ::-1]
        inv = np.empty_like(perm)
        inv[perm] = np.arange(len(perm))
        ligs.append({**g, "bonds": nb, "rot_edge": inv[g["rot_edge"]].astype(np.int32)})
    return from_ligands(ligs)
