"""Independent restatements used to pin the oracle.

Each helper reaches the same quantity as the oracle by a different route:
networkx connected components for fragments, scipy's Rotation for quaternions,
torsions and rigid motion, and scipy's RegularGridInterpolator for trilinear
sampling. None of it imports the oracle or the CUDA library.
"""
from __future__ import annotations

import networkx as nx
import numpy as np
from scipy.interpolate import RegularGridInterpolator
from scipy.spatial.transform import Rotation


def fragments(xyz, bonds, rot_edge):
    """Moving side of each rotatable bond via graph components.

    Returns (mask [n, N] bool, axis [n, 2] (fixed u, moving v)).
    """
    N = len(xyz)
    G = nx.Graph()
    G.add_nodes_from(range(N))
    G.add_edges_from(map(tuple, np.asarray(bonds)))
    masks, axes = [], []
    for e in rot_edge:
        a, b = (int(v) for v in bonds[e])
        H = G.copy()
        H.remove_edge(a, b)
        ca = nx.node_connected_component(H, a)
        cb = set(range(N)) - ca
        if len(ca) < len(cb) or (len(ca) == len(cb) and 0 not in ca):
            mv, u, v = ca, b, a
        else:
            mv, u, v = cb, a, b
        m = np.zeros(N, bool)
        m[list(mv)] = True
        masks.append(m)
        axes.append((u, v))
    return np.array(masks, bool).reshape(len(rot_edge), N), np.array(axes, int).reshape(-1, 2)


def rot_from_wxyz(q) -> Rotation:
    q = np.asarray(q, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]])


def pose_coords(xyz, bonds, rot_edge, pose, order=None, frags=None):
    """Atom positions of pose (t, q, theta), torsions applied in `order`.

    Any order gives the same result because moving fragments are nested or
    disjoint; the default is index order.
    """
    xyz = np.asarray(xyz, np.float64)
    mask, axis = fragments(xyz, bonds, rot_edge) if frags is None else frags
    y = xyz.copy()
    order = range(len(rot_edge)) if order is None else order
    for b in order:
        u, v = axis[b]
        k = y[v] - y[u]
        k = k / np.linalg.norm(k)
        R = Rotation.from_rotvec(pose[7 + b] * k)
        y[mask[b]] = R.apply(y[mask[b]] - y[v]) + y[v]
    c0 = xyz.mean(0)
    return rot_from_wxyz(pose[3:7]).apply(y - c0) + np.asarray(pose[:3])


def trilinear_sampler(values, origin, spacing):
    """f(c, pts) -> (E, inbox) using scipy's linear grid interpolation."""
    nz, ny, nx_, nc = values.shape
    axes = [origin[2] + spacing * np.arange(nz), origin[1] + spacing * np.arange(ny),
            origin[0] + spacing * np.arange(nx_)]
    interp = [RegularGridInterpolator(axes, values[..., c], method="linear", bounds_error=False,
                                      fill_value=np.nan) for c in range(nc)]
    lo = np.asarray(origin, np.float64)
    hi = lo + spacing * (np.array([nx_, ny, nz]) - 1)

    def f(c, pts):
        pts = np.atleast_2d(np.asarray(pts, np.float64))
        inb = np.all((pts >= lo) & (pts <= hi), axis=1)
        out = np.zeros(len(pts))
        if inb.any():
            out[inb] = interp[c](pts[inb][:, ::-1])
        return out, inb

    return f


def score_coords(sampler, types, pts, penalty=5.0):
    """(S, D, E) with S = -sum E, D = max(|S|, sum |E|)."""
    E = np.zeros(len(pts))
    for c in np.unique(types):
        sel = types == c
        e, inb = sampler(int(c), pts[sel])
        e[~inb] = penalty
        E[sel] = e
    S = -E.sum()
    return S, max(abs(S), np.abs(E).sum()), E
