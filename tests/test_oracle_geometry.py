"""Pins of the oracle's fragments and pose geometry (no GPU)."""
import numpy as np
import pytest

import gen
import indep


def _ligands(lib, idx):
    import oracle
    return [oracle.OLigand.from_library(lib, l) for l in idx]


def _random_pose(rng, n, center):
    q = rng.normal(size=4)
    t = center + rng.uniform(-2, 2, 3)
    th = rng.uniform(-np.pi, np.pi, n)
    return np.concatenate([t, q, th])


def test_fragments_match_graph_components(oracle_lib, small32, screen_sample):
    for _, lib, _ in (small32, screen_sample):
        for variant in (lib, gen.shuffle_bonds(lib, 5)):
            for lig in _ligands(variant, range(variant.n_ligands)):
                st, mask, axis = oracle_lib.fragments(lig)
                assert st == 0
                m2, a2 = indep.fragments(lig.xyz, lig.bonds, lig.rot_edge)
                assert np.array_equal(mask, m2)
                assert np.array_equal(axis, a2)


def test_fragment_encoding_invariance(oracle_lib, screen_sample):
    _, lib, _ = screen_sample
    shuf = gen.shuffle_bonds(lib, 11)
    for a, b in zip(_ligands(lib, range(lib.n_ligands)), _ligands(shuf, range(lib.n_ligands))):
        _, ma, aa = oracle_lib.fragments(a)
        _, mb, ab = oracle_lib.fragments(b)
        assert np.array_equal(ma, mb) and np.array_equal(aa, ab)


def test_fragment_tie_takes_side_without_atom0(oracle_lib):
    import oracle
    xyz = np.array([[0, 0, 0], [1.5, 0, 0], [2, 1.4, 0], [3.5, 1.4, 0]], float)
    lig = oracle.OLigand(xyz, [0, 0, 0, 0], [[0, 1], [1, 2], [2, 3]], [1])
    st, mask, axis = oracle_lib.fragments(lig)
    assert st == 0
    assert mask[0].tolist() == [False, False, True, True]
    assert axis[0].tolist() == [1, 2]
    # same molecule numbered from the other end: atom 0 is now on the far side
    lig2 = oracle.OLigand(xyz[::-1].copy(), [0] * 4, [[3, 2], [2, 1], [1, 0]], [1])
    _, mask2, axis2 = oracle_lib.fragments(lig2)
    assert mask2[0].tolist() == [False, False, True, True]
    assert axis2[0].tolist() == [1, 2]


def test_fragments_are_laminar(oracle_lib, screen_sample):
    _, lib, _ = screen_sample
    for lig in _ligands(lib, range(lib.n_ligands)):
        _, mask, _ = oracle_lib.fragments(lig)
        for i in range(len(mask)):
            for j in range(len(mask)):
                inter = mask[i] & mask[j]
                assert (not inter.any()) or np.array_equal(inter, mask[i]) or np.array_equal(inter, mask[j])


@pytest.mark.parametrize("bad", ["cycle", "range", "rot_range", "type", "empty"])
def test_invalid_ligands_rejected(oracle_lib, bad):
    import oracle
    xyz = np.zeros((4, 3))
    bonds, rot, types = [[0, 1], [1, 2], [2, 3]], [1], [0, 1, 2, 3]
    if bad == "cycle":
        bonds = [[0, 1], [1, 2], [2, 0]]
    elif bad == "range":
        bonds = [[0, 1], [1, 2], [2, 4]]
    elif bad == "rot_range":
        rot = [3]
    elif bad == "type":
        types = [0, 1, 2, 9]
    elif bad == "empty":
        xyz, bonds, rot, types = np.zeros((0, 3)), np.zeros((0, 2)), [], []
    lig = oracle.OLigand(xyz, types, bonds, rot)
    assert oracle_lib.validate(lig, 4) == 1


def test_pose_coords_match_scipy(oracle_lib, small32, screen_sample):
    rng = np.random.default_rng(5)
    for _, lib, grid in (small32, screen_sample):
        for lig in _ligands(lib, range(0, lib.n_ligands, 3)):
            pose = _random_pose(rng, lig.n_rot, grid.center)
            got = oracle_lib.pose_coords(lig, pose)
            ref = indep.pose_coords(lig.xyz, lig.bonds, lig.rot_edge, pose)
            np.testing.assert_allclose(got, ref, atol=1e-12)
            # torsions commute: any order of application gives the same pose
            order = rng.permutation(lig.n_rot)
            ref2 = indep.pose_coords(lig.xyz, lig.bonds, lig.rot_edge, pose, order=order)
            np.testing.assert_allclose(got, ref2, atol=1e-12)


def test_rigid_motion_preserves_all_distances(oracle_lib, screen_sample):
    _, lib, grid = screen_sample
    rng = np.random.default_rng(6)
    for lig in _ligands(lib, range(16)):
        pose = _random_pose(rng, lig.n_rot, grid.center)
        pose[7:] = 0
        x = oracle_lib.pose_coords(lig, pose)
        d0 = np.linalg.norm(lig.xyz[:, None] - lig.xyz[None], axis=-1)
        d1 = np.linalg.norm(x[:, None] - x[None], axis=-1)
        np.testing.assert_allclose(d1, d0, atol=1e-12)
        np.testing.assert_allclose(x.mean(0), pose[:3], atol=1e-12)   # centroid goes to t


def test_torsions_preserve_bonds_and_fragment_shapes(oracle_lib, screen_sample):
    _, lib, grid = screen_sample
    rng = np.random.default_rng(7)
    for lig in _ligands(lib, range(32)):
        if lig.n_rot == 0:
            continue
        pose = _random_pose(rng, lig.n_rot, grid.center)
        x = oracle_lib.pose_coords(lig, pose)
        b0 = np.linalg.norm(lig.xyz[lig.bonds[:, 0]] - lig.xyz[lig.bonds[:, 1]], axis=1)
        b1 = np.linalg.norm(x[lig.bonds[:, 0]] - x[lig.bonds[:, 1]], axis=1)
        np.testing.assert_allclose(b1, b0, atol=1e-12)
        _, mask, axis = oracle_lib.fragments(lig)
        # atoms of the innermost fragment of every bond keep their distances
        for b in range(lig.n_rot):
            inner = mask[b].copy()
            for c in range(lig.n_rot):
                if c != b and (mask[c] & mask[b]).any() and mask[c].sum() < mask[b].sum():
                    inner &= ~mask[c]
            sel = np.nonzero(inner)[0]
            d0 = np.linalg.norm(lig.xyz[sel, None] - lig.xyz[None, sel], axis=-1)
            d1 = np.linalg.norm(x[sel, None] - x[None, sel], axis=-1)
            np.testing.assert_allclose(d1, d0, atol=1e-12)


def test_full_turn_pose_is_identity(oracle_lib, screen_sample):
    _, lib, grid = screen_sample
    rng = np.random.default_rng(8)
    for lig in _ligands(lib, range(8)):
        pose = _random_pose(rng, lig.n_rot, grid.center)
        turned = pose.copy()
        turned[7:] += 2 * np.pi
        np.testing.assert_allclose(oracle_lib.pose_coords(lig, turned), oracle_lib.pose_coords(lig, pose),
                                   atol=1e-12)
