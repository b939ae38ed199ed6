"""Pins of the oracle's random numbers and rotations (no GPU)."""
import itertools
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import indep

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def _golden_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def test_splitmix64_known_answers(oracle_lib):
    # SplitMix64 known-answer values from the published reference generator.
    for row in _golden_rows("splitmix64.txt"):
        state = int(row[0], 0)
        for expect in row[1:]:
            assert oracle_lib.splitmix64(state) == int(expect, 0)
            state = (state + GAMMA) & M64


def test_uniform_is_24_bit_and_uniform(oracle_lib):
    u = np.array([oracle_lib.uniform(123, l, r, k) for l in range(40) for r in range(50) for k in range(6)])
    assert np.all((u >= 0) & (u < 1))
    scaled = u * (1 << 24)
    assert np.all(scaled == np.floor(scaled))          # exactly 24 fractional bits
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005
    hist = np.histogram(u, bins=20, range=(0, 1))[0]
    chi2 = ((hist - len(u) / 20) ** 2 / (len(u) / 20)).sum()
    assert chi2 < 45                                     # 19 dof, p ~ 1e-3
    assert len(np.unique(u)) > 0.99 * len(u)             # distinct counters


def test_uniform_streams_differ_by_seed_ligand_restart(oracle_lib):
    base = oracle_lib.uniform(7, 3, 5, 0)
    assert oracle_lib.uniform(8, 3, 5, 0) != base
    assert oracle_lib.uniform(7, 4, 5, 0) != base
    assert oracle_lib.uniform(7, 3, 6, 0) != base
    assert oracle_lib.uniform(7, 3, 5, 1) != base


def test_quat_to_mat_matches_scipy(oracle_lib):
    rng = np.random.default_rng(1)
    for _ in range(200):
        q = rng.normal(size=4) * rng.uniform(0.2, 3.0)     # not unit on purpose
        m = oracle_lib.quat_to_mat(q)
        np.testing.assert_allclose(m, indep.rot_from_wxyz(q).as_matrix(), atol=1e-14)
        assert abs(np.linalg.det(m) - 1) < 1e-14
        np.testing.assert_allclose(m @ m.T, np.eye(3), atol=1e-14)


def test_quat_mul_composes_like_scipy(oracle_lib):
    rng = np.random.default_rng(2)
    for _ in range(100):
        a, b = rng.normal(size=4), rng.normal(size=4)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        ab = oracle_lib.quat_mul(a, b)
        ref = (indep.rot_from_wxyz(a) * indep.rot_from_wxyz(b)).as_matrix()
        np.testing.assert_allclose(oracle_lib.quat_to_mat(ab), ref, atol=1e-14)


def test_shoemake_unit_and_uniform_on_s3(oracle_lib):
    rng = np.random.default_rng(3)
    qs = np.array([oracle_lib.shoemake(rng.random(3)) for _ in range(20000)])
    np.testing.assert_allclose(np.linalg.norm(qs, axis=1), 1.0, atol=1e-15)
    # uniform on S^3: E[q_i^2] = 1/4, E[q_i^4] = 1/8, E[q_i q_j] = 0
    np.testing.assert_allclose((qs ** 2).mean(0), 0.25, atol=0.01)
    np.testing.assert_allclose((qs ** 4).mean(0), 0.125, atol=0.006)
    cov = (qs.T @ qs) / len(qs)
    assert np.abs(cov - np.diag(np.diag(cov))).max() < 0.01


def test_shoemake_special_values(oracle_lib):
    np.testing.assert_allclose(oracle_lib.shoemake([0, 0, 0]), [0, 0, 1, 0], atol=1e-16)
    np.testing.assert_allclose(oracle_lib.shoemake([1, 0.3, 0]), [1, 0, 0, 0], atol=1e-16)
    np.testing.assert_allclose(oracle_lib.shoemake([0, 0.25, 0]), [0, 1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(oracle_lib.shoemake([1, 0, 0.25]), [0, 0, 0, 1], atol=1e-15)


def _signed_permutations_det1():
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            m = np.zeros((3, 3))
            for r in range(3):
                m[r, perm[r]] = signs[r]
            if round(np.linalg.det(m)) == 1:
                out.append(m)
    return out


def test_octahedral_group_is_the_cube_rotation_group(oracle_lib):
    mats = [oracle_lib.quat_to_mat(oracle_lib.octahedral(k)) for k in range(24)]
    rounded = [np.round(m) for m in mats]
    for m, r in zip(mats, rounded):
        assert np.abs(m - r).max() < 1e-15
    keys = {tuple(r.astype(int).ravel()) for r in rounded}
    assert len(keys) == 24
    brute = {tuple(m.astype(int).ravel()) for m in _signed_permutations_det1()}
    assert keys == brute
    for a in rounded:                                   # closed under composition
        for b in rounded:
            assert tuple((a @ b).astype(int).ravel()) in keys


def test_octahedral_order(oracle_lib):
    def rotvec(k):
        return indep.rot_from_wxyz(oracle_lib.octahedral(k)).as_rotvec()
    np.testing.assert_allclose(rotvec(0), 0, atol=1e-15)
    for k, ax in zip((1, 2, 3), np.eye(3)):
        rv = rotvec(k)
        assert abs(np.linalg.norm(rv) - np.pi) < 1e-12
        np.testing.assert_allclose(np.abs(rv / np.pi), ax, atol=1e-12)
    for k in range(4, 10):
        a, sgn = (k - 4) // 2, 1 if (k - 4) % 2 == 0 else -1
        np.testing.assert_allclose(rotvec(k), sgn * np.pi / 2 * np.eye(3)[a], atol=1e-12)
    for k in range(10, 18):
        m = k - 10
        d = np.array([-1 if m & 4 else 1, -1 if m & 2 else 1, -1 if m & 1 else 1]) / np.sqrt(3)
        np.testing.assert_allclose(rotvec(k), 2 * np.pi / 3 * d, atol=1e-12)
    diag = [(1, 1, 0), (1, -1, 0), (0, 1, 1), (0, 1, -1), (1, 0, 1), (1, 0, -1)]
    for k, d in zip(range(18, 24), diag):
        rv = rotvec(k)
        d = np.array(d) / np.sqrt(2)
        assert abs(np.linalg.norm(rv) - np.pi) < 1e-12
        assert abs(abs(rv @ d) - np.pi) < 1e-12


def test_rodrigues_matches_scipy_rotvec(oracle_lib):
    rng = np.random.default_rng(4)
    for _ in range(200):
        p, a, d = rng.normal(size=(3, 3))
        th = rng.uniform(-7, 7)
        ref = Rotation.from_rotvec(th * d / np.linalg.norm(d)).apply(p - a) + a
        np.testing.assert_allclose(oracle_lib.rodrigues(p, a, d, th), ref, atol=1e-13)


@pytest.mark.parametrize("step", [30, 10])
def test_incremental_full_turn_is_identity(oracle_lib, step):
    rng = np.random.default_rng(step)
    p, a, d = rng.normal(size=(3, 3)) * 3
    x = p.copy()
    for _ in range(360 // step):
        x = oracle_lib.rodrigues(x, a, d, np.radians(step))
    np.testing.assert_allclose(x, p, atol=1e-12)


def test_torsion_angle_wraps(oracle_lib):
    for step in (10, 30, 45):
        for count in range(-40, 80):
            th = oracle_lib.torsion_angle(count, step)
            assert -np.pi <= th < np.pi
            assert abs(np.cos(th) - np.cos(np.radians(count * step))) < 1e-12
            assert abs(np.sin(th) - np.sin(np.radians(count * step))) < 1e-12
