"""Pins of the oracle's greedy search, exhaustive search and top-K (no GPU)."""
import numpy as np
import pytest

import indep


def _setup(lib, grid, l):
    import oracle
    lig = oracle.OLigand.from_library(lib, l)
    samp = indep.trilinear_sampler(grid.values, grid.origin, grid.spacing)
    frags = indep.fragments(lig.xyz, lig.bonds, lig.rot_edge)
    return lig, samp, frags


def _indep_score(lig, samp, frags, t, rot, theta, penalty):
    """Independent score: torsions via scipy, then rotation `rot`, translation t."""
    pose = np.concatenate([np.zeros(3), [1, 0, 0, 0], theta])
    y = indep.pose_coords(lig.xyz, lig.bonds, lig.rot_edge, pose, frags=frags)
    pts = rot.apply(y) + t
    S, D, _ = indep.score_coords(samp, lig.type, pts, penalty)
    return S, D


def _replay(oracle_lib, w, lib, grid, l, restarts):
    """Re-derive every greedy decision with the independent scorer."""
    search = w["search"]
    og = oracle_lib.OGrid.from_grid(grid)
    lig, samp, frags = _setup(lib, grid, l)
    res = oracle_lib.dock_ligand(lig, og, search, l, restarts)
    step, P, n = search["torsion_step_deg"], search["passes"], lig.n_rot
    nt = 360 // step
    pen = search["out_penalty"]
    for j, r in enumerate(restarts):
        qr, tr = oracle_lib.restart_init(og, search, l, r)
        u = [oracle_lib.uniform(search["seed"], l, r, k) for k in range(6)]
        np.testing.assert_allclose(qr, oracle_lib.shoemake(u[:3]), atol=0)
        np.testing.assert_allclose(tr, grid.center + (2 * np.array(u[3:]) - 1) * search["jitter"], atol=1e-12)
        Rr = indep.rot_from_wxyz(qr)
        rig = [_indep_score(lig, samp, frags, tr, Rr * indep.rot_from_wxyz(oracle_lib.octahedral(k)),
                            np.zeros(n), pen) for k in range(search["n_rigid"])]
        s = np.array([v[0] for v in rig])
        k = int(np.argmax(s))
        srt = np.sort(s)[::-1]
        assert res["trace"][j, 0] == k
        assert abs(res["gap"][j, 0] - (srt[0] - srt[1])) <= 1e-10 * rig[k][1]
        rot = Rr * indep.rot_from_wxyz(oracle_lib.octahedral(k))
        counts = np.zeros(n, int)
        for p in range(P):
            for b in range(n):
                cand = []
                for jj in range(nt):
                    c = counts.copy()
                    c[b] += jj
                    cand.append(_indep_score(lig, samp, frags, tr, rot, np.radians(c * step), pen))
                s = np.array([v[0] for v in cand])
                jb = int(np.argmax(s))
                srt = np.sort(s)[::-1]
                d = 1 + p * n + b
                if srt[0] - srt[1] > 1e-9 * cand[jb][1]:
                    assert res["trace"][j, d] == jb
                jb = int(res["trace"][j, d])
                assert abs(res["gap"][j, d] - (srt[0] - srt[1])) <= 1e-10 * cand[jb][1]
                assert abs(res["dnorm"][j, d] - cand[jb][1]) <= 1e-10 * cand[jb][1]
                counts[b] = (counts[b] + jb) % nt
        # final pose: canonical quaternion, wrapped angles, consistent score
        pose = res["pose"][j]
        assert pose[3] >= 0 and abs(np.linalg.norm(pose[3:7]) - 1) < 1e-14
        assert np.all((pose[7:] >= -np.pi) & (pose[7:] < np.pi))
        S, D = _indep_score(lig, samp, frags, pose[:3], indep.rot_from_wxyz(pose[3:7]), pose[7:], pen)
        assert abs(res["score"][j] - S) <= 1e-10 * D
    return res


def test_greedy_decisions_are_argmaxes_small32(oracle_lib, small32):
    w, lib, grid = small32
    for l in range(0, lib.n_ligands, 4):
        _replay(oracle_lib, w, lib, grid, l, range(0, 3))


def test_greedy_decisions_are_argmaxes_screen(oracle_lib, screen_sample):
    w, lib, grid = screen_sample
    small = [l for l in range(lib.n_ligands) if lib.n_rot[l] <= 3 and lib.n_atoms[l] <= 30][:3]
    assert small
    for l in small:
        _replay(oracle_lib, w, lib, grid, l, range(5, 6))


def _touch_masks(frags):
    """Bit b of entry b': turning b' moves (its moving side without v_b') an
    atom that b's sweep reads (b's moving side or its fixed end u_b)."""
    mask, axis = frags
    n = len(mask)
    touch = []
    for bp in range(n):
        moved = mask[bp].copy()
        moved[axis[bp, 1]] = False
        t = 1 << bp
        for b in range(n):
            reads = mask[b].copy()
            reads[axis[b, 0]] = True
            if (moved & reads).any():
                t |= 1 << b
        touch.append(t)
    return touch


def test_clean_bonds_would_keep_their_torsion(oracle_lib, screen_sample):
    """The rule the docking kernel uses to skip sweeps, checked against the
    method with an independent FP64 scorer: a bond is clean after its own
    sweep (kept or turned) until a turn of a bond whose touch mask names it.
    At every decision the rule calls clean, a full re-sweep from that state
    (candidates recomputed from the accumulated torsions) has its maximum at
    j = 0 up to rounding, so deciding 0 without sampling is the method's own
    choice (exactly, or at a tie of rounding size)."""
    w, lib, grid = screen_sample
    search = w["search"]
    og = oracle_lib.OGrid.from_grid(grid)
    step, P = search["torsion_step_deg"], search["passes"]
    nt = 360 // step
    pen = search["out_penalty"]
    ligs = [l for l in range(lib.n_ligands) if 3 <= lib.n_rot[l] <= 6 and lib.n_atoms[l] <= 40][:3]
    assert ligs
    checked = turned_then_clean = 0
    for l in ligs:
        lig, samp, frags = _setup(lib, grid, l)
        touch = _touch_masks(frags)
        n = lig.n_rot
        res = oracle_lib.dock_ligand(lig, og, search, l, range(0, 2))
        for j, r in enumerate(range(0, 2)):
            qr, tr = oracle_lib.restart_init(og, search, l, r)
            rot = indep.rot_from_wxyz(qr) * indep.rot_from_wxyz(oracle_lib.octahedral(int(res["trace"][j, 0])))
            counts = np.zeros(n, int)
            dirty, turned = (1 << n) - 1, 0
            for d in range(P * n):
                b = d % n
                jb = int(res["trace"][j, 1 + d])
                if not dirty >> b & 1:
                    cand = []
                    for jj in range(nt):
                        c = counts.copy()
                        c[b] += jj
                        cand.append(_indep_score(lig, samp, frags, tr, rot, np.radians(c * step), pen))
                    s = np.array([v[0] for v in cand])
                    assert s.max() - s[0] <= 1e-9 * cand[0][1], (l, r, d, s.max() - s[0])
                    checked += 1
                    turned_then_clean += turned >> b & 1
                counts[b] = (counts[b] + jb) % nt
                turned = (turned | (1 << b)) if jb else turned & ~(1 << b)
                dirty = ((dirty | touch[b]) if jb else dirty) & ~(1 << b)
    assert checked > 0 and turned_then_clean > 0


def _rigid_copy(lib, l):
    import gen
    g = dict(lib.ligand(l))
    g["rot_edge"] = np.zeros(0, np.int32)
    return gen.from_ligands([g])


def test_rigid_ligand_greedy_equals_brute_force(oracle_lib, small32):
    w, lib, grid = small32
    og = oracle_lib.OGrid.from_grid(grid)
    for l in range(6):
        rl = _rigid_copy(lib, l)
        lig, samp, frags = _setup(rl, grid, 0)
        g = oracle_lib.dock_ligand(lig, og, w["search"], l)
        e = oracle_lib.dock_exhaustive(lig, og, w["search"], l)
        np.testing.assert_array_equal(g["score"], e["score"])
        for r in range(w["search"]["restarts"]):
            qr, tr = oracle_lib.restart_init(og, w["search"], l, r)
            Rr = indep.rot_from_wxyz(qr)
            s = [_indep_score(lig, samp, frags, tr, Rr * indep.rot_from_wxyz(oracle_lib.octahedral(k)),
                              np.zeros(0), 5.0)[0] for k in range(24)]
            assert abs(max(s) - g["score"][r]) <= 1e-10 * abs(max(s)) + 1e-12


@pytest.mark.parametrize("l", [0, 1, 2, 4, 5, 13])      # 1, 2 and 3 torsions (ligands 1 and 13: three)
def test_greedy_never_beats_exhaustive(oracle_lib, small32, l):
    w, lib, grid = small32
    og = oracle_lib.OGrid.from_grid(grid)
    lig, samp, frags = _setup(lib, grid, l)
    rs = range(0, 4)
    g = oracle_lib.dock_ligand(lig, og, w["search"], l, rs)
    e = oracle_lib.dock_exhaustive(lig, og, w["search"], l, rs)
    assert np.all(g["score"] <= e["score"] + 1e-12)
    # brute force over (k, j) for the first restart, independent scorer
    if lig.n_rot == 1:
        qr, tr = oracle_lib.restart_init(og, w["search"], l, 0)
        Rr = indep.rot_from_wxyz(qr)
        best = max(_indep_score(lig, samp, frags, tr, Rr * indep.rot_from_wxyz(oracle_lib.octahedral(k)),
                                np.radians([jj * 30.0]), 5.0)[0] for k in range(24) for jj in range(12))
        assert abs(best - e["score"][0]) <= 1e-10 * max(1.0, abs(best))


def test_top_k_order(oracle_lib):
    rng = np.random.default_rng(9)
    for _ in range(50):
        s = np.round(rng.normal(size=40), 1)            # many exact ties
        K = int(rng.integers(1, 40))
        ref = sorted(range(40), key=lambda i: (-s[i], i))[:K]
        assert oracle_lib.top_k(s, K).tolist() == ref


def test_refinement_is_monotone_and_consistent(oracle_lib, small32):
    """Accepted steps raise the score, rejected steps halve the steps; the
    returned pose re-scores to the returned score (independent scorer)."""
    w, lib, grid = small32
    og = oracle_lib.OGrid.from_grid(grid)
    samp = indep.trilinear_sampler(grid.values, grid.origin, grid.spacing)
    res = oracle_lib.dock_library(lib, grid, w["search"], ligands=range(0, 32, 4))
    for r_ in res:
        lig, _, frags = _setup(lib, grid, r_["ligand"])
        for k in range(2):
            p0 = r_["top_pose"][k]
            s0 = oracle_lib.score_pose(lig, og, p0)[0]
            pose, S, acc, gap = oracle_lib.refine_pose(lig, og, p0, steps=20)
            assert S >= s0 - 1e-12
            assert np.all(gap[acc == 1] > 0) and np.all(gap[acc == 0] <= 0)
            assert pose[3] >= 0 and abs(np.linalg.norm(pose[3:7]) - 1) < 1e-12
            S2, D = _indep_score(lig, samp, frags, pose[:3], indep.rot_from_wxyz(pose[3:7]), pose[7:], 5.0)
            assert abs(S2 - S) <= 1e-10 * D
    # a first step along the gradient of a smooth field is accepted
    lig = oracle_lib.OLigand.from_library(lib, 0)
    zz, yy, xx = np.meshgrid(*(0.5 * np.arange(40),) * 3, indexing="ij")
    vals = np.repeat((-(0.05 * xx + 0.03 * yy - 0.02 * zz))[..., None], 4, axis=3)
    lin = oracle_lib.OGrid(vals, (0.0, 0.0, 0.0), 0.5)
    p0 = np.concatenate([grid.center, [1, 0, 0, 0], np.zeros(lig.n_rot)])
    _, S, acc, _ = oracle_lib.refine_pose(lig, lin, p0, steps=5)
    assert acc[0] == 1 and S > oracle_lib.score_pose(lig, lin, p0)[0]


def test_zero_field_search_is_the_identity(oracle_lib, small32):
    """On a zero field every candidate scores exactly 0 (all atoms inside a
    40 A box), so every decision is a tie and the lowest index must win
    everywhere: k = 0, j = 0, every gap 0, the final pose is the restart's
    initial pose (canonical quaternion, zero torsions), and the top K are
    restarts 0..K-1 (equal scores: lower restart first). The exhaustive
    search keeps its first combination."""
    w, lib, _ = small32
    s = w["search"]
    zero = oracle_lib.OGrid(np.zeros((41, 41, 41, 4)), (0.0, 0.0, 0.0), 1.0)
    for l in range(0, lib.n_ligands, 3):
        lig = oracle_lib.OLigand.from_library(lib, l)
        res = oracle_lib.dock_ligand(lig, zero, s, l)
        assert np.all(res["score"] == 0.0)
        assert np.all(res["trace"] == 0) and np.all(res["gap"] == 0.0)
        for r in range(s["restarts"]):
            q, t = oracle_lib.restart_init(zero, s, l, r)
            q = np.sign(q[0]) * q / np.linalg.norm(q)
            np.testing.assert_allclose(res["pose"][r], np.concatenate([t, q, np.zeros(lig.n_rot)]), atol=1e-15)
        assert oracle_lib.top_k(res["score"], s["top_k"]).tolist() == list(range(s["top_k"]))
        if lig.n_rot <= 2:
            e = oracle_lib.dock_exhaustive(lig, zero, s, l, range(0, 2))
            np.testing.assert_array_equal(e["score"], 0.0)
            np.testing.assert_allclose(e["pose"], res["pose"][:2], atol=1e-15)


def test_refinement_rules_on_a_one_dimensional_bowl(oracle_lib):
    """One atom in a field that varies along x only: node values
    E(x) = (x - 5)^2 on a 0.5 A lattice, linear between nodes. The
    translation gradient points along +-x, so every step proposes x +- st
    (the quaternion and the y, z position have zero gradient and stay). The
    expected accept flags follow from the rules alone, replayed here with
    numpy's interpolation: accept only a strictly higher score, halve the
    step on a rejection, never grow it. From x = 3.25 with st = 0.5 the
    fourth proposal lands on a point of exactly equal score, which must be
    rejected."""
    h, n = 0.5, 21
    xs = h * np.arange(n)
    ex = (xs - 5.0) ** 2
    vals = np.ascontiguousarray(np.broadcast_to(ex[None, None, :, None], (n, n, n, 1)))
    g = oracle_lib.OGrid(vals, (0.0, 0.0, 0.0), h)
    one = oracle_lib.OLigand(np.zeros((1, 3)), [0], np.zeros((0, 2)), [])
    start = np.array([3.25, 4.0, 4.0, 1.0, 0.0, 0.0, 0.0])
    steps = 10
    pose, S, acc, gap = oracle_lib.refine_pose(one, g, start, steps=steps, step_t=0.5, step_q=0.02,
                                               step_theta=0.05)

    def energy(x):
        return float(np.interp(x, xs, ex))

    def slope(x):          # derivative inside the cell that holds x (the upper cell on a node)
        i = min(int(np.floor(x / h)), n - 2)
        return (ex[i + 1] - ex[i]) / h

    x, st, want = start[0], 0.5, []
    for _ in range(steps):
        prop = min(max(x - st * np.sign(slope(x)), 0.0), xs[-1])
        if -energy(prop) > -energy(x):
            x = prop
            want.append(1)
        else:
            st *= 0.5
            want.append(0)
    assert want[:5] == [1, 1, 1, 0, 1] and gap[3] == 0.0
    assert acc.tolist() == want
    assert pose[0] == x and pose[1] == 4.0 and pose[2] == 4.0
    np.testing.assert_array_equal(pose[3:], [1.0, 0.0, 0.0, 0.0])
    assert S == -energy(x)
