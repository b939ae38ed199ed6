"""Edge cases of the docking path against the oracle (needs a GPU).

Maximum ligand size (256 atoms, 32 rotatable bonds), degenerate search
settings (no sweep pass, one rigid rotation, a 360-degree step, one restart,
restart counts that leave a partial chunk), a one-atom ligand, a rotatable
bond whose moving side is a single atom (an empty moving list), and a grid
of a single cell that most atoms fall outside of; the maximum sizes and the
single-cell grid also with 16-bit grid records (against the oracle on the
rounded node values)."""
import numpy as np
import pytest
import torch

import gen
import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lg():
    import paper_2303_06150_gb300 as lg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lg


def _dock_and_check(lg, oracle_lib, lib, grid, s, restarts=None, min_clean=0.9, fmt="f32"):
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    R, K = s["restarts"], s["top_k"]
    res = lg.dock_batch(L, G, restarts=R, torsion_step_deg=s["torsion_step_deg"], passes=s["passes"], top_k=K,
                        seed=s["seed"], n_rigid=s["n_rigid"], jitter=s["jitter"], out_penalty=s["out_penalty"],
                        trace=True, top_restart=True, grid_format=fmt)
    torch.cuda.synchronize()
    assert int(res.status.abs().sum()) == 0
    trace, scores, top = res.trace.cpu().numpy(), res.scores.cpu().numpy(), res.top_restart.cpu().numpy()
    ref = oracle_lib.dock_library(lib, parity.oracle_grid(oracle_lib, grid, fmt), s, restarts=restarts)
    tot = parity.new_stats()
    for r_ in ref:
        l = r_["ligand"]
        gt = parity.ligand_trace(trace, lib.rot_off, R, s["passes"], l)
        final = {int(top[l, k]): float(scores[l, k]) for k in range(K)}
        st = parity.check_dock_ligand(l, r_, gt, final)
        parity.merge(tot, st)
        assert np.all(np.diff(scores[l]) <= 0)
    print(tot)
    assert tot["clean"] >= min_clean * tot["restarts"] and tot["scores"] > 0
    return res


@pytest.mark.parametrize("fmt", ["f32", "f16"])
def test_maximum_size_ligands(lg, oracle_lib, fmt):
    spec = dict(kind="uniform", n_ligands=3, n_atoms=(256, 256), n_rot=(32, 32), n_types=8, seed=11)
    lib = gen.make_library(spec)
    assert lib.n_atoms.max() == 256 and lib.n_rot.max() == 32
    grid = gen.make_grid(gen.WORKLOADS["screen20k"]["grid"])
    s = dict(gen.WORKLOADS["screen20k"]["search"], restarts=16, top_k=16, passes=2, torsion_step_deg=30)
    _dock_and_check(lg, oracle_lib, lib, grid, s, restarts=range(0, 4), min_clean=0.75, fmt=fmt)


@pytest.mark.parametrize("over", [dict(passes=0), dict(n_rigid=1), dict(torsion_step_deg=360),
                                  dict(restarts=1, top_k=1), dict(restarts=13, top_k=13),
                                  dict(restarts=37, top_k=5)])
def test_degenerate_search_settings(lg, oracle_lib, small32, over):
    w, lib, grid = small32
    s = dict(w["search"], **over)
    res = _dock_and_check(lg, oracle_lib, lib, grid, s)
    trace = res.trace.cpu().numpy()
    if over.get("n_rigid") == 1:
        for l in range(lib.n_ligands):
            assert np.all(parity.ligand_trace(trace, lib.rot_off, s["restarts"], s["passes"], l)[:, 0] == 0)
    if over.get("torsion_step_deg") == 360:   # one increment: every sweep keeps the torsion
        for l in range(lib.n_ligands):
            assert np.all(parity.ligand_trace(trace, lib.rot_off, s["restarts"], s["passes"], l)[:, 1:] == 0)


def test_one_atom_ligand_and_empty_moving_list(lg, oracle_lib, small32):
    w, _, grid = small32
    one = dict(xyz=np.zeros((1, 3)), type=np.array([2], np.uint8), bonds=np.zeros((0, 2), np.int32),
               rot_edge=np.zeros(0, np.int32))
    # atoms 0-1-2-3 in a chain, plus atom 4 on atom 1: bond 3 (1-4) turns atom 4 alone,
    # bond 1 (1-2) turns atoms 2 and 3
    xyz = np.array([[0, 0, 0], [1.5, 0, 0], [2.0, 1.4, 0], [3.5, 1.4, 0.2], [1.9, -1.0, 1.0]], float)
    chain = dict(xyz=xyz, type=np.array([0, 1, 2, 3, 1], np.uint8),
                 bonds=np.array([[0, 1], [1, 2], [2, 3], [1, 4]], np.int32), rot_edge=np.array([1, 3], np.int32))
    lib = gen.from_ligands([one, chain, one])
    s = dict(w["search"], restarts=8, top_k=8)
    _dock_and_check(lg, oracle_lib, lib, grid, s)


@pytest.mark.parametrize("fmt", ["f32", "f16", "bf16"])
def test_single_cell_grid(lg, oracle_lib, small32, fmt):
    w, lib, _ = small32
    rng = np.random.default_rng(5)
    values = rng.normal(-1.0, 0.5, (2, 2, 2, 4))
    grid = gen.Grid(values=values, origin=(-0.4, -0.3, -0.2), spacing=0.9, centers=np.zeros((0, 3)),
                    weights=np.zeros((0, 4)))
    s = dict(w["search"], restarts=8, top_k=8, jitter=0.3)
    sub = lib.subset(range(0, 8))
    _dock_and_check(lg, oracle_lib, sub, grid, s, fmt=fmt)


@pytest.mark.parametrize("P", [15, 16, 33])    # group-per-pose kernel, then one pose per lane (1 and 2 warps)
def test_scoring_at_maximum_sizes(lg, oracle_lib, P):
    """ligen_score_poses and the prepared form on 256-atom, 32-bond ligands
    (the largest shared-memory carve-ups of both scoring kernels) plus a
    rigid and a one-atom ligand, against the oracle; the FP64 re-score of
    docked poses of the same ligands (its largest carve-up) against the
    oracle's FP64 score of the same poses."""
    spec = dict(kind="uniform", n_ligands=2, n_atoms=(256, 256), n_rot=(32, 32), n_types=8, seed=12)
    big = gen.make_library(spec)
    one = dict(xyz=np.zeros((1, 3)), type=np.array([1], np.uint8), bonds=np.zeros((0, 2), np.int32),
               rot_edge=np.zeros(0, np.int32))
    rigid = dict(big.ligand(0), rot_edge=np.zeros(0, np.int32))
    lib = gen.from_ligands([big.ligand(0), one, rigid, big.ligand(1)])
    grid = gen.make_grid(gen.WORKLOADS["screen20k"]["grid"])
    rng = np.random.default_rng(13)
    poses = []
    for l in range(lib.n_ligands):
        for _ in range(P):
            poses.append(np.concatenate([grid.center + rng.uniform(-3, 3, 3), rng.normal(size=4),
                                         rng.uniform(-np.pi, np.pi, lib.n_rot[l])]))
    poses = np.concatenate(poses).astype(np.float32)
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    pt = torch.tensor(poses, device="cuda")
    out = lg.score_poses(L, G, pt, P).cpu().numpy()
    prep = lg.prepare_scoring(L, G)
    assert np.array_equal(prep.score(pt, P).cpu().numpy(), out)
    prep.release()
    og = oracle_lib.OGrid.from_grid(grid)
    off = lg.pose_offsets(lib.rot_off, P)
    for l in range(lib.n_ligands):
        lig = oracle_lib.OLigand.from_library(lib, l)
        Pl = poses[off[l]:off[l + 1]].astype(np.float64).reshape(P, -1)
        for p in range(0, P, 4):
            S, D, _, Gs = oracle_lib.score_pose(lig, og, Pl[p], 5.0, sensitivity=True)
            assert abs(out[l, p] - S) <= parity.score_tol(D, Gs), (l, p, out[l, p], S)
    if P == 16:   # FP64 re-score of docked poses of the same ligands
        s = dict(gen.WORKLOADS["screen20k"]["search"], restarts=16, top_k=16, passes=1, torsion_step_deg=60)
        res = lg.dock_batch(L, G, restarts=16, torsion_step_deg=60, passes=1, top_k=16, seed=s["seed"],
                            rescore_fp64=True)
        s64 = res.scores_f64.cpu().numpy()
        dp = res.poses.cpu().numpy()
        o32 = oracle_lib.OGrid(np.asarray(grid.values, np.float32).astype(np.float64), grid.origin, grid.spacing)
        offk = lg.pose_offsets(lib.rot_off, 16)
        xyz32 = np.asarray(lib.xyz, np.float32).astype(np.float64)
        for l in range(lib.n_ligands):
            g = lib.ligand(l)
            lig32 = oracle_lib.OLigand(xyz32[lib.atom_off[l]:lib.atom_off[l + 1]], g["type"], g["bonds"],
                                       g["rot_edge"])
            Pl = dp[offk[l]:offk[l + 1]].astype(np.float64).reshape(16, -1)
            for k in range(0, 16, 5):
                S, D, _ = oracle_lib.score_pose(lig32, o32, Pl[k], 5.0)
                assert abs(s64[l, k] - S) <= 1e-9 * D, (l, k, s64[l, k], S)
            assert np.all(np.diff(s64[l]) <= 0)
