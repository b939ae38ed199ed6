"""Exhaustive search (mode 1) vs the oracle's brute force (needs a GPU).

Per restart the GPU's best score equals the oracle's exhaustive maximum
within the score tolerance, and the GPU's chosen pose scores (in the
oracle, FP64) within the decision tolerance of that maximum: where several
combinations are near-ties, either may be chosen. The greedy search never
beats the exhaustive one, restart by restart."""
import numpy as np
import pytest
import torch

import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lg():
    import paper_2303_06150_gb300 as lg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lg


def _kw(s, R):
    return dict(restarts=R, torsion_step_deg=s["torsion_step_deg"], passes=s["passes"], top_k=R, seed=s["seed"],
                n_rigid=s["n_rigid"], jitter=s["jitter"], out_penalty=s["out_penalty"], top_restart=True)


@pytest.mark.parametrize("fmt", ["f32", "f16"])
def test_exhaustive_matches_oracle_brute_force(lg, oracle_lib, small32, fmt):
    w, lib, grid = small32
    s = w["search"]
    R = 4
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    ex = lg.dock_batch(L, G, mode="exhaustive", grid_format=fmt, **_kw(s, R))
    gr = lg.dock_batch(L, G, mode="greedy", grid_format=fmt, **_kw(s, R))
    torch.cuda.synchronize()
    sc, top, poses = ex.scores.cpu().numpy(), ex.top_restart.cpu().numpy(), ex.poses.cpu().numpy()
    gsc, gtop = gr.scores.cpu().numpy(), gr.top_restart.cpu().numpy()
    og = oracle_lib.OGrid.from_grid(grid)
    off = lg.pose_offsets(lib.rot_off, R)
    checked = 0
    # FP16 records round the grid: compare against the oracle with the record error allowed for
    rec_tol = 0.0 if fmt == "f32" else 1e-3
    for l in range(lib.n_ligands):
        lig = oracle_lib.OLigand.from_library(lib, l)
        rs = range(0, R) if lig.n_rot <= 2 else range(0, 2)
        ref = oracle_lib.dock_exhaustive(lig, og, s, l, rs)
        gpu_best = {int(top[l, k]): float(sc[l, k]) for k in range(R)}
        gpu_pose = {int(top[l, k]): poses[off[l]:off[l + 1]].reshape(R, -1)[k] for k in range(R)}
        greedy = {int(gtop[l, k]): float(gsc[l, k]) for k in range(R)}
        for j, r in enumerate(rs):
            S_ref = ref["score"][j]
            _, D, _, Gs = oracle_lib.score_pose(lig, og, ref["pose"][j], 5.0, sensitivity=True)
            tol = parity.score_tol(D, Gs) + rec_tol * D
            assert abs(gpu_best[r] - S_ref) <= tol + parity.gap_tol(D, Gs), (l, r, gpu_best[r], S_ref)
            S_of_gpu, _, _ = oracle_lib.score_pose(lig, og, gpu_pose[r].astype(np.float64), 5.0)
            assert S_of_gpu >= S_ref - parity.gap_tol(D, Gs) - rec_tol * D, (l, r, S_of_gpu, S_ref)
            assert greedy[r] <= gpu_best[r] + tol, (l, r, greedy[r], gpu_best[r])
            checked += 1
    assert checked >= 80


def test_exhaustive_zero_field_takes_first_combination(lg, small32):
    w, lib, _ = small32
    s = w["search"]
    R = 6
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(np.zeros((41, 41, 41, 4)), (0.0, 0.0, 0.0), 1.0, "cuda")
    ex = lg.dock_batch(L, G, mode="exhaustive", **_kw(s, R))
    gr = lg.dock_batch(L, G, mode="greedy", **_kw(s, R))
    torch.cuda.synchronize()
    assert torch.all(ex.scores == 0)
    assert torch.equal(ex.top_restart.cpu(), torch.arange(R, dtype=torch.int32).repeat(lib.n_ligands, 1))
    # the first combination (k = 0, every j = 0) is the greedy search's all-ties result
    assert torch.equal(ex.poses, gr.poses)


def test_exhaustive_limits(lg, small32, screen_sample):
    w, lib, grid = screen_sample
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    assert lib.n_rot.max() > 4
    with pytest.raises(lg.LigenError) as e:
        lg.dock_batch(L, G, mode="exhaustive", **_kw(w["search"], 4))
    assert e.value.code == -2
    w, lib, grid = small32
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    with pytest.raises(lg.LigenError) as e:
        lg.dock_batch(L, G, mode="exhaustive", **dict(_kw(w["search"], 4), trace=True))
    assert e.value.code == -1
