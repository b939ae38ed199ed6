"""Precision forms: 16-bit grid records and the FP64 re-score (needs a GPU).

* FP64 re-score: the GPU's FP64 scores of the kept poses equal the oracle's
  scores of the same poses on the same FP32 grid values within 1e-9 * D (both
  are FP64 evaluations; only the order of the sums differs).
* FP16 / BF16 records: relative score error of every kept pose against the
  oracle's FP64 score of that pose (error / D) and best-pose agreement: the
  form's best pose scores, in the oracle, within 1e-3 * D of the best final
  score of the oracle's own search. The bar for a precision form is <= 1e-3
  relative error and >= 99% agreement."""
import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lg():
    import paper_2303_06150_gb300 as lg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lg


def _kw(s, **over):
    d = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"], top_k=s["top_k"],
             seed=s["seed"], n_rigid=s["n_rigid"], jitter=s["jitter"], out_penalty=s["out_penalty"])
    d.update(over)
    return d


@pytest.mark.parametrize("fmt", ["f32", "f16"])
def test_fp64_rescore_matches_oracle(lg, oracle_lib, small32, fmt):
    w, lib, grid = small32
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    res = lg.dock_batch(L, G, rescore_fp64=True, top_restart=True, grid_format=fmt, **_kw(w["search"]))
    torch.cuda.synchronize()
    s64 = res.scores_f64.cpu().numpy()
    sc = res.scores.cpu().numpy()
    top = res.top_restart.cpu().numpy()
    K = s64.shape[1]
    assert np.all(np.diff(s64, axis=1) <= 0)
    np.testing.assert_array_equal(sc, s64.astype(np.float32))
    og32 = oracle_lib.OGrid(grid.values.astype(np.float32).astype(np.float64), grid.origin, grid.spacing)
    poses = res.poses.cpu().numpy()
    off = lg.pose_offsets(lib.rot_off, K)
    for l in range(lib.n_ligands):
        lig = oracle_lib.OLigand.from_library(lib, l)
        lig32 = oracle_lib.OLigand(lig.xyz.astype(np.float32).astype(np.float64), lig.type, lig.bonds,
                                   lig.rot_edge)
        P = poses[off[l]:off[l + 1]].reshape(K, -1).astype(np.float64)
        for k in range(K):
            S, D, _ = oracle_lib.score_pose(lig32, og32, P[k], 5.0)
            assert abs(s64[l, k] - S) <= 1e-9 * D, (l, k, s64[l, k], S)
        for k in range(K - 1):   # equal FP64 scores keep the lower restart first
            if s64[l, k] == s64[l, k + 1]:
                assert top[l, k] < top[l, k + 1]


@pytest.mark.parametrize("fmt, max_err, min_agree", [("f16", 1e-3, 0.99), ("bf16", 1e-2, 0.9)])
def test_16bit_grid_error_and_best_pose_agreement(lg, oracle_lib, screen_sample, fmt, max_err, min_agree):
    w, lib, grid = screen_sample
    s = dict(w["search"], restarts=64, top_k=8)
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    res = lg.dock_batch(L, G, grid_format=fmt, **_kw(s))
    torch.cuda.synchronize()
    sc = res.scores.cpu().numpy()
    poses = res.poses.cpu().numpy()
    K = s["top_k"]
    og = oracle_lib.OGrid.from_grid(grid)
    off = lg.pose_offsets(lib.rot_off, K)
    ref = oracle_lib.dock_library(lib, grid, s)
    errs, agree = [], 0
    for r_ in ref:
        l = r_["ligand"]
        lig = oracle_lib.OLigand.from_library(lib, l)
        P = poses[off[l]:off[l + 1]].reshape(K, -1).astype(np.float64)
        best_oracle_of_gpu = -np.inf
        for k in range(K):
            S, D, _ = oracle_lib.score_pose(lig, og, P[k], 5.0)
            errs.append(abs(sc[l, k] - S) / D)
            best_oracle_of_gpu = max(best_oracle_of_gpu, S)
        j = int(np.argmax(r_["score"]))
        D = r_["dnorm"][j, -1]
        agree += best_oracle_of_gpu >= r_["score"][j] - 1e-3 * D
    errs = np.array(errs)
    rate = agree / len(ref)
    print(f"{fmt}: relative score error max {errs.max():.2e} mean {errs.mean():.2e}; "
          f"best-pose agreement {rate:.3f}")
    assert errs.max() <= max_err and rate >= min_agree
