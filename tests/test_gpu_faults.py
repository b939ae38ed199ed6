"""Failure handling that needs a GPU but faults nothing (needs a GPU).

An allocation failure is injected with the workspace cap: the call returns
LIGEN_ERR_OOM before any device work, the context stays usable, and the
next call after the cap is lifted gives the same results. Malformed ligands
are covered by the packer tests (per-ligand status, no trap)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lg():
    import paper_2303_06150_gb300 as lg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lg


def test_workspace_cap_injects_oom_and_recovers(lg, small32):
    w, lib, grid = small32
    s = w["search"]
    kw = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
              top_k=s["top_k"], seed=s["seed"])
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    ref = lg.dock_batch(L, G, **kw)
    poses = ref.poses.clone()
    torch.cuda.synchronize()
    lg.release_workspaces()
    lg.set_workspace_limit(4096)
    try:
        for call in (lambda: lg.dock_batch(L, G, **kw), lambda: lg.score_poses(L, G, poses, s["top_k"]),
                     lambda: lg.pose_grad(L, G, poses, s["top_k"])):
            with pytest.raises(lg.LigenError) as e:
                call()
            assert e.value.code == -3 and "limit" in str(e.value)
    finally:
        lg.set_workspace_limit(0)
    again = lg.dock_batch(L, G, **kw)
    torch.cuda.synchronize()
    assert torch.equal(again.scores, ref.scores) and torch.equal(again.poses, ref.poses)
