"""ligen_dock_batch_static: the docking call that allocates nothing.

Some callers cannot allocate device memory while they run: a framework whose
caching allocator already owns the device's memory, or a latency-bound
service that cannot afford the device-wide synchronisation of cudaMalloc.
This entry point docks with the library's fixed device scratch array instead
of an allocated workspace. It is checked here against ligen_dock_batch on the
same inputs, on two calls in a row (the array keeps the previous call's
contents, which must not leak into the next result). Needs a GPU; this file
is collected last."""
import numpy as np
import pytest
import torch

import gen
import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2303_06150_gb300 as lg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = gen.WORKLOADS["small32"]
    lib = gen.make_library(w["library"])
    grid = gen.make_grid(w["grid"])
    s = w["search"]
    kw = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
              top_k=s["top_k"], seed=s["seed"], n_rigid=s["n_rigid"], jitter=s["jitter"],
              out_penalty=s["out_penalty"])
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    return lg, lib, grid, kw, L, G


def test_static_scratch_call_matches_dock_batch_twice(setup):
    lg, lib, grid, kw, L, G = setup
    ref = lg.dock_batch(L, G, **kw)
    torch.cuda.synchronize()
    ref_scores = ref.scores.cpu().numpy()
    ref_poses = ref.poses.cpu().numpy()
    # outputs allocated up front, so the two calls below allocate nothing
    out = lg.DockResult(poses=torch.empty_like(ref.poses), scores=torch.empty_like(ref.scores),
                        status=torch.empty_like(ref.status), trace=None, top_restart=None, stage_ms=None)
    other = gen.make_library(dict(gen.WORKLOADS["small32"]["library"], seed=9))
    Lo = lg.Ligands.from_arrays(other, "cuda")
    for call in range(2):
        if call == 1:
            # a different batch in between leaves different contents in the array
            lg.dock_batch_static(Lo, G, **dict(kw, seed=kw["seed"] + 5))
        out.scores.fill_(float("nan"))
        out.poses.fill_(float("nan"))
        lg.dock_batch_static(L, G, out=out, **kw)
        torch.cuda.synchronize()
        sc = out.scores.cpu().numpy()
        po = out.poses.cpu().numpy()
        assert int(out.status.abs().sum()) == 0
        tol = parity.SCORE_RTOL * np.maximum(np.abs(ref_scores), 1.0)
        assert np.all(np.abs(sc - ref_scores) <= tol), call
        np.testing.assert_allclose(po, ref_poses, atol=1e-5)


def test_static_scratch_rejects_batches_beyond_its_size(setup):
    lg, lib, grid, kw, L, G = setup
    big = gen.make_grid(gen.WORKLOADS["screen20k"]["grid"])       # 96^3 x 8: 219 MB of records
    Gb = lg.PocketGrid.from_array(big.values, big.origin, big.spacing, "cuda")
    with pytest.raises(lg.LigenError) as e:
        lg.dock_batch_static(L, Gb, **kw)
    assert e.value.code == -2 and "scratch" in str(e.value)
