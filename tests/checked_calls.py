"""Calls that exercise every kernel of the library on small seeded inputs;
used by test_gpu_checked.py to run them once with the bounds-checked build
(libligen_checked.so, in a child process) and once with the normal build.

Run as a script: python tests/checked_calls.py <library.so> <out.npz>."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def run_all(lg) -> dict:
    import torch

    import gen
    out = {}
    w = gen.WORKLOADS["small32"]
    lib, grid = gen.make_library(w["library"]), gen.make_grid(w["grid"])
    ws = gen.scaled("screen20k", 48)
    libs, grids = gen.make_library(ws["library"]), gen.make_grid(ws["grid"])
    s = w["search"]
    kw = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
              top_k=s["top_k"], seed=s["seed"])
    kws = dict(restarts=32, torsion_step_deg=10, passes=2, top_k=8, seed=3)
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
    Ls = lg.Ligands.from_arrays(libs, "cuda")
    Gs = lg.PocketGrid.from_array(grids.values, grids.origin, grids.spacing, "cuda")

    def keep(name, res):
        for f in ("scores", "poses", "trace", "top_restart", "scores_f64", "status"):
            v = getattr(res, f)
            if v is not None:
                out[f"{name}.{f}"] = v.cpu().numpy()

    for fmt in ("f32", "f16", "bf16"):
        keep(f"small_{fmt}", lg.dock_batch(L, G, grid_format=fmt, trace=True, top_restart=True, **kw))
        keep(f"screen_{fmt}", lg.dock_batch(Ls, Gs, grid_format=fmt, trace=True, top_restart=True, **kws))
    keep("screen_buckets", lg.dock_batch(Ls, Gs, batching="buckets", trace=True, **kws))
    keep("screen_static_buckets", lg.dock_batch(Ls, Gs, batching="buckets_static", trace=True, **kws))
    keep("screen_rescore", lg.dock_batch(Ls, Gs, rescore_fp64=True, top_restart=True, **kws))
    keep("small_exhaustive", lg.dock_batch(L, G, mode="exhaustive", top_restart=True, **dict(kw, restarts=2,
                                                                                              top_k=2)))
    sites = [lg.PocketGrid.from_array(g.values, g.origin, g.spacing, "cuda")
             for g in (gen.make_grid(sp) for sp in gen.site_grids(w["grid"], 2))]
    keep("small_sites", lg.dock_sites(L, sites, trace=True, **kw))
    keep("small_static", lg.dock_batch_static(L, G, **kw))
    keep("screen_queue", lg.dock_batch(Ls, Gs, batching="queue", trace=True, **kws))
    docked = lg.dock_batch(Ls, Gs, **kws)
    K = kws["top_k"]
    out["score"] = lg.score_poses(Ls, Gs, docked.poses, K).cpu().numpy()
    # 30 poses per ligand: the pose-per-lane scoring kernel, one-shot and prepared
    d30 = lg.dock_batch(Ls, Gs, **dict(kws, top_k=30))
    out["score30"] = lg.score_poses(Ls, Gs, d30.poses, 30).cpu().numpy()
    prep = lg.prepare_scoring(Ls, Gs)
    out["score30_prepared"] = prep.score(d30.poses, 30).cpu().numpy()
    prep.release()
    # gradients: 8 poses per ligand (4 lanes per pose), 16 (2
    # lanes), 30 (1 lane) and 2 (the 16-lane group kernel)
    for k, poses in ((K, docked.poses), (30, d30.poses)):
        sc, gr = lg.pose_grad(Ls, Gs, poses, k)
        out[f"grad.scores{k}"], out[f"grad.grads{k}"] = sc.cpu().numpy(), gr.cpu().numpy()
    for k in (2, 16):
        dk = lg.dock_batch(Ls, Gs, **dict(kws, top_k=k))
        sc, gr = lg.pose_grad(Ls, Gs, dk.poses, k)
        out[f"grad.scores{k}"], out[f"grad.grads{k}"] = sc.cpu().numpy(), gr.cpu().numpy()
    refined, rs, acc = lg.refine_poses(Ls, Gs, docked.poses, K, steps=10, accept=True)
    out["refine.poses"], out["refine.scores"] = refined.cpu().numpy(), rs.cpu().numpy()
    out["refine.accept"] = acc.cpu().numpy()
    bits, axis, bucket, status = lg.pack_ligands(Ls, grids.dims[3])
    out["pack.bits"], out["pack.axis"] = bits.cpu().numpy(), axis.cpu().numpy()
    out["pack.bucket"], out["pack.status"] = bucket.cpu().numpy(), status.cpu().numpy()
    out["pack.touch"] = lg.pack_touch(Ls, grids.dims[3]).cpu().numpy()
    saved = lg.tune_get()
    try:
        tuned = lg.autotune(Ls, Gs, sample=16, **kws)
        out["autotune.buckets"] = np.array(sorted(tuned))
    finally:
        lg.tune_set(saved)
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    from paper_2303_06150_gb300 import _abi
    _abi.load(sys.argv[1])
    import paper_2303_06150_gb300 as lg
    np.savez(sys.argv[2], **run_all(lg))
    print("ok")
