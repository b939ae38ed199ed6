"""Multi-site docking (one library, several docking sites) vs single-site
docking and the oracle (needs a GPU).

Each site's slice of ligen_dock_sites must equal ligen_dock_batch on that
site's grid bit for bit (same seed and settings, same kernels); the oracle
checks one site whose box is off the origin and has another size and
spacing than the others."""
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


@pytest.fixture(scope="module")
def sites(small32):
    w, lib, _ = small32
    specs = gen.site_grids(w["grid"], 3)
    specs[2] = dict(specs[2], points=34, spacing=0.6)      # a larger box at a coarser spacing
    return w, lib, [gen.make_grid(s) for s in specs]


def _kw(s, **over):
    d = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"], top_k=s["top_k"],
             seed=s["seed"], n_rigid=s["n_rigid"], jitter=s["jitter"], out_penalty=s["out_penalty"])
    d.update(over)
    return d


def _grids(lg, grids, device, pin=False):
    return [lg.PocketGrid.from_array(g.values, g.origin, g.spacing, device, pin=pin) for g in grids]


FIELDS = ("poses", "scores", "trace", "top_restart", "scores_f64")


def _equal_per_site(multi, singles):
    for g, one in enumerate(singles):
        for f in FIELDS:
            a, b = getattr(multi, f), getattr(one, f)
            assert (a is None) == (b is None), f
            if a is not None:
                assert torch.equal(a[g].cpu(), b.cpu()), (g, f)
        assert torch.equal(multi.status.cpu(), one.status.cpu())


@pytest.mark.parametrize("batching, fmt, rescore", [("plain", "f32", False), ("buckets", "f32", False),
                                                    ("plain", "f16", True)])
def test_sites_equal_single_site_calls(lg, sites, batching, fmt, rescore):
    w, lib, grids = sites
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = _grids(lg, grids, "cuda")
    kw = _kw(w["search"], trace=True, top_restart=True, batching=batching, grid_format=fmt, rescore_fp64=rescore)
    multi = lg.dock_sites(L, G, **kw)
    singles = [lg.dock_batch(L, g, **kw) for g in G]
    torch.cuda.synchronize()
    assert multi.scores.shape == (3, lib.n_ligands, w["search"]["top_k"])
    _equal_per_site(multi, singles)
    # the sites are different problems: their results differ
    assert not torch.equal(multi.scores[0], multi.scores[1])


def test_sites_host_memory_and_one_site(lg, sites):
    w, lib, grids = sites
    kw = _kw(w["search"], trace=True, top_restart=True, stage_ms=True)
    Ld = lg.Ligands.from_arrays(lib, "cuda")
    dev = lg.dock_sites(Ld, _grids(lg, grids, "cuda"), **kw)
    Lh = lg.Ligands.from_arrays(lib, "cpu", pin=True)
    host = lg.dock_sites(Lh, _grids(lg, grids, "cpu", pin=True), **kw)
    torch.cuda.synchronize()
    for f in ("poses", "scores", "trace", "top_restart", "status"):
        assert torch.equal(getattr(host, f), getattr(dev, f).cpu()), f
    assert host.stage_ms.sum() > 0
    one = lg.dock_sites(Ld, _grids(lg, grids[1:2], "cuda"), **kw)
    torch.cuda.synchronize()
    assert torch.equal(one.scores[0], dev.scores[1]) and torch.equal(one.trace[0], dev.trace[1])


def test_site_off_origin_matches_oracle(lg, oracle_lib, sites):
    w, lib, grids = sites
    s = w["search"]
    R = s["restarts"]
    L = lg.Ligands.from_arrays(lib, "cuda")
    res = lg.dock_sites(L, _grids(lg, grids, "cuda"), **_kw(s, top_k=R, trace=True, top_restart=True))
    torch.cuda.synchronize()
    tot = parity.new_stats()
    for g in (1, 2):
        trace = res.trace[g].cpu().numpy()
        scores = res.scores[g].cpu().numpy()
        top = res.top_restart[g].cpu().numpy()
        ref = oracle_lib.dock_library(lib, grids[g], s, ligands=range(0, lib.n_ligands, 2))
        for r_ in ref:
            l = r_["ligand"]
            gt = parity.ligand_trace(trace, lib.rot_off, R, s["passes"], l)
            final = {int(top[l, k]): float(scores[l, k]) for k in range(R)}
            st = parity.check_dock_ligand(l, r_, gt, final)
            parity.merge(tot, st)
    print(tot)
    assert tot["clean"] >= 0.9 * tot["restarts"] and tot["scores"] > 0
