"""Bucketed (batched) layout vs the plain launch and the oracle (needs a GPU).

The bucketed layout changes only where work runs: every decision must be
bit-identical to the plain launch; final scores may differ in the last bits
(the per-restart final sum is reduced over a different number of lanes when a
bucket is tuned to another shape)."""
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
def bimodal():
    w = gen.scaled("bimodal200k", 1500)
    w["search"] = dict(w["search"], restarts=32, top_k=8)
    return w, gen.make_library(w["library"]), gen.make_grid(w["grid"])


def _kw(s, **over):
    d = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"], top_k=s["top_k"],
             seed=s["seed"], n_rigid=s["n_rigid"], jitter=s["jitter"], out_penalty=s["out_penalty"])
    d.update(over)
    return d


def _dev(lg, lib, grid):
    return (lg.Ligands.from_arrays(lib, "cuda"),
            lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda"))


def _same_decisions_close_scores(a, b):
    assert torch.equal(a.trace, b.trace)
    sa, sb = a.scores.cpu().numpy(), b.scores.cpu().numpy()
    assert np.all(np.abs(sa - sb) <= 1e-5 * np.maximum(np.abs(sa), 1.0))


@pytest.mark.parametrize("fmt", ["f32", "f16"])
def test_buckets_match_plain_and_replay(lg, bimodal, fmt):
    w, lib, grid = bimodal
    L, G = _dev(lg, lib, grid)
    kw = _kw(w["search"], trace=True, top_restart=True, grid_format=fmt)
    plain = lg.dock_batch(L, G, batching="plain", **kw)
    b1 = lg.dock_batch(L, G, batching="buckets", **kw)
    b2 = lg.dock_batch(L, G, batching="buckets", **kw)     # graph replay
    torch.cuda.synchronize()
    _same_decisions_close_scores(plain, b1)
    assert torch.equal(b1.scores, b2.scores) and torch.equal(b1.poses, b2.poses)
    assert torch.equal(b1.trace, b2.trace)


@pytest.mark.parametrize("fmt", ["f32", "f16"])
def test_single_queue_launch_matches_plain(lg, bimodal, small32, fmt):
    """The whole library in one persistent launch (default shape, bucket
    order): same kernel shape as the plain launch, so bit-identical results."""
    for w, lib, grid in (bimodal, small32):
        L, G = _dev(lg, lib, grid)
        kw = _kw(w["search"], trace=True, top_restart=True, grid_format=fmt)
        plain = lg.dock_batch(L, G, batching="plain", **kw)
        q1 = lg.dock_batch(L, G, batching="queue", **kw)
        q2 = lg.dock_batch(L, G, batching="queue", **kw)     # graph replay
        torch.cuda.synchronize()
        for name in ("trace", "scores", "poses", "top_restart", "status"):
            assert torch.equal(getattr(plain, name), getattr(q1, name)), name
            assert torch.equal(getattr(q1, name), getattr(q2, name)), name


@pytest.mark.parametrize("lanes,rpc", [(16, 8), (32, 4)])
def test_wide_lane_shapes_match_plain(lg, bimodal, lanes, rpc):
    """16 and 32 lanes per restart (a gather request covers consecutive
    increments of one atom of one restart): the same decisions as the
    default 8-lane shape."""
    w, lib, grid = bimodal
    L, G = _dev(lg, lib, grid)
    saved = lg.tune_get()
    try:
        for fmt in ("f32", "f16"):
            kw = _kw(w["search"], trace=True, top_restart=True, grid_format=fmt)
            plain = lg.dock_batch(L, G, batching="plain", **kw)
            lg.tune_set({b: (lanes, rpc) for b in range(44)})
            wide = lg.dock_batch(L, G, batching="buckets_static", **kw)
            torch.cuda.synchronize()
            _same_decisions_close_scores(plain, wide)
    finally:
        lg.tune_set(saved)


@pytest.mark.parametrize("fmt", ["f32", "f16"])
def test_static_bucket_launches_match_plain(lg, bimodal, small32, fmt):
    for w, lib, grid in (bimodal, small32):
        L, G = _dev(lg, lib, grid)
        kw = _kw(w["search"], trace=True, top_restart=True, grid_format=fmt)
        plain = lg.dock_batch(L, G, batching="plain", **kw)
        st1 = lg.dock_batch(L, G, batching="buckets_static", **kw)
        st2 = lg.dock_batch(L, G, batching="buckets_static", **kw)     # graph replay
        torch.cuda.synchronize()
        _same_decisions_close_scores(plain, st1)
        assert torch.equal(st1.scores, st2.scores) and torch.equal(st1.trace, st2.trace)


def test_buckets_with_mixed_shapes_after_tuning(lg, bimodal):
    w, lib, grid = bimodal
    L, G = _dev(lg, lib, grid)
    kw = _kw(w["search"], trace=True, top_restart=True)
    saved = lg.tune_get()
    try:
        # one shape per atom class, different from the default
        table = {b: ((4, 32) if (b // 11) % 2 == 0 else (8, 8)) for b in range(44)}
        lg.tune_set(table)
        assert lg.tune_get()[0] == (4, 32) and lg.tune_get()[11] == (8, 8)
        plain = lg.dock_batch(L, G, batching="plain", **kw)
        mixed = lg.dock_batch(L, G, batching="buckets", **kw)
        torch.cuda.synchronize()
        _same_decisions_close_scores(plain, mixed)
        tuned = lg.autotune(L, G, sample=64, **_kw(w["search"]))
        present = {int(b) for b in lg.pack_ligands(L, grid.dims[3])[2].cpu().numpy()}
        assert set(tuned) == present
        for lanes, rpc, ms in tuned.values():
            assert lanes in (2, 4, 8, 16, 32) and rpc * lanes <= 128 and ms > 0
        after = lg.dock_batch(L, G, batching="buckets", **kw)
        torch.cuda.synchronize()
        _same_decisions_close_scores(plain, after)
    finally:
        lg.tune_set(saved)


def test_buckets_on_default_stream_and_host_memory(lg, small32):
    w, lib, grid = small32
    kw = _kw(w["search"], trace=True)
    L, G = _dev(lg, lib, grid)
    ref = lg.dock_batch(L, G, batching="plain", **kw)
    with torch.cuda.stream(torch.cuda.default_stream()):
        d = lg.dock_batch(L, G, batching="buckets", **kw)       # legacy stream: no graph
    torch.cuda.synchronize()
    _same_decisions_close_scores(ref, d)
    Lh = lg.Ligands.from_arrays(lib, "cpu", pin=True)
    Gh = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cpu", pin=True)
    h = lg.dock_batch(Lh, Gh, batching="buckets", **kw)
    assert torch.equal(h.trace, d.trace.cpu())


def test_buckets_bimodal_sample_matches_oracle(lg, oracle_lib, bimodal):
    w, lib, grid = bimodal
    s = w["search"]
    L, G = _dev(lg, lib, grid)
    R = s["restarts"]
    res = lg.dock_batch(L, G, batching="buckets", **_kw(s, top_k=R, trace=True, top_restart=True))
    torch.cuda.synchronize()
    trace = res.trace.cpu().numpy()
    scores = res.scores.cpu().numpy()
    top = res.top_restart.cpu().numpy()
    small = [l for l in range(lib.n_ligands) if lib.n_atoms[l] <= 35][:6]
    large = [l for l in range(lib.n_ligands) if lib.n_atoms[l] >= 60][:3]
    ref = oracle_lib.dock_library(lib, grid, s, ligands=small + large, restarts=range(0, 6))
    tot = parity.new_stats()
    for r_ in ref:
        l = r_["ligand"]
        gt = parity.ligand_trace(trace, lib.rot_off, R, s["passes"], l)
        final = {int(top[l, k]): float(scores[l, k]) for k in range(R)}
        st = parity.check_dock_ligand(l, r_, gt, final)
        parity.merge(tot, st)
    print(tot)
    assert tot["clean"] >= 0.9 * tot["restarts"] and tot["scores"] > 0
