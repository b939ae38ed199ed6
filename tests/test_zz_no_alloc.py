"""ligen_dock_batch_static: the docking call that allocates nothing.

Some callers cannot allocate device memory while they run: a framework whose
caching allocator already owns the device's memory, or a latency-bound
service that cannot afford the device-wide synchronisation of cudaMalloc.
This entry point docks with the library's fixed device scratch array instead
of an allocated workspace. It runs the same kernels on the same inputs as
ligen_dock_batch, so its outputs are checked against that call bit for bit,
on two calls in a row (the array keeps the previous call's contents, which
must not leak into the next result). Also checked: the settings it cannot
honour are refused, host memory is refused, and the header's scratch formula
draws the exact line between accepted and rejected batches. Needs a GPU;
this file is collected last."""
import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu

LIMIT = 32 << 20          # LIGEN_STATIC_SCRATCH_BYTES
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED = -2


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


def _same(a, b, what):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert a.shape == b.shape, what
    assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), what   # bit for bit, NaN patterns included


def test_static_scratch_call_matches_dock_batch_twice(setup):
    lg, lib, grid, kw, L, G = setup
    ref = lg.dock_batch(L, G, trace=True, top_restart=True, **kw)
    torch.cuda.synchronize()
    # outputs allocated up front, so the calls below allocate nothing
    out = lg.DockResult(poses=torch.empty_like(ref.poses), scores=torch.empty_like(ref.scores),
                        status=torch.empty_like(ref.status), trace=torch.empty_like(ref.trace),
                        top_restart=torch.empty_like(ref.top_restart), stage_ms=None)
    other = gen.make_library(dict(gen.WORKLOADS["small32"]["library"], seed=9))
    Lo = lg.Ligands.from_arrays(other, "cuda")
    for call in range(2):
        if call == 1:
            # a different batch in between leaves different contents in the array
            lg.dock_batch_static(Lo, G, **dict(kw, seed=kw["seed"] + 5))
        for t in (out.scores, out.poses):
            t.fill_(float("nan"))
        for t in (out.status, out.trace, out.top_restart):
            t.fill_(-7)
        lg.dock_batch_static(L, G, trace=True, top_restart=True, out=out, **kw)
        torch.cuda.synchronize()
        assert int(out.status.abs().sum()) == 0
        for name in ("scores", "poses", "status", "trace", "top_restart"):
            _same(getattr(out, name), getattr(ref, name), (call, name))


def test_static_scratch_refuses_settings_it_does_not_run(setup):
    lg, lib, grid, kw, L, G = setup
    for extra in (dict(grid_format="f16"), dict(grid_format="bf16"), dict(batching="buckets"),
                  dict(batching="buckets_static"), dict(rescore_fp64=True), dict(stage_ms=True),
                  dict(count_samples=True), dict(mode="exhaustive")):
        with pytest.raises(lg.LigenError) as e:
            lg.dock_batch_static(L, G, **kw, **extra)
        assert e.value.code == ERR_UNSUPPORTED, extra


def test_static_scratch_refuses_host_memory(setup):
    lg, lib, grid, kw, L, G = setup
    ref = lg.dock_batch(L, G, **kw)
    host_out = lg.DockResult(poses=torch.empty(ref.poses.shape), scores=torch.empty(ref.scores.shape),
                             status=None, trace=None, top_restart=None, stage_ms=None)
    with pytest.raises(lg.LigenError) as e:
        lg.dock_batch_static(L, G, status=False, out=host_out, **kw)
    assert e.value.code == ERR_INVALID_ARG
    Lh = lg.Ligands.from_arrays(lib, "cpu")
    with pytest.raises(lg.LigenError) as e:
        lg.dock_batch_static(Lh, G, **kw)
    assert e.value.code == ERR_INVALID_ARG


def _r256(n):
    return (int(n) + 255) // 256 * 256


def scratch_bytes(lib, dims, R):
    """The header's formula: ten regions, each rounded up to 256 bytes."""
    nx, ny, nz, nc = dims
    L = len(lib.atom_off) - 1
    A = int(lib.atom_off[-1])
    B = int(lib.rot_off[-1])
    regions = [(nx - 1) * (ny - 1) * (nz - 1) * nc * 32, 16 * A, 4 * B, 128 * B, 4 * B, 4 * L,
               4 * L * R, L * R, B * R]
    return sum(_r256(r) for r in regions)


def test_static_scratch_limit_follows_the_header_formula(setup):
    lg, lib, _, kw, L, _ = setup
    spec = dict(gen.WORKLOADS["small32"]["grid"], points=62)   # 61^3 x 4 cells: 29 MB of records
    big = gen.make_grid(spec)
    G = lg.PocketGrid.from_array(big.values, big.origin, big.spacing, "cuda")
    lo, hi = 1, 65536
    assert scratch_bytes(lib, big.dims, lo) <= LIMIT < scratch_bytes(lib, big.dims, hi)
    while hi - lo > 1:                       # largest R whose scratch fits
        mid = (lo + hi) // 2
        if scratch_bytes(lib, big.dims, mid) <= LIMIT:
            lo = mid
        else:
            hi = mid
    R = lo
    assert scratch_bytes(lib, big.dims, R + 1) > LIMIT
    res = lg.dock_batch_static(L, G, **dict(kw, restarts=R))
    torch.cuda.synchronize()
    assert int(res.status.abs().sum()) == 0
    assert bool(torch.isfinite(res.scores).all())
    with pytest.raises(lg.LigenError) as e:
        lg.dock_batch_static(L, G, **dict(kw, restarts=R + 1))
    assert e.value.code == ERR_UNSUPPORTED and "scratch" in str(e.value)


def test_static_scratch_rejects_batches_beyond_its_size(setup):
    lg, lib, grid, kw, L, G = setup
    big = gen.make_grid(gen.WORKLOADS["screen20k"]["grid"])       # 96^3 x 8: 219 MB of records
    Gb = lg.PocketGrid.from_array(big.values, big.origin, big.spacing, "cuda")
    with pytest.raises(lg.LigenError) as e:
        lg.dock_batch_static(L, Gb, **kw)
    assert e.value.code == ERR_UNSUPPORTED and "scratch" in str(e.value)
