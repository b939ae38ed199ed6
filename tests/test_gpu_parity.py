"""CUDA path vs the oracle on the same seeded inputs (needs a GPU)."""
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


def _dev(lg, lib, grid, device="cuda"):
    return (lg.Ligands.from_arrays(lib, device),
            lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, device))


def _bad_ligands():
    xyz = np.array([[0, 0, 0], [1.5, 0, 0], [2, 1.4, 0], [3.5, 1.4, 0]], float)
    good = dict(xyz=xyz, type=np.array([0, 1, 2, 3], np.uint8), bonds=np.array([[0, 1], [1, 2], [2, 3]]),
                rot_edge=np.array([1], np.int32))
    cycle = dict(good, bonds=np.array([[0, 1], [1, 2], [2, 0]]))
    rng_id = dict(good, bonds=np.array([[0, 1], [1, 2], [2, 7]]))
    rot_rng = dict(good, rot_edge=np.array([5], np.int32))
    typ = dict(good, type=np.array([0, 1, 2, 9], np.uint8))
    dup = dict(good, bonds=np.array([[0, 1], [0, 1], [2, 3]]))
    return [good, cycle, rng_id, rot_rng, typ, dup], [0, 1, 1, 1, 1, 1]


# ------------------------------------------------------------- packer ---
@pytest.mark.parametrize("which", ["small32", "screen64", "screen64_shuffled", "bad"])
def test_packer_bit_exact(lg, oracle_lib, small32, screen_sample, which):
    if which == "small32":
        _, lib, grid = small32
        nc = 4
    elif which == "bad":
        ligs, _ = _bad_ligands()
        lib = gen.from_ligands(ligs)
        nc = 4
    else:
        _, lib, grid = screen_sample
        nc = 8
        if which.endswith("shuffled"):
            lib = gen.shuffle_bonds(lib, 3)
    L = lg.Ligands.from_arrays(lib, "cuda")
    bits, axis, bucket, status = (t.cpu().numpy() for t in lg.pack_ligands(L, nc))
    for l in range(lib.n_ligands):
        g = lib.ligand(l)
        lig = oracle_lib.OLigand(g["xyz"], g["type"], g["bonds"], g["rot_edge"])
        bad = oracle_lib.validate(lig, nc)
        assert status[l] == (-6 if bad else 0), l
        assert bucket[l] == oracle_lib.bucket_id(lig.n_atoms, lig.n_rot)
        if bad:
            continue
        _, mask, ax = oracle_lib.fragments(lig)
        r0, r1 = lib.rot_off[l], lib.rot_off[l + 1]
        assert np.array_equal(parity.unpack_bits(bits[r0:r1], lig.n_atoms), mask), l
        assert np.array_equal(axis[r0:r1], ax), l


@pytest.mark.parametrize("which", ["small32", "screen64", "bad"])
def test_touch_masks_bit_exact(lg, oracle_lib, small32, screen_sample, which):
    """Bond interaction masks, against their definition on the oracle's
    fragments: bit b of bond b' is set when b' moves (its moving side minus
    its own v) an atom of b's moving side or b's fixed end; always for b = b'."""
    if which == "bad":
        ligs, _ = _bad_ligands()
        lib, nc = gen.from_ligands(ligs), 4
    else:
        _, lib, _ = small32 if which == "small32" else screen_sample
        nc = 4 if which == "small32" else 8
    L = lg.Ligands.from_arrays(lib, "cuda")
    touch = lg.pack_touch(L, nc).cpu().numpy()
    for l in range(lib.n_ligands):
        g = lib.ligand(l)
        lig = oracle_lib.OLigand(g["xyz"], g["type"], g["bonds"], g["rot_edge"])
        r0, n = lib.rot_off[l], lib.n_rot[l]
        if oracle_lib.validate(lig, nc):
            assert np.all(touch[r0:r0 + n] == 0)
            continue
        _, mask, axis = oracle_lib.fragments(lig)
        mask = mask.reshape(n, -1).astype(bool)
        for bp in range(n):
            moved = mask[bp].copy()
            moved[axis[bp][1]] = False
            want = 0
            for b in range(n):
                reads = mask[b].copy()
                reads[axis[b][0]] = True
                if b == bp or np.any(moved & reads):
                    want |= 1 << b
            assert int(touch[r0 + bp]) == want, (l, bp)


# ------------------------------------------------------------ scoring ---
def _random_poses(rng, lib, grid, K):
    out = []
    for l in range(lib.n_ligands):
        n = lib.n_rot[l]
        for _ in range(K):
            q = rng.normal(size=4)
            out.append(np.concatenate([grid.center + rng.uniform(-4, 4, 3), q, rng.uniform(-np.pi, np.pi, n)]))
    return np.concatenate(out)


@pytest.mark.parametrize("K", [8, 40])       # a lane group per pose / a lane per pose, 2 warps per ligand
@pytest.mark.parametrize("which", ["small32", "screen64"])
def test_score_poses_within_1e5(lg, oracle_lib, small32, screen_sample, which, K):
    w, lib, grid = small32 if which == "small32" else screen_sample
    rng = np.random.default_rng(11)
    poses = _random_poses(rng, lib, grid, K)
    Ld, Gd = _dev(lg, lib, grid)
    out = lg.score_poses(Ld, Gd, torch.tensor(poses, dtype=torch.float32, device="cuda"), K).cpu().numpy()
    og = oracle_lib.OGrid.from_grid(grid)
    off = lg.pose_offsets(lib.rot_off, K)
    worst = 0.0
    bare = []
    for l in range(lib.n_ligands):
        lig = oracle_lib.OLigand.from_library(lib, l)
        P = poses[off[l]:off[l + 1]].astype(np.float32).astype(np.float64).reshape(K, -1)
        for p in range(K):
            S, D, _, Gs = oracle_lib.score_pose(lig, og, P[p], 5.0, sensitivity=True)
            err = abs(out[l, p] - S)
            worst = max(worst, err / parity.score_tol(D, Gs))
            bare.append(parity.bare_ratio(err, D))
            assert err <= parity.score_tol(D, Gs), (l, p, out[l, p], S, D, Gs)
    bare = np.array(bare)
    print(f"worst score error as a fraction of the tolerance {worst:.2e}; within the bare 1e-5 D: "
          f"{np.mean(bare <= 1.0):.4f} of {len(bare)} poses, worst {bare.max():.2f} x 1e-5 D")


@pytest.mark.parametrize("K", [8, 30, 33])
def test_prepared_scoring_equals_score_poses(lg, screen_sample, K):
    """ligen_score_prepared runs the scoring kernels of ligen_score_poses on
    inputs prepared once: bit-identical scores, call after call, from device
    or host poses."""
    w, lib, grid = screen_sample
    rng = np.random.default_rng(12)
    poses = torch.tensor(_random_poses(rng, lib, grid, K), dtype=torch.float32, device="cuda")
    Ld, Gd = _dev(lg, lib, grid)
    ref = lg.score_poses(Ld, Gd, poses, K)
    prep = lg.prepare_scoring(Ld, Gd)
    for _ in range(2):
        got = prep.score(poses, K)
        assert torch.equal(got, ref)
    host = prep.score(poses.cpu(), K)
    assert host.device.type == "cpu" and torch.equal(host, ref.cpu())
    Lh = lg.Ligands.from_arrays(lib, "cpu")
    Gh = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cpu")
    prep_h = lg.prepare_scoring(Lh, Gh)        # host inputs, copied in and released by the call
    assert torch.equal(prep_h.score(poses, K), ref)
    prep.release()
    prep_h.release()
    with pytest.raises(ValueError):
        prep.score(poses, K)


def test_scoring_graph_paths_agree(lg, screen_sample):
    """The class launches of pose-per-lane scoring replay from a cached CUDA
    graph: captured on a side stream for the legacy default stream and
    launched on it, captured directly on a user stream, and inside a
    caller's own capture issued into that graph. Every path, first call and replay, gives the
    same scores, and work queued before and after on the calling stream is
    ordered around it."""
    w, lib, grid = screen_sample
    K = 30
    rng = np.random.default_rng(21)
    poses = torch.tensor(_random_poses(rng, lib, grid, K), dtype=torch.float32, device="cuda")
    Ld, Gd = _dev(lg, lib, grid)
    prep = lg.prepare_scoring(Ld, Gd)
    ref = prep.score(poses, K)                      # default stream, first call: captured
    assert torch.equal(prep.score(poses, K), ref)   # replayed
    from paper_2303_06150_gb300 import api
    dev = torch.device("cuda", torch.cuda.current_device())
    assert (api._stream_handle(dev).value or 0) == torch.cuda.current_stream().cuda_stream
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        assert api._stream_handle(dev).value == side.cuda_stream          # the binding passes the current stream
        assert api._stream_handle(torch.device("cuda")).value == side.cuda_stream
        outs = [torch.full_like(ref, 7.0) for _ in range(3)]
        for o in outs:
            prep.score(poses, K, out=o)               # user stream: captured on it, then replayed
        shifted = outs[-1] + 1.0                      # ordered after the scoring on `side`
    torch.cuda.current_stream().wait_stream(side)
    for o in outs:
        assert torch.equal(o, ref)
    assert torch.equal(shifted, ref + 1.0)
    cap = torch.full_like(ref, 7.0)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):                          # the caller's own capture
        prep.score(poses, K, out=cap)
    cap.fill_(7.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(cap, ref)
    # releasing the workspaces frees the cached graphs and side streams; the
    # next calls recreate them, and the caller's own graph still replays
    lg.release_workspaces()
    assert torch.equal(prep.score(poses, K), ref)
    cap.fill_(7.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(cap, ref)
    del g
    prep.release()


# ------------------------------------------------------------ docking ---
def _dock_and_compare(lg, oracle_lib, w, lib, grid, restarts=None, ligands=None, device="cuda", fmt="f32"):
    s = dict(w["search"])
    R = s["restarts"]
    Ld, Gd = _dev(lg, lib, grid, device)
    res = lg.dock_batch(Ld, Gd, restarts=R, torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
                        top_k=R, seed=s["seed"], n_rigid=s.get("n_rigid", 24), trace=True, top_restart=True,
                        grid_format=fmt)
    if device == "cuda":
        torch.cuda.synchronize()
    trace = res.trace.cpu().numpy()
    scores = res.scores.cpu().numpy()
    top = res.top_restart.cpu().numpy()
    status = res.status.cpu().numpy()
    ref = oracle_lib.dock_library(lib, parity.oracle_grid(oracle_lib, grid, fmt), s, ligands=ligands,
                                  restarts=restarts)
    tot = parity.new_stats()
    for r_ in ref:
        l = r_["ligand"]
        assert status[l] == 0
        gt = parity.ligand_trace(trace, lib.rot_off, R, s["passes"], l)
        final = {int(top[l, k]): float(scores[l, k]) for k in range(R)}
        st = parity.check_dock_ligand(l, r_, gt, final)
        parity.merge(tot, st)
        # ranking: scores sorted, ties by restart index, every restart once
        assert np.all(np.diff(scores[l]) <= 0)
        assert sorted(top[l].tolist()) == list(range(R))
    return res, ref, tot


# 16-bit records are compared with the oracle run on their rounded node
# values (parity.oracle_grid): same decisions, scores within the FP32 bar.
@pytest.mark.parametrize("fmt", ["f32", "f16", "bf16"])
def test_dock_small32_matches_oracle(lg, oracle_lib, small32, fmt):
    w, lib, grid = small32
    _, _, tot = _dock_and_compare(lg, oracle_lib, w, lib, grid, fmt=fmt)
    print(tot)
    assert tot["clean"] >= 0.9 * tot["restarts"] and tot["scores"] > 0


@pytest.mark.parametrize("fmt", ["f32", "f16", "bf16"])
def test_dock_screen_sample_matches_oracle(lg, oracle_lib, screen_sample, fmt):
    w, lib, grid = screen_sample
    _, _, tot = _dock_and_compare(lg, oracle_lib, w, lib, grid, restarts=range(0, 24),
                                  ligands=range(0, 64, 2), fmt=fmt)
    print(tot)
    assert tot["clean"] >= 0.9 * tot["restarts"] and tot["scores"] > 0


@pytest.mark.parametrize("which", ["small32", "screen64"])
def test_docking_coordinates_within_pos_ulps(lg, oracle_lib, small32, screen_sample, which):
    """The position term of the score tolerance, measured: the docking
    kernel's final FP32 atom positions (grid units, the debug `coords`
    output) against the oracle's FP64 positions of the same final pose, on
    every restart whose trajectory equals the oracle's. The error of atom i
    in units of 2^-24 |u_i| (u_i its grid-unit distance from the origin)
    must stay within parity.POS_ULPS."""
    w, lib, grid = small32 if which == "small32" else screen_sample
    s = dict(w["search"])
    R = s["restarts"]
    rr = None if which == "small32" else range(0, 16)
    Ld, Gd = _dev(lg, lib, grid)
    res = lg.dock_batch(Ld, Gd, restarts=R, torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
                        top_k=R, seed=s["seed"], n_rigid=s.get("n_rigid", 24), trace=True, coords=True)
    trace = res.trace.cpu().numpy()
    coords = res.coords.cpu().numpy()
    ref = oracle_lib.dock_library(lib, grid, s, restarts=rr)
    origin, h = np.asarray(grid.origin, np.float64), float(grid.spacing)
    ulps, restarts = [], 0
    for r_ in ref:
        l = r_["ligand"]
        N, a0 = int(lib.n_atoms[l]), int(lib.atom_off[l])
        gt = parity.ligand_trace(trace, lib.rot_off, R, s["passes"], l)
        lig = oracle_lib.OLigand.from_library(lib, l)
        for j, r in enumerate(r_["restarts"]):
            if not np.array_equal(gt[r], r_["trace"][j]):
                continue          # a near-tie went the other (valid) way: another pose
            u_ref = (oracle_lib.pose_coords(lig, r_["pose"][j]) - origin) / h
            base = 3 * (R * a0 + int(r) * N)
            ulps.append(parity.coord_ulps(coords[base:base + 3 * N].reshape(N, 3), u_ref))
            restarts += 1
    ulps = np.concatenate(ulps)
    q = np.quantile(ulps, [0.5, 0.99, 0.999])
    print(f"{which}: {restarts} restarts, {len(ulps)} atom positions; error in units of 2^-24 |u|: median "
          f"{q[0]:.2f}, 99% {q[1]:.2f}, 99.9% {q[2]:.2f}, max {ulps.max():.2f} (POS_ULPS {parity.POS_ULPS})")
    assert restarts > 0.9 * sum(len(r_["restarts"]) for r_ in ref)
    assert ulps.max() <= parity.POS_ULPS


def test_restart_initial_poses_match_oracle(lg, oracle_lib, small32):
    """Restart initialisation on its own: with one rigid candidate (the
    identity) and no sweep pass, every restart's pose is its initial one,
    the Shoemake quaternion and jittered translation of the counter hash."""
    w, lib, grid = small32
    s = dict(w["search"], restarts=8, top_k=8, n_rigid=1, passes=0)
    Ld, Gd = _dev(lg, lib, grid)
    res = lg.dock_batch(Ld, Gd, restarts=8, torsion_step_deg=s["torsion_step_deg"], passes=0, top_k=8,
                        seed=s["seed"], n_rigid=1, jitter=s["jitter"], top_restart=True)
    torch.cuda.synchronize()
    poses = res.poses.cpu().numpy()
    top = res.top_restart.cpu().numpy()
    og = oracle_lib.OGrid.from_grid(grid)
    off = lg.pose_offsets(lib.rot_off, 8)
    for l in range(lib.n_ligands):
        P = poses[off[l]:off[l + 1]].reshape(8, -1)
        assert np.all(P[:, 7:] == 0)                          # torsions untouched
        for k in range(8):
            q, t = oracle_lib.restart_init(og, s, l, int(top[l, k]))
            q = q * (1.0 if q[0] >= 0 else -1.0)
            np.testing.assert_allclose(P[k, :3], t, atol=4e-6, rtol=0)    # FP32 at ~10 A
            np.testing.assert_allclose(P[k, 3:7], q, atol=1e-6, rtol=0)
    # with the 24 cube rotations, the kept orientation is q_r (x) g_k (body
    # frame) for the rotation k the restart chose
    res = lg.dock_batch(Ld, Gd, restarts=8, torsion_step_deg=s["torsion_step_deg"], passes=0, top_k=8,
                        seed=s["seed"], n_rigid=24, jitter=s["jitter"], top_restart=True, trace=True)
    torch.cuda.synchronize()
    poses = res.poses.cpu().numpy()
    top = res.top_restart.cpu().numpy()
    trace = res.trace.cpu().numpy()
    for l in range(lib.n_ligands):
        P = poses[off[l]:off[l + 1]].reshape(8, -1)
        tr = parity.ligand_trace(trace, lib.rot_off, 8, 0, l)
        for k in range(8):
            r = int(top[l, k])
            qr, _ = oracle_lib.restart_init(og, s, l, r)
            q = oracle_lib.quat_mul(qr, oracle_lib.octahedral(int(tr[r, 0])))
            q = q / np.linalg.norm(q) * (1.0 if q[0] >= 0 else -1.0)
            np.testing.assert_allclose(P[k, 3:7], q, atol=1e-6, rtol=0)


def test_dock_top_k_and_poses(lg, oracle_lib, small32):
    w, lib, grid = small32
    s = w["search"]
    Ld, Gd = _dev(lg, lib, grid)
    full = lg.dock_batch(Ld, Gd, restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"],
                         passes=s["passes"], top_k=s["restarts"], seed=s["seed"], top_restart=True, trace=True)
    trace = full.trace.cpu().numpy()
    kept = lg.dock_batch(Ld, Gd, restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"],
                         passes=s["passes"], top_k=s["top_k"], seed=s["seed"], top_restart=True)
    K = s["top_k"]
    assert torch.equal(full.scores[:, :K], kept.scores)
    assert torch.equal(full.top_restart[:, :K], kept.top_restart)
    # kept poses re-score to the reported scores (same FP32 path, different route)
    rescored = lg.score_poses(Ld, Gd, kept.poses, K).cpu().numpy()
    sc = kept.scores.cpu().numpy()
    og = oracle_lib.OGrid.from_grid(grid)
    poses = kept.poses.cpu().numpy()
    off = lg.pose_offsets(lib.rot_off, K)
    ref = oracle_lib.dock_library(lib, grid, s)
    for l in range(lib.n_ligands):
        lig = oracle_lib.OLigand.from_library(lib, l)
        P = poses[off[l]:off[l + 1]].reshape(K, -1)
        for k in range(K):
            S, D, _, Gs = oracle_lib.score_pose(lig, og, P[k].astype(np.float64), 5.0, sensitivity=True)
            assert abs(rescored[l, k] - sc[l, k]) <= parity.score_tol(D, Gs)
            assert abs(S - sc[l, k]) <= parity.score_tol(D, Gs)
            assert P[k, 3] >= 0 and abs(np.linalg.norm(P[k, 3:7]) - 1) < 1e-6
            assert np.all(np.abs(P[k, 7:]) <= np.pi + 1e-6)
        # where the oracle's top-K is separated by more than the gap tolerance,
        # the kept restarts and their poses agree
        r_ = ref[l]
        gt = parity.ligand_trace(trace, lib.rot_off, s["restarts"], s["passes"], l)
        if all(parity.clean_restart(r_, j, gt[j]) for j in range(len(r_["score"]))):
            os_ = np.sort(r_["score"])[::-1]
            tol = parity.gap_tol(r_["dnorm"][:, -1].max(), r_["gsens"][:, -1].max())
            for k in range(K):
                sep = (k == 0 or os_[k - 1] - os_[k] > tol) and (os_[k] - os_[k + 1] > tol
                                                                 if k + 1 < len(os_) else True)
                if sep:
                    assert kept.top_restart[l, k].item() == r_["top_restart"][k]
                    np.testing.assert_allclose(P[k], r_["top_pose"][k], atol=2e-5)


@pytest.mark.parametrize("variant", ["ragged_R13", "step5_chunked", "passes0", "rigid7", "step45"])
def test_dock_search_variants(lg, oracle_lib, small32, variant):
    w, lib, grid = small32
    w = dict(w, search=dict(w["search"]))
    s = w["search"]
    if variant == "ragged_R13":
        s["restarts"] = 13
    elif variant == "step5_chunked":
        s["torsion_step_deg"] = 5
        s["passes"] = 1
    elif variant == "passes0":
        s["passes"] = 0
    elif variant == "rigid7":
        s["n_rigid"] = 7
    elif variant == "step45":
        s["torsion_step_deg"] = 45
    sub = lib.subset(range(0, 32, 4))
    _, _, tot = _dock_and_compare(lg, oracle_lib, w, sub, grid)
    assert tot["restarts"] > 0 and tot["clean"] >= 0.9 * tot["restarts"]


def test_dock_edge_ligands(lg, oracle_lib, small32):
    """Single atom, rigid (no rotatable bond), terminal-bond torsion, 256 atoms / 32 bonds."""
    w, lib, grid = small32
    one = dict(xyz=np.zeros((1, 3)), type=np.zeros(1, np.uint8), bonds=np.zeros((0, 2), np.int32),
               rot_edge=np.zeros(0, np.int32))
    rigid = dict(lib.ligand(0), rot_edge=np.zeros(0, np.int32))
    term = dict(lib.ligand(1))
    term["rot_edge"] = np.array([len(term["bonds"]) - 1], np.int32)   # last atom is a leaf
    big_lib = gen.make_library(dict(kind="uniform", n_ligands=1, n_atoms=(256, 256), n_rot=(32, 32),
                                    n_types=4, seed=5))
    big = big_lib.ligand(0)
    ligs = [one, rigid, term, big]
    sub = gen.from_ligands(ligs)
    assert sub.n_atoms.max() == 256 and sub.n_rot.max() >= 24
    w2 = dict(w, search=dict(w["search"], passes=1))
    _, _, tot = _dock_and_compare(lg, oracle_lib, w2, sub, grid)
    assert tot["restarts"] == 4 * w["search"]["restarts"]


def test_bad_ligands_do_not_fail_the_batch(lg, small32):
    w, lib, grid = small32
    ligs, bad = _bad_ligands()
    mixed = gen.from_ligands([lib.ligand(0)] + ligs + [lib.ligand(1)])
    s = w["search"]
    Ld, Gd = _dev(lg, mixed, grid)
    res = lg.dock_batch(Ld, Gd, restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"],
                        passes=s["passes"], top_k=s["top_k"], seed=s["seed"])
    st = res.status.cpu().numpy()
    assert st.tolist() == [0] + [-6 * b for b in bad] + [0]
    sc = res.scores.cpu().numpy()
    for i, b in enumerate([0] + bad + [0]):
        assert np.all(np.isneginf(sc[i])) == bool(b)
    # a good ligand docks the same alone and inside the mixed batch
    alone = lg.dock_batch(*_dev(lg, lib.subset([0]), grid), restarts=s["restarts"],
                          torsion_step_deg=s["torsion_step_deg"], passes=s["passes"], top_k=s["top_k"],
                          seed=s["seed"])
    assert torch.equal(alone.scores[0], res.scores[0])


def test_empty_library(lg, small32):
    w, lib, grid = small32
    empty = gen.from_ligands([])
    Ld, Gd = _dev(lg, empty, grid)
    s = w["search"]
    res = lg.dock_batch(Ld, Gd, restarts=8, torsion_step_deg=30, passes=2, top_k=4, seed=0)
    assert res.scores.numel() == 0


def test_host_memory_path_equals_device_path(lg, small32):
    w, lib, grid = small32
    s = w["search"]
    kw = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
              top_k=s["top_k"], seed=s["seed"], trace=True)
    dev = lg.dock_batch(*_dev(lg, lib, grid, "cuda"), **kw)
    host = lg.dock_batch(lg.Ligands.from_arrays(lib, "cpu", pin=True),
                         lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cpu", pin=True), **kw)
    assert host.scores.device.type == "cpu"
    assert torch.equal(dev.scores.cpu(), host.scores)
    assert torch.equal(dev.poses.cpu(), host.poses)
    assert torch.equal(dev.trace.cpu(), host.trace)


def test_side_stream_and_determinism(lg, small32):
    w, lib, grid = small32
    s = w["search"]
    Ld, Gd = _dev(lg, lib, grid)
    kw = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
              top_k=s["top_k"], seed=s["seed"])
    a = lg.dock_batch(Ld, Gd, **kw)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b = lg.dock_batch(Ld, Gd, **kw)
    st.synchronize()
    assert torch.equal(a.scores, b.scores) and torch.equal(a.poses, b.poses)
    c = lg.dock_batch(Ld, Gd, **dict(kw, seed=s["seed"] + 1))
    assert not torch.equal(a.scores, c.scores)


def test_bucket_size_eq1(lg):
    for max_atoms in (32, 64, 128, 256):
        f = lg.bucket_size(max_atoms)
        assert f["b"] >= 1 and f["sm"] > 0 and f["ws"] == 32
        assert f["l"] == f["b"] * f["sm"] * f["t"] // f["ws"]
    assert lg.bucket_size(32)["b"] >= lg.bucket_size(256)["b"]


@pytest.mark.parametrize("fmt, restarts", [("f32", 8), ("f16", 8), ("f32", 300)])
def test_zero_field_ties_take_the_lowest_index(lg, oracle_lib, small32, fmt, restarts):
    """Degenerate case: on a zero field every candidate of every stage scores
    exactly 0 on both sides, so every decision is an exact tie and the lowest
    index must win (k = 0, j = 0), the kept poses are restarts 0..K-1 in
    order, and each pose is the restart's initial pose (the oracle's).
    300 restarts exceed what the top-K keeps in registers (256)."""
    w, lib, _ = small32
    s = dict(w["search"], restarts=restarts, top_k=min(restarts, 40))
    zero = np.zeros((41, 41, 41, 4))
    L = lg.Ligands.from_arrays(lib, "cuda")
    G = lg.PocketGrid.from_array(zero, (0.0, 0.0, 0.0), 1.0, "cuda")
    res = lg.dock_batch(L, G, restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
                        top_k=s["top_k"], seed=s["seed"], trace=True, top_restart=True, grid_format=fmt)
    torch.cuda.synchronize()
    assert torch.all(res.trace == 0) and torch.all(res.scores == 0)
    K = s["top_k"]
    assert torch.equal(res.top_restart.cpu(), torch.arange(K, dtype=torch.int32).repeat(lib.n_ligands, 1))
    og = oracle_lib.OGrid(zero, (0.0, 0.0, 0.0), 1.0)
    poses = res.poses.cpu().numpy()
    off = lg.pose_offsets(lib.rot_off, K)
    for l in range(lib.n_ligands):
        lig = oracle_lib.OLigand.from_library(lib, l)
        ref = oracle_lib.dock_ligand(lig, og, s, l, range(0, K))
        assert np.all(ref["trace"] == 0)
        np.testing.assert_allclose(poses[off[l]:off[l + 1]].reshape(K, -1), ref["pose"], atol=1e-5)


@pytest.mark.parametrize("restarts", [200, 300])
def test_top_k_total_order_both_paths(lg, small32, restarts):
    """All R restarts kept (K = R): every restart once, scores non-increasing,
    equal scores in ascending restart order; a smaller K is the prefix. 200
    restarts rank in registers, 300 from memory."""
    w, lib, grid = small32
    s = w["search"]
    L, G = _dev(lg, lib, grid)
    kw = dict(restarts=restarts, torsion_step_deg=s["torsion_step_deg"], passes=s["passes"], seed=s["seed"],
              top_restart=True)
    full = lg.dock_batch(L, G, top_k=restarts, **kw)
    part = lg.dock_batch(L, G, top_k=30, **kw)
    torch.cuda.synchronize()
    sc, top = full.scores.cpu().numpy(), full.top_restart.cpu().numpy()
    for l in range(lib.n_ligands):
        assert sorted(top[l].tolist()) == list(range(restarts))
        assert np.all(np.diff(sc[l]) <= 0)
        eq = np.diff(sc[l]) == 0
        assert np.all(np.diff(top[l])[eq] > 0)
    assert torch.equal(part.scores, full.scores[:, :30]) and torch.equal(part.top_restart, full.top_restart[:, :30])


def test_sample_count_follows_the_clean_bond_rule(lg, small32, screen_sample):
    """The kernel's count of needed samples equals the count replayed from
    its own decisions: per restart n_rigid * N, plus (n_theta - 1) * (moving
    atoms - 1) for each decision of a bond that was not clean. A bond is
    clean after its own sweep (kept or turned), until a turn of another bond
    whose touch mask names it."""
    for w, lib, grid in (small32, screen_sample):
        s = dict(w["search"], restarts=16, top_k=4)
        L = lg.Ligands.from_arrays(lib, "cuda")
        G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cuda")
        res = lg.dock_batch(L, G, restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"],
                            passes=s["passes"], top_k=s["top_k"], seed=s["seed"], trace=True, count_samples=True)
        trace = res.trace.cpu().numpy()
        touch = lg.pack_touch(L, grid.dims[3]).cpu().numpy()
        nt = 360 // s["torsion_step_deg"]
        P, R = s["passes"], s["restarts"]
        bits, _, _, _ = lg.pack_ligands(L, grid.dims[3])
        moving = np.unpackbits(bits.cpu().numpy().view(np.uint8), bitorder="little").reshape(len(bits), -1).sum(1)
        want = 0
        for l in range(lib.n_ligands):
            n, r0 = int(lib.n_rot[l]), int(lib.rot_off[l])
            tr = parity.ligand_trace(trace, lib.rot_off, R, P, l)
            for r in range(R):
                want += 24 * int(lib.n_atoms[l])
                dirty = (1 << n) - 1
                for d in range(P * n):
                    b = d % n
                    jb = int(tr[r, 1 + d])
                    if dirty >> b & 1:
                        want += (nt - 1) * (int(moving[r0 + b]) - 1)
                    else:
                        assert jb == 0
                    dirty = (dirty | int(touch[r0 + b]) if jb else dirty) & ~(1 << b)
        assert res.samples == want
