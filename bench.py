"""Throughput of the docking pose search on synthetic libraries.

One step = one ligen_dock_batch call over the whole library (grid
preparation, ligand packer, docking kernel, top-K), inputs resident in HBM.
Default workload: 20,000 ligands (atoms ~ N(38, 14) in [8, 100], rotatable
bonds ~ Poisson(6) in [0, 24]) into a 96^3 x 8 grid at 0.375 A, 256 restarts,
24 cube rotations, 10-degree torsion steps, 3 sweep passes, top 30 kept.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): every rank docks its own library shard of the same
size (its own seed); no data exchange, so scaling is weak. Rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ligands/s and poses/s on 1 GB300: chosen form vs plain FP32 at <=1e-3 score err"
WORKLOAD = "screen20k"
WORKLOAD_DESCS = {
    "screen20k": ("screen20k: 20,000 synthetic ligands (atoms ~N(38,14) in [8,100], rotatable bonds "
                  "~Poisson(6) in [0,24]), 96^3x8 FP32 pocket grid at 0.375 A, 256 restarts x 24 cube "
                  "rotations, 10 deg torsion steps, 3 passes, top-30"),
    "bimodal200k": ("bimodal200k: 200,000 synthetic ligands, 70% with 15-35 atoms and 0-8 rotatable bonds, "
                    "30% with 60-120 atoms and 8-30; 96^3x8 FP32 grid at 0.375 A, 256 restarts x 24 cube "
                    "rotations, 10 deg steps, 3 passes, top-30"),
}
WORKLOAD_DESC = WORKLOAD_DESCS[WORKLOAD]
BYTES_PER_SAMPLE = 32   # one trilinear sample = one 32-byte record of 8 FP32 coefficients


SCORE_ROT_CAPS = (0, 2, 4, 6, 8, 12, 16, 24, 32)   # rotatable-bond classes of the pose-per-lane launches


def score_classes(lib) -> int:
    """Launches of one pose-per-lane scoring or gradient call: one per
    rotatable-bond class present in the library."""
    import bisect
    return len({bisect.bisect_left(SCORE_ROT_CAPS, int(n)) for n in np.diff(lib.rot_off)})


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ligands", type=int, default=None, help="cut the library (testing only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOAD_DESCS))
    ap.add_argument("--refine-steps", type=int, default=50,
                    help="gradient-refinement steps of the top-16 poses (0 disables the leg)")
    ap.add_argument("--sites", type=int, default=12,
                    help="docking sites of the multi-site leg (0 disables it)")
    ap.add_argument("--bimodal-ligands", type=int, default=200000,
                    help="ligands of the bimodal batching leg (0 disables it)")
    ap.add_argument("--forms", default="plain,buckets,buckets_static,queue,f16,bf16,f16_rescore",
                    help="docking layouts to time; the fastest is the reported form")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_spec(rank: int, n_ligands=None, workload: str = WORKLOAD) -> dict:
    """Workload of one rank: the same recipe and size on every rank, with the
    library and restart seeds offset by the rank, so each GPU docks its own
    shard of a world_size-times larger library (weak scaling)."""
    import gen
    w = gen.scaled(workload, n_ligands or gen.WORKLOADS[workload]["library"]["n_ligands"])
    w["library"]["seed"] = int(w["library"]["seed"]) + 1000 * rank
    w["search"]["seed"] = int(w["search"]["seed"]) + 1000 * rank
    return w


def workload(n_ligands=None, rank=0, name: str = WORKLOAD):
    import gen
    w = shard_spec(rank, n_ligands, name)
    return w, gen.make_library(w["library"]), gen.make_grid(w["grid"])


def max_over_ranks(x: float, world: int) -> float:
    """Max of a per-rank number over all ranks (timing: the slowest rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ligands_per_rank: int, world: int, steps: int, ms_total_max: float) -> float:
    """Whole-job ligands/s: every rank's ligands over the slowest rank's time."""
    return ligands_per_rank * world * steps / (ms_total_max * 1e-3)


def choose_form(forms, ms_total: dict, accuracy: dict, world: int = 1) -> str:
    """The reported form: the fastest one with relative score error <= 1e-3
    and best-pose agreement >= 0.99 (forms without an accuracy entry count as
    meeting it). Only rank 0 measures accuracy, so under torchrun rank 0's
    choice is broadcast and every rank runs the later legs in that form."""
    meets = [f for f in forms if f not in accuracy or (accuracy[f]["rel_err_max"] <= 1e-3
                                                        and accuracy[f]["best_pose_agreement"] >= 0.99)]
    form = min(meets or forms, key=lambda f: ms_total[f])
    if world > 1:
        import torch.distributed as dist
        box = [form]
        dist.broadcast_object_list(box, src=0)
        form = box[0]
    return form


# Docking layouts and grid formats the benchmark times (ligen_dock_batch options).
FORMS = {
    "plain": dict(batching="plain", grid_format="f32"),
    "buckets": dict(batching="buckets", grid_format="f32"),
    "buckets_static": dict(batching="buckets_static", grid_format="f32"),
    "queue": dict(batching="queue", grid_format="f32"),
    "f16": dict(batching="plain", grid_format="f16"),
    "bf16": dict(batching="plain", grid_format="bf16"),
    # FP16 records, then the K kept poses re-scored in FP64 and re-ranked (C3's re-score)
    "f16_rescore": dict(batching="plain", grid_format="f16", rescore_fp64=True),
    # static per-bucket launches on FP16 records (timed on the bimodal library)
    "f16_buckets_static": dict(batching="buckets_static", grid_format="f16"),
}

# FP32-pipe operations per atom sample of the sweep, counted from the samplers'
# source: rotation of the atom by the increment (6 FMA), box test (6 compares),
# cell and fraction (3 floor + 3 subtract, FP32 records also 3 clamps), then
# FP32 records: the cell polynomial (7 FMA); 16-bit records: 8 conversions to
# FP32 and 7 lerps (2 operations each); and the accumulation (1).
OPS_PER_SAMPLE = {"f32": 6 + 6 + 9 + 7 + 1, "f16": 6 + 6 + 6 + 8 + 14 + 1, "bf16": 6 + 6 + 6 + 8 + 14 + 1}
FP32_LANES_PER_SM = 128


def form_accuracy(lib, grid, s, outs: dict, lg, n_sample: int = 64) -> dict:
    """Score error and best-pose agreement of each form against the oracle.

    On n_sample ligands spread over the library: relative error of every kept
    pose's score (|S_form - S_oracle(pose)| / D, D = max(|S|, sum |E_i|)),
    and the fraction of ligands whose best kept pose scores, in the oracle,
    within 1e-3 * D of the best final score of the oracle's own search."""
    import oracle
    idx = np.linspace(0, lib.n_ligands - 1, n_sample).astype(int)
    ref = oracle.dock_library(lib, grid, s, ligands=idx)
    og = oracle.OGrid.from_grid(grid)
    K = s["top_k"]
    off = lg.pose_offsets(lib.rot_off, K)
    out = {}
    for f, res in outs.items():
        poses = res.poses.cpu().numpy()
        sc = (res.scores_f64 if res.scores_f64 is not None else res.scores).cpu().numpy()
        errs, agree = [], 0
        for r_ in ref:
            l = r_["ligand"]
            lig = oracle.OLigand.from_library(lib, l)
            P = poses[off[l]:off[l + 1]].reshape(K, -1).astype(np.float64)
            best = -np.inf
            for k in range(K):
                S, D, _ = oracle.score_pose(lig, og, P[k], s["out_penalty"])
                errs.append(abs(sc[l, k] - S) / D)
                best = max(best, S)
            j = int(np.argmax(r_["score"]))
            agree += best >= r_["score"][j] - 1e-3 * r_["dnorm"][j, -1]
        out[f] = {"rel_err_max": float(np.max(errs)), "rel_err_mean": float(np.mean(errs)),
                  "best_pose_agreement": agree / len(ref), "accuracy_sample_ligands": int(n_sample)}
    return out


def algorithmic_counts(lib, s, moving_atoms):
    """Nominal poses and algorithmic atom samples of one step.

    poses   = R * (24 + P * n * n_theta) per ligand
    samples = R * (24 * N + P * sum_b (n_theta - 1) * (m_b - 1)) per ligand:
              every atom of every rigid candidate, and in the sweep only the
              atoms whose position changes (the moving side of bond b has m_b
              atoms; its axis atom does not move) for the n_theta - 1
              increments other than the current one. `moving_atoms` is
              sum_b m_b over the library.
    """
    R, P = s["restarts"], s["passes"]
    nt = 360 // s["torsion_step_deg"]
    n = lib.n_rot.astype(np.int64)
    N = lib.n_atoms.astype(np.int64)
    poses = int(np.sum(R * (s.get("n_rigid", 24) + P * n * nt)))
    moved = int(moving_atoms) - int(n.sum())
    samples = int(np.sum(R * s.get("n_rigid", 24) * N) + R * P * (nt - 1) * moved)
    return poses, samples


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up (NVML initialisation) competes with the
            # launches of the first timed steps: wait for its first sample
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 10.0:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("k_dock.cu", "device_common.cuh"):
        with open(os.path.join(ROOT, "paper_2303_06150_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(form: str):
    """DRAM bytes of one full-size docking launch from the committed ncu capture.

    The docking kernel's DRAM traffic is the grid's hot region read once, so it
    does not grow with the number of ligands and a small-case capture cannot be
    scaled; only a full-size capture of the unchanged kernel is reported."""
    path = os.path.join(ROOT, "profiles", f"dock_kernel_traffic_{form}.txt")
    if not os.path.exists(path):
        return None, "no ncu summary"
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_hash") != kernel_source_hash():
        return None, "kernel changed since the full-size ncu capture"
    if kv.get("form") != form:
        return None, f"the full-size capture is of form {kv.get('form')}, not {form}"
    try:
        return float(kv["dram_bytes_per_launch"]), kv.get("command", "")
    except (KeyError, ValueError):
        return None, "no full-size figure"


def cpu_baseline(lib, grid, s, n_sample=96, threads=None):
    import oracle
    idx = np.linspace(0, lib.n_ligands - 1, n_sample).astype(int)
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.dock_library(lib, grid, s, ligands=idx, threads=threads)
    dt = time.perf_counter() - t0
    one = idx[::12]                                   # every 12th of the same sample, one thread
    t1 = time.perf_counter()
    oracle.dock_library(lib, grid, s, ligands=one, threads=1)
    d1 = time.perf_counter() - t1
    return {"value": n_sample / dt, "unit": "ligands/s", "cores": threads, "kind": "oracle",
            "sample": f"{n_sample} ligands evenly spaced over the {lib.n_ligands}-ligand library, all "
                      f"{s['restarts']} restarts, FP64 C++ oracle, {dt:.1f} s wall",
            "one_core": {"value": len(one) / d1, "unit": "ligands/s", "cores": 1,
                         "sample": f"{len(one)} of those ligands on one thread, {d1:.1f} s"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w, lib, grid = workload(args.ligands, 0, args.workload)
    s = w["search"]
    import oracle
    oracle.lib()
    threads = os.cpu_count() or 1
    per_step = 32
    rng = np.random.default_rng(0)
    for _ in range(args.warmup):
        oracle.dock_library(lib, grid, s, ligands=rng.choice(lib.n_ligands, 4, replace=False), threads=threads)
    times = []
    for k in range(args.steps):
        idx = rng.choice(lib.n_ligands, per_step, replace=False)
        t0 = time.perf_counter()
        oracle.dock_library(lib, grid, s, ligands=idx, threads=threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ligands/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD_DESCS[args.workload], "parallelism": "host threads"},
           "cpu_baseline": {"value": value, "unit": "ligands/s", "cores": threads, "kind": "oracle",
                            "sample": f"{per_step} random ligands of the library per step, all restarts"},
           "e2e": {"value": value, "unit": "ligands/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def time_dock(lg, L, G, fkw, flush, stream, steps, warmup, local, world):
    """Time `steps` ligen_dock_batch calls (L2 flushed before each) with CUDA
    events on the launching stream, after `warmup` untimed calls; the
    library's own stage events give the docking kernel's time per call."""
    import torch
    import torch.distributed as dist
    out = lg.dock_batch(L, G, stage_ms=True, **fkw)   # allocates outputs and workspace
    for _ in range(warmup):
        flush.fill_(1)
        lg.dock_batch(L, G, out=out, **fkw)
    torch.cuda.synchronize()
    dock_ms = []
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            flush.fill_(1)
            lg.dock_batch(L, G, out=out, **fkw)
            dock_ms.append(float(out.stage_ms[3]))
        t1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms_total = max_over_ranks(t0.elapsed_time(t1), world)
    return dict(ms_total=ms_total, dock_ms=float(np.mean(dock_ms)), stage=out.stage_ms.copy(),
                clocks=clk.summary(), out=out)


def bimodal_leg(args, lg, G_screen, screen_grid_spec, flush, stream, dev, rank, local, world):
    """The batching comparison on the bimodal library (paper §3's uneven
    atoms x rotamers mix): plain launch, bucketed persistent launches, the
    static per-bucket launches, the single persistent queue over the whole
    library and the FP16 plain launch, each timed like the
    headline (L2 flushed, CUDA events), with the per-bucket kernel shapes the
    autotuner picks for this library."""
    import gen
    w = shard_spec(rank, args.bimodal_ligands, "bimodal200k")
    lib = gen.make_library(w["library"], workers=os.cpu_count() or 1)
    grid_spec = w["grid"]
    G = G_screen if grid_spec == screen_grid_spec else None
    if G is None:
        grid = gen.make_grid(grid_spec)
        G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, dev)
    s = w["search"]
    kw = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
              top_k=s["top_k"], seed=s["seed"], n_rigid=s["n_rigid"], jitter=s["jitter"],
              out_penalty=s["out_penalty"])
    L = lg.Ligands.from_arrays(lib, dev)
    bits, _, buckets, _ = lg.pack_ligands(L, grid_spec["channels"])
    moving = np.unpackbits(bits.cpu().numpy().view(np.uint8), bitorder="little").sum() if bits.numel() else 0
    poses_step, samples_step = algorithmic_counts(lib, s, moving)
    tuned = lg.autotune(L, G, sample=256, **kw)
    steps = max(2, min(args.steps, 3))
    forms = ["plain", "buckets", "buckets_static", "queue", "f16"]
    timed = {f: time_dock(lg, L, G, dict(kw, **FORMS[f]), flush, stream, steps, 2, local, world) for f in forms}
    # the tuning table holds one shape per bucket, for the record format it
    # was timed with: retuned on FP16 records for the FP16 bucketed form
    tuned16 = lg.autotune(L, G, sample=256, grid_format="f16", **kw)
    timed["f16_buckets_static"] = time_dock(lg, L, G, dict(kw, **FORMS["f16_buckets_static"]), flush, stream,
                                            steps, 2, local, world)
    out = {"workload": WORKLOAD_DESCS["bimodal200k"].replace("200,000", f"{lib.n_ligands:,}"),
           "ligands": lib.n_ligands, "steps": steps, "warmup": 2,
           "nominal_poses_per_step": poses_step, "nominal_samples_per_step": samples_step,
           "forms": {f: {"value": job_throughput(lib.n_ligands, world, steps, t["ms_total"]), "unit": "ligands/s",
                         "ms_per_step": t["ms_total"] / steps, "dock_ms": t["dock_ms"],
                         "vs_plain_fp32": timed["plain"]["ms_total"] / t["ms_total"], **FORMS[f]}
                     for f, t in timed.items()},
           "buckets_vs_static": timed["buckets_static"]["ms_total"] / timed["buckets"]["ms_total"],
           "queue_vs_buckets": timed["buckets"]["ms_total"] / timed["queue"]["ms_total"],
           "tuning": {str(b): list(v[:2]) for b, v in sorted(tuned.items())},
           "tuning_f16": {str(b): list(v[:2]) for b, v in sorted(tuned16.items())},
           "clocks": timed["plain"]["clocks"],
           "how": "each form: 2 untimed calls, then steps calls with the L2 flushed before each, CUDA events "
                  "on the launching stream; accuracy of the FP16 form is measured on the headline workload "
                  "(the FP16 static-bucket form makes the FP16 plain launch's decisions, tested)"}
    del L, timed
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2303_06150_gb300 as lg

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, lib, grid = workload(args.ligands, rank, args.workload)
    s = w["search"]
    kw = dict(restarts=s["restarts"], torsion_step_deg=s["torsion_step_deg"], passes=s["passes"],
              top_k=s["top_k"], seed=s["seed"], n_rigid=s["n_rigid"], jitter=s["jitter"],
              out_penalty=s["out_penalty"])
    L = lg.Ligands.from_arrays(lib, dev)
    G = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, dev)
    bits, _, buckets, _ = lg.pack_ligands(L, grid.dims[3])
    present = sorted({int(b) for b in buckets.cpu().numpy()})
    moving = np.unpackbits(bits.cpu().numpy().view(np.uint8), bitorder="little").sum() if bits.numel() else 0
    poses_step, samples_step = algorithmic_counts(lib, s, moving)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > L2: written between steps
    stream = torch.cuda.current_stream(dev)
    forms = [f for f in args.forms.split(",") if f]
    tuned = None
    if any(f.startswith("buckets") for f in forms):
        # per-bucket kernel shapes for this library (not timed)
        tuned = lg.autotune(L, G, sample=256, **kw)

    def time_form(form):
        return time_dock(lg, L, G, dict(kw, **FORMS[form]), flush, stream, args.steps, args.warmup, local, world)

    timed = {f: time_form(f) for f in forms}
    accuracy = form_accuracy(lib, grid, s, {f: t["out"] for f, t in timed.items()}, lg) if rank == 0 else {}
    form = choose_form(forms, {f: t["ms_total"] for f, t in timed.items()}, accuracy, world)
    best = timed[form]
    stage = best["stage"]
    ms_total = best["ms_total"]
    ms_step = ms_total / args.steps
    value = job_throughput(lib.n_ligands, world, args.steps, ms_total)
    out = best["out"]

    # Roofline of the docking kernel, on the chosen form's event-timed kernel
    # duration. One atom sample reads one grid record: 32 bytes (FP32
    # coefficients) or 16 (FP16/BF16 corners). Algorithmic samples per step:
    # the nominal count R (24 N + P sum_b (n_theta - 1)(m_b - 1)) per ligand
    # (exact, from the generated library), and the samples the search needed
    # (the nominal count minus the sweeps of clean bonds, counted by the
    # kernel in one untimed call of the same form; the count is deterministic).
    fmt = FORMS[form]["grid_format"]
    rec_bytes = BYTES_PER_SAMPLE if fmt == "f32" else BYTES_PER_SAMPLE // 2
    dock = best["dock_ms"]
    needed = lg.dock_batch(L, G, count_samples=True, **dict(kw, **FORMS[form])).samples
    nominal_bytes = samples_step * rec_bytes
    # the bound's L2 term: streaming (coalesced) L2 reads of a 20 MB buffer,
    # the size of the grid's hot region, measured in this run
    probe_buf = torch.randn((20 << 20) // 32, 8, device=dev)
    l2_stream = max(lg.probe_stream(probe_buf, 20)["gbs"] for _ in range(3))
    # achievable gather ceiling: the same access (random records, one load of
    # rec_bytes each), no pose math, same buffer
    probe = max((lg.probe_gather(probe_buf, 512, rec_bytes) for _ in range(5)), key=lambda p: p["gbs"])
    # the bound's FP32 term: SMs x 128 lanes x the SM clock sampled during the timed steps
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = best["clocks"]["sm_mhz"] or 2070.0
    fp32_ops_per_s = sms * FP32_LANES_PER_SM * clk_mhz * 1e6
    ops = OPS_PER_SAMPLE[fmt]
    bound_l2 = l2_stream * 1e9 / rec_bytes                    # samples/s
    bound_fp32 = fp32_ops_per_s / ops                         # samples/s
    nominal_rate = samples_step / (dock * 1e-3)
    needed_rate = needed / (dock * 1e-3)
    achieved = nominal_bytes / (dock * 1e-3) / 1e9
    traffic, traffic_note = recorded_traffic(form)
    roofline = {"bound": "l2", "achieved": achieved, "peak": l2_stream, "unit": "GB/s",
                "frac": achieved / l2_stream, "traffic": traffic,
                "kernel": "dock_kernel", "kernel_ms": dock,
                "peak_source": "measured in this run: ligen_probe_stream, coalesced 16-byte ld.global.cg "
                               "reads of a 20 MB L2-resident buffer, best of 3",
                "achieved_counts": "nominal algorithmic samples (every sweep of every bond) x bytes per sample",
                "algorithmic_bytes": nominal_bytes, "bytes_per_sample": rec_bytes,
                "samples_nominal": samples_step, "samples_needed": needed,
                "clean_bond_skip_fraction": 1.0 - needed / samples_step,
                "frac_needed": needed * rec_bytes / (dock * 1e-3) / 1e9 / l2_stream,
                "frac_gather": needed_rate / probe["loads_per_s"],
                "gather_peak_gbs": probe["gbs"], "gather_peak_loads_per_s": probe["loads_per_s"],
                "frac_fp32": needed_rate * ops / fp32_ops_per_s,
                "ops_per_sample": ops,
                "bound_samples_per_s": {"l2": bound_l2, "fp32": bound_fp32,
                                        "binding": "l2" if bound_l2 <= bound_fp32 else "fp32"},
                "frac_of_bound": nominal_rate / min(bound_l2, bound_fp32),
                "fractions": "frac = nominal samples x bytes / kernel time / streaming L2; frac_needed = the "
                             "same with the samples the search needed; frac_gather = needed samples/s / the "
                             "random-gather probe's loads/s; frac_fp32 = needed samples/s x FP32 ops per "
                             "sample / (SMs x 128 x sampled SM clock); frac_of_bound = nominal samples/s / "
                             "min(L2 / bytes per sample, FP32 peak / ops per sample)",
                "hbm_context": {"peak_gbs": 6801.0, "source": "MEASURED_PEAKS.json hbm_gbs (context: the "
                                "grid's hot region is L2-resident)", "frac_if_hbm": achieved / 6801.0},
                "traffic_note": traffic_note}

    result = {"metric": METRIC, "value": value, "unit": "ligands/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32", "data": "synthetic",
              "config": {"workload": WORKLOAD_DESCS[args.workload], "ligands": lib.n_ligands,
                         "restarts": s["restarts"], "torsion_step_deg": s["torsion_step_deg"],
                         "passes": s["passes"], "top_k": s["top_k"],
                         "form": f"{form}: {FORMS[form]} (fastest of {'/'.join(forms)} meeting the bar)",
                         "l2": "flushed between steps (512 MB write)",
                         "parallelism": f"replicas x{world} (one library shard per GPU, no collective)"},
              "forms": {f: {"value": job_throughput(lib.n_ligands, world, args.steps, t["ms_total"]),
                            "ms_per_step": t["ms_total"] / args.steps, "dock_ms": t["dock_ms"],
                            "vs_plain_fp32": (timed["plain"]["ms_total"] / t["ms_total"]) if "plain" in timed
                            else None, **FORMS[f], **accuracy.get(f, {})}
                        for f, t in timed.items()},
              "chosen_form_rule": "fastest form with relative score error <= 1e-3 and best-pose agreement "
                                  ">= 0.99 on the oracle sample",
              "poses_per_s": poses_step * world * args.steps / (ms_total * 1e-3),
              "samples_per_s": needed * world * args.steps / (ms_total * 1e-3),
              "nominal_samples_per_s": samples_step * world * args.steps / (ms_total * 1e-3),
              "stage_ms_last_step": dict(zip(["h2d", "grid_prep", "pack", "dock", "topk_d2h"],
                                             [float(x) for x in stage])),
              "roofline": roofline,
              "gpu_launches": None,
              "clocks": best["clocks"]}
    # our kernels per step: grid preparation, packer, top-K, and one docking
    # launch (plain) or one per (atom class, kernel shape) group (buckets)
    table = lg.tune_get()
    per_step = (3 + (len({(b // 11, table[b]) for b in present}) if FORMS[form]["batching"] != "plain" else 1)
                + int(bool(FORMS[form].get("rescore_fp64"))))
    result["gpu_launches"] = per_step * args.steps
    if tuned is not None:
        result["tuning"] = {str(b): list(v[:2]) for b, v in sorted(tuned.items())}

    if not args.no_e2e:
        Lh = lg.Ligands.from_arrays(lib, "cpu", pin=True)
        Gh = lg.PocketGrid.from_array(grid.values, grid.origin, grid.spacing, "cpu", pin=True)
        outh = lg.dock_batch(Lh, Gh, **dict(kw, **FORMS[form]))
        for _ in range(max(1, args.warmup // 2)):
            lg.dock_batch(Lh, Gh, out=outh, **dict(kw, **FORMS[form]))
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for _ in range(args.steps):
            lg.dock_batch(Lh, Gh, out=outh, **dict(kw, **FORMS[form]))   # copies in, runs, copies out, syncs
        e_ms = max_over_ranks((time.perf_counter() - e0) * 1e3, world)
        h2d = Lh.nbytes() + Gh.values.numel() * 4
        d2h = (outh.poses.numel() + outh.scores.numel() + outh.status.numel()) * 4
        result["e2e"] = {"value": job_throughput(lib.n_ligands, world, args.steps, e_ms), "unit": "ligands/s",
                         "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                         "how": "ligen_dock_batch with pinned host inputs and outputs: H2D, kernels, D2H "
                                "and a stream sync per step, host wall clock"}
        result["gpu_launches"] += per_step * args.steps

    if args.refine_steps > 0 and args.workload == "screen20k":
        # gradient refinement of the top 16 poses per ligand after the sweep
        K16 = 16
        seeds = lg.dock_batch(L, G, **dict(kw, top_k=K16))
        before = seeds.scores.clone()
        lg.refine_poses(L, G, seeds.poses, K16, steps=args.refine_steps)   # warm-up
        times = []
        for _ in range(3):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            refined, after, _ = lg.refine_poses(L, G, seeds.poses, K16, steps=args.refine_steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
        gain = (after - before).cpu().numpy()
        b = before.cpu().numpy()
        result["refine"] = {
            "poses": int(lib.n_ligands * K16), "steps": args.refine_steps,
            "ms": float(min(times)), "poses_per_s": lib.n_ligands * K16 / (min(times) * 1e-3),
            "score_gain_mean": float(gain.mean()), "score_gain_median": float(np.median(gain)),
            "relative_gain_mean": float(np.mean(gain / np.maximum(np.abs(b), 1e-6))),
            "improved_fraction": float((gain > 0).mean()),
            "best_pose_gain_mean": float((after.max(1).values - before.max(1).values).mean().item()),
            "launches_per_call": 3 + score_classes(lib),
            "how": "top-16 poses per ligand of the sweep, normalised-step projected ascent "
                   "(0.1 A, 0.02, 0.05 rad; halve on rejection); per call grid preparation, packer, "
                   "forward-kinematics table and one refinement launch per rotatable-bond class "
                   "(side by side on forked streams), timed with CUDA events (best of 3)"}

    if args.workload == "screen20k":
        # ligen_score_poses on the kept poses of the timed form (all K per ligand):
        # the whole call (grid records, packer, scoring), and the scoring kernels
        # alone on inputs prepared once (ligen_prepare_scoring / ligen_score_prepared)
        K = s["top_k"]

        def best_ms(fn, reps=5):
            fn()   # warm-up
            times = []
            for _ in range(reps):
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                fn()
                ev1.record(stream)
                torch.cuda.synchronize()
                times.append(ev0.elapsed_time(ev1))
            return min(times)

        ms = best_ms(lambda: lg.score_poses(L, G, out.poses, K), 3)
        prep = lg.prepare_scoring(L, G)
        sc_out = torch.empty((lib.n_ligands, K), dtype=torch.float32, device=dev)
        ms_k = best_ms(lambda: prep.score(out.poses, K, out=sc_out), 10)
        prep.release()
        n_poses = lib.n_ligands * K
        n_samples = float(K * lib.n_atoms.sum())
        probe32 = max((lg.probe_gather(probe_buf, 512, 32) for _ in range(3)), key=lambda p: p["gbs"])
        result["score"] = {
            "poses": n_poses, "ms": ms, "poses_per_s": n_poses / (ms * 1e-3),
            "kernel_ms": ms_k, "kernel_poses_per_s": n_poses / (ms_k * 1e-3),
            "atom_samples_per_s": n_samples / (ms_k * 1e-3),
            "frac_gather": n_samples / (ms_k * 1e-3) / probe32["loads_per_s"],
            "frac_l2": n_samples * 32 / (ms_k * 1e-3) / 1e9 / l2_stream,
            "gather_peak_loads_per_s": probe32["loads_per_s"],
            "launches_per_call": score_classes(lib),
            "how": "ligen_score_poses on the kept poses of the timed form (20,000 ligands x top 30), FP32 grid "
                   "records: 'ms' is the whole call (grid records, packer, forward-kinematics table, scoring "
                   "launches), 'kernel_ms' the whole ligen_score_prepared call on inputs prepared once (one "
                   "launch per rotatable-bond class, side by side, replayed from a CUDA graph; host issue "
                   "included); CUDA events, best of 3 and 10; frac_gather = atom samples/s over the 32-byte "
                   "random-gather probe's loads/s, frac_l2 = 32 bytes per sample over the streaming L2 "
                   "bandwidth"}

    if args.sites > 0 and args.workload == "screen20k":
        # the same library docked into several sites of one target in one call
        import gen
        specs = gen.site_grids(w["grid"], args.sites)
        site_grids = [gen.make_grid(sp) for sp in specs]
        GS = [lg.PocketGrid.from_array(g.values, g.origin, g.spacing, dev) for g in site_grids]
        skw = dict(kw, **FORMS[form])
        outs = lg.dock_sites(L, GS, **skw)
        lg.dock_sites(L, GS, out=outs, **skw)      # warm-up
        times = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            lg.dock_sites(L, GS, out=outs, **skw)
            ev1.record(stream)
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
        ms = max_over_ranks(float(np.mean(times)), world)
        result["sites"] = {
            "n_sites": args.sites, "form": form, "ms_per_call": ms,
            "ligand_sites_per_s": lib.n_ligands * args.sites * world / (ms * 1e-3),
            "vs_single_site": (lib.n_ligands * args.sites / (ms * 1e-3)) / (lib.n_ligands / (ms_step * 1e-3)),
            "how": "ligen_dock_sites: library staged and packed once, then per site grid records, docking "
                   "and top-K into site-major outputs; device inputs, CUDA events, mean of up to 3 calls"}
        del outs, GS

    if args.bimodal_ligands > 0 and args.workload == "screen20k":
        result["bimodal"] = bimodal_leg(args, lg, G, w["grid"], flush, stream, dev, rank, local, world)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(lib, grid, s)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
