"""Helpers that compare the CUDA path with the oracle (test infrastructure).

Tolerances:
  * scores: |S_gpu - S_ref| <= 1e-5 * D + POS_ULPS * eps32 * Gs, with
    D = max(|S_ref|, sum_i |E_i|) and Gs = sum_i |grad E_i| |x_i - origin| the
    score's sensitivity to a relative perturbation of the atom coordinates
    (eps32 = 2^-24). The second term is the FP32 rounding of atom positions,
    which no FP32 evaluation avoids: at ~10 A an FP32 coordinate is off by up
    to 1e-6 A, and the grid's clash-plateau edges change E by up to ~12 per A;
  * decisions (chosen cube rotation, chosen torsion increment): equal at every
    decision whose oracle top-2 gap exceeds 1e-4 * D + 2 * POS_ULPS * eps32 * Gs (the
    score tolerance of both candidates). At a decision under that gap either
    choice is valid: when the GPU made the oracle's choice, both searches are
    still on the same trajectory and the comparison goes on; when it chose
    otherwise, the rest of that restart is not compared;
  * fragment masks, axes, buckets, statuses: bit-exact.

The 16-bit grid records hold each cell's corner values rounded to nearest
(FP16 or BF16) and interpolate them in FP32, so the search over them is the
oracle's search over a grid whose node values are those rounded values
(`record_values`); the same tolerances then apply.
"""
from __future__ import annotations

import numpy as np

SCORE_RTOL = 1e-5
GAP_RTOL = 1e-4
EPS32 = 2.0 ** -24
# Position term of the score tolerance: the docking kernel's final FP32 atom
# positions were measured against the oracle's FP64 positions of the same
# pose (test_docking_coordinates_within_pos_ulps): on 42,109 atom positions of
# small32 and the screening sample the error was at most 16.2 units of
# 2^-24 |u| (99.9% below 9.3); 24 is that maximum with a margin of 1.5.
POS_ULPS = 24


def record_values(values: np.ndarray, fmt: str) -> np.ndarray:
    """Node values as a grid record of format `fmt` holds them, in FP64: the
    FP32 values the caller passes, rounded to nearest-even in IEEE binary16
    ("f16") or bfloat16 ("bf16", the upper half of the binary32 pattern);
    "f32" keeps the FP32 values."""
    v32 = np.ascontiguousarray(values, np.float32)
    if fmt == "f32":
        return v32.astype(np.float64)
    if fmt == "f16":
        return v32.astype(np.float16).astype(np.float64)
    if fmt == "bf16":
        bits = v32.view(np.uint32).astype(np.uint64)
        upper = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16
        return (upper.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    raise ValueError(fmt)


def oracle_grid(oracle_lib, grid, fmt: str = "f32"):
    """The oracle's grid for a GPU run with records of format `fmt`: the
    generator's FP64 values for FP32 records (their FP32 rounding is inside
    the score tolerance), the rounded node values for 16-bit records."""
    if fmt == "f32":
        return oracle_lib.OGrid.from_grid(grid)
    return oracle_lib.OGrid(record_values(grid.values, fmt), grid.origin, grid.spacing)


def score_tol(D, Gs):
    return SCORE_RTOL * D + POS_ULPS * EPS32 * Gs


def gap_tol(D, Gs):
    return GAP_RTOL * D + 2 * POS_ULPS * EPS32 * Gs


def ligand_trace(trace: np.ndarray, rot_off: np.ndarray, R: int, passes: int, l: int) -> np.ndarray:
    n = np.diff(rot_off)
    start = R * (l + passes * int(rot_off[l]))
    D = 1 + passes * int(n[l])
    return trace[start:start + R * D].reshape(R, D)


def compare_restart(gpu_trace_row, ref: dict, j: int) -> tuple[int, bool]:
    """Compare one restart's decisions.

    Returns (decisions compared, whole trajectory identical)."""
    gap, dn, gs, tr = ref["gap"][j], ref["dnorm"][j], ref["gsens"][j], ref["trace"][j]
    for d in range(len(tr)):
        if gap[d] <= gap_tol(dn[d], gs[d]):
            if gpu_trace_row[d] != tr[d]:
                return d, False          # a near-tie resolved the other way: both valid
            continue
        assert gpu_trace_row[d] == tr[d], f"decision {d}: gpu {gpu_trace_row[d]} oracle {tr[d]}, gap {gap[d]}"
    return len(tr), True


def new_stats() -> dict:
    """Counters of a parity run: decisions compared, restarts, restarts on the
    oracle's trajectory, scores compared, how many of those meet the bare
    1e-5 * D (without the position term) and the worst |error| / (1e-5 D)."""
    return dict(decisions=0, restarts=0, clean=0, scores=0, bare_ok=0, bare_worst=0.0)


def merge(tot: dict, st: dict) -> dict:
    for k in tot:
        tot[k] = max(tot[k], st[k]) if k == "bare_worst" else tot[k] + st[k]
    return tot


def bare_ratio(err: float, D: float) -> float:
    """|S_gpu - S_ref| as a fraction of the bare relative bar 1e-5 * D."""
    return float(err) / (SCORE_RTOL * float(D))


def check_dock_ligand(l: int, ref: dict, gpu_trace: np.ndarray, gpu_final: dict | None) -> dict:
    """Per-restart parity of one ligand.

    gpu_final maps restart -> the GPU's final score for the restarts it
    reports (all of them when top_k = R, the kept ones otherwise)."""
    stats = new_stats()
    for j, r in enumerate(ref["restarts"]):
        nd, clean = compare_restart(gpu_trace[r], ref, j)
        stats["decisions"] += nd
        stats["restarts"] += 1
        if clean:
            stats["clean"] += 1
            if gpu_final is not None and int(r) in gpu_final:
                D, Gs = ref["dnorm"][j, -1], ref["gsens"][j, -1]
                g = gpu_final[int(r)]
                assert abs(g - ref["score"][j]) <= score_tol(D, Gs), (l, r, g, ref["score"][j], D, Gs)
                stats["scores"] += 1
                b = bare_ratio(abs(g - ref["score"][j]), D)
                stats["bare_ok"] += int(b <= 1.0)
                stats["bare_worst"] = max(stats["bare_worst"], b)
    return stats


def coord_ulps(u_gpu: np.ndarray, u_ref: np.ndarray) -> np.ndarray:
    """Per-atom position error in units of 2^-24 |u_ref| (u: grid-unit
    positions, distance from the grid origin): the measure the position term
    of the score tolerance assumes, |dx_i| <= POS_ULPS * eps32 * |x_i - origin|."""
    err = np.linalg.norm(np.asarray(u_gpu, np.float64) - u_ref, axis=-1)
    return err / (EPS32 * np.maximum(np.linalg.norm(u_ref, axis=-1), 1e-30))


def clean_restart(ref: dict, j: int, gpu_trace_row=None) -> bool:
    """True when restart j's trajectory is determined: no decision is a
    near-tie, or (given the GPU's trace) every near-tie went the same way."""
    near = ref["gap"][j] <= gap_tol(ref["dnorm"][j], ref["gsens"][j])
    if gpu_trace_row is None:
        return not bool(near.any())
    return bool(np.all(np.asarray(gpu_trace_row)[near] == ref["trace"][j][near]))


def unpack_bits(words: np.ndarray, N: int) -> np.ndarray:
    w = words.astype(np.uint32)
    bits = (w[:, :, None] >> np.arange(32, dtype=np.uint32)[None, None, :]) & 1
    return bits.reshape(len(words), -1)[:, :N].astype(bool)
