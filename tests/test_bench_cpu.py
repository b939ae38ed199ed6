"""The benchmark's own arithmetic (no GPU): the nominal sample and pose
counts that the roofline and poses/s rest on, against counts built ligand by
ligand from the oracle's fragments, and the rule that drops a recorded DRAM
traffic figure once the kernel source changes."""
import pytest

import gen


def test_algorithmic_counts_match_fragment_sums(oracle_lib):
    import bench
    w = gen.scaled("screen20k", 40)
    lib = gen.make_library(w["library"])
    s = w["search"]
    R, P = s["restarts"], s["passes"]
    nt = 360 // s["torsion_step_deg"]
    poses = samples = moving = 0
    for l in range(lib.n_ligands):
        lig = oracle_lib.OLigand.from_library(lib, l)
        n, N = lig.n_rot, lig.n_atoms
        poses += R * (24 + P * n * nt)
        samples += R * 24 * N
        if n:
            _, mask, _ = oracle_lib.fragments(lig)
            m = mask.reshape(n, N).sum(1)           # moving side, v included
            moving += int(m.sum())
            samples += R * P * (nt - 1) * int((m - 1).sum())
    got_poses, got_samples = bench.algorithmic_counts(lib, s, moving)
    assert got_poses == poses and got_samples == samples


def test_recorded_traffic_requires_matching_source_and_form(monkeypatch):
    import bench
    for form in ("f16", "plain"):
        value, _ = bench.recorded_traffic(form)
        assert value is not None and value > 0           # the committed capture matches this source
    assert bench.recorded_traffic("bf16")[0] is None       # a form without a capture
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")   # an edited kernel
    assert bench.recorded_traffic("f16") == (None, "kernel changed since the full-size ncu capture")


def test_job_throughput_counts_every_rank():
    import bench
    assert bench.job_throughput(1000, 4, 5, 2000.0) == pytest.approx(1000 * 4 * 5 / 2.0)
