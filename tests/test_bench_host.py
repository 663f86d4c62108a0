"""Host logic of bench.py, without a GPU: the algorithmic byte counts behind
the roofline, the profile-traffic lookup that turns null once the kernel
sources change, and the peak lookup."""
import json
import os
import shutil

import pytest

import bench


def test_algorithmic_bytes_per_unit():
    live = {"em": 1000, "ep": 10, "ph": 200, "ion": 300}
    # e- ion launch: 24 B per electron and ion record, 8 B of start + count
    # for each of the two species, 4 B material + 16 B ledger per cell,
    # 12 B per changed projectile, 32 B per secondary
    assert bench.ei_bytes(live, 50, 7, 5) == 24 * 1300 + (16 + 20) * 50 + 12 * 7 + 32 * 5
    # full step: every species' records and all four species' metadata
    assert bench.step_bytes(live, 50, 7, 5) == 24 * 1510 + (32 + 20) * 50 + 12 * 7 + 32 * 5


def _fake_root(tmp_path, traffic, source_hash):
    root = tmp_path / "root"
    csrc = root / "paper_1907_02814_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.COLLIDE_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_1907_02814_gb300", "csrc", f), csrc / f)
    prof = root / "profiles"
    prof.mkdir()
    (prof / "k.txt").write_text(f"kernel: k\ndram_bytes_per_launch_full_workload: {traffic}\n"
                                f"source_hash: {source_hash}\n")
    return str(root)


def test_profiled_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    h = bench.source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    monkeypatch.setattr(bench, "ROOT", _fake_root(tmp_path, 12345, h))
    assert bench.source_hash() == h
    assert bench.profiled_traffic("k") == 12345.0
    assert bench.profiled_traffic("missing") is None
    # a changed kernel source invalidates the committed counters
    src = os.path.join(bench.ROOT, "paper_1907_02814_gb300", "csrc", bench.COLLIDE_SOURCES[0])
    with open(src, "a") as f:
        f.write("\n// changed\n")
    assert bench.source_hash() != h
    assert bench.profiled_traffic("k") is None


def test_committed_profile_names_its_hash_and_command():
    p = os.path.join(bench.ROOT, "profiles", "collide_ei_batched.txt")
    text = open(p).read()
    assert "source_hash:" in text and "dram_bytes_per_launch_full_workload:" in text
    assert "ncu " in text and "--clock-control none" in text


def test_peaks_prefer_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.FALLBACK_HBM, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6657.6}))
    assert bench.peaks() == (6657.6, "measured")


def test_emission_instruction_counts_follow_the_kernel_sources(tmp_path, monkeypatch):
    root = tmp_path / "root"
    csrc = root / "paper_1907_02814_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.EMISSION_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_1907_02814_gb300", "csrc", f), csrc / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = bench.emission_source_hash()
    (root / "profiles").mkdir()
    (root / "profiles" / bench.EMISSION_PROFILE).write_text(
        f"# x\nsource_hash: {h}\n\n## void emission_kernel<0>  (forward)\n- warp instructions: 1000.0 inst\n"
        "## void emission_kernel<1>  (adjoint)\n- duration: 1 ms\n- warp instructions: 2500.5 inst\n")
    assert bench.emission_instructions() == {"fwd": 1000.0, "bwd": 2500.5}
    with open(csrc / bench.EMISSION_SOURCES[0], "a") as f:
        f.write("\n// changed\n")
    assert bench.emission_instructions() is None


def test_cpu_baseline_states_its_cores(monkeypatch):
    """Both oracle legs on a small case of the bench workload: single-threaded
    and on every core this process may use, with the core count stated."""
    from paper_1907_02814_gb300 import workloads as W
    counts = bench.workload_counts(W, 1 << 14, 3)
    out = bench.cpu_baseline(counts, budget_s=0.2)
    assert out["cores_available"] == bench.host_cores() >= 1
    assert out["value_1t"] > 0 and out["value_omp"] > 0 and out["value"] == out["value_omp"]
    assert 1 <= out["cores"] <= out["cores_available"] and out["kind"] == "oracle"
    assert "fixed subset" in out["sample"]


def test_live_records_gather_the_live_slots():
    """The end-to-end leg's gather of a cell-region layout: every cell's live
    slots in storage order, with their cell index, and nothing of the slack."""
    import types
    torch = pytest.importorskip("torch")
    start = torch.tensor([0, 3, 3, 7], dtype=torch.int32)
    count = torch.tensor([2, 0, 3], dtype=torch.int32)
    vals = torch.arange(7, dtype=torch.float32) * 10
    sp = types.SimpleNamespace(cell_start=start, cell_count=count, ux=vals, uy=vals + 1, uz=vals + 2, w=vals + 3,
                               pid=torch.arange(7, dtype=torch.int64) + 100)
    d = bench.live_records(torch, sp)
    assert d["n"] == 5
    assert d["ux"].tolist() == [0.0, 10.0, 30.0, 40.0, 50.0]
    assert d["pid"].tolist() == [100, 101, 103, 104, 105]
    assert d["cell"].tolist() == [0, 0, 2, 2, 2]
