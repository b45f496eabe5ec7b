"""Host logic of bench.py that needs no GPU: the committed DRAM-traffic
counters are reported only while the kernel sources they were captured on
are unchanged (a hash of the sources' code, comments and whitespace
ignored), and the algorithmic work per launch follows the per-unit counts."""
import json
import os
import shutil

import bench


def test_traffic_reported_only_for_the_sources_it_was_captured_on():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "dram_traffic.json")))
    h = bench._kernel_hash()
    for wl, kinds in d.items():
        if wl.startswith("_"):
            continue
        for kind, ent in kinds.items():
            assert ent["bytes_per_launch"] > 0 and ent["scale"] >= 1
            want = ent["bytes_per_launch"] if ent["kernel_source_sha"] == h else None
            assert bench._traffic(wl, kind) == want
    assert bench._traffic("no_such_workload", "volume") is None


def test_kernel_hash_ignores_comments_and_whitespace_not_code(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2006_15698_gb300", "csrc")
    dst = tmp_path / "paper_2006_15698_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._kernel_hash()
    f = dst / "dg_kernels.cuh"
    text = f.read_text()
    f.write_text(text + "\n// a comment\n/* a block\n   comment */\n\n   \n")
    assert bench._kernel_hash() == h0
    f.write_text(text.replace("kKindVolume", "kKindVolumeRenamed"))
    assert bench._kernel_hash() != h0


def test_algorithmic_counts_per_launch():
    E, N = 1000, 5
    nodes, fpts = E * N ** 3, 3 * E * N ** 2
    assert bench.kernel_flops("volume", N, E) == nodes * (113 + 30 * N)
    assert bench.kernel_flops("face", N, E) == fpts * (69 + 20 * N)
    assert bench.kernel_bytes("volume", N, E, 8) == nodes * 5 * 8 * 4 + fpts * 5 * 8
    assert bench.kernel_bytes("stage", N, E, 4) == nodes * 80


def test_paper_volume_rate_from_its_operation_count():
    """Reading of the paper's counts (Sec. IV operation count 38 N^3 + 30 N^4
    per element and right-hand side; Table II volume kernel): its largest run,
    512 x 512 x 768 elements at p = 6, for 100 LSERK45 steps (500 right-hand
    sides) in 1.77 s of volume-kernel time, is the table's 4.84 PFLOP/s.  This
    fixes the step/stage counting of the metric (one RK stage = one
    right-hand side per element)."""
    N = 7
    elements = 512 * 512 * 768
    flops = elements * (38 * N ** 3 + 30 * N ** 4) * 5 * 100
    assert abs(flops / 1.77 / 4.84e15 - 1.0) < 2e-3
