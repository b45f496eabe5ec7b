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
