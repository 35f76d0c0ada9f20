"""Host-side logic of bench.py that needs no GPU: the reference arm's extrapolation record and the
keying of the committed DRAM counters to the kernel source, instantiation and launch shape."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_extrapolation_record_relates_the_sample_to_a_full_step():
    r = bench.extrapolation(full_updates=7_340_032 * 100, sample_updates=1_048_576 * 144, mlups=25.0)
    assert r["factor"] == pytest.approx(7_340_032 * 100 / (1_048_576 * 144))
    assert r["full_step_ms_at_this_rate"] == pytest.approx(7_340_032 * 100 / 25e6 * 1e3)
    assert r["sample_updates_per_step"] == 1_048_576 * 144 and r["value_is_rate_of_sample"]


def test_step_kernel_names_follow_the_template_arguments():
    assert bench.step_kernel_name("f32", {"wall_inline": 1, "block_threads": 128}) == "k_step<float, float, 0, 1, 128>"
    assert bench.step_kernel_name("f16", {"wall_inline": 0, "block_threads": 64}) == "k_step<__half, float, 0, 0, 64>"


def test_committed_traffic_only_for_the_launch_it_was_taken_on(tmp_path, monkeypatch):
    """The counters file is used only while the kernel sources hash to the recorded value and the
    recorded instantiation, rows and grid equal the timed launch's."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash()
    (prof / "k_step_f32_counters.txt").write_text(
        "# test\n"
        f"kernel_source_sha256_16: {h}\n"
        "kernel: k_step<float, float, 0, 1, 128>\nblock_rows: 46\ngrid_blocks: 456\nworkload: sweep\n"
        "nodes_per_launch: 1000\ndram_bytes_per_launch: 150000\n")
    # counters from the temporary tree; the source hash as computed on the real one
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda sources=None: h)
    good = {"workload": "sweep", "kernel": "k_step<float, float, 0, 1, 128>", "block_rows": 46, "grid_blocks": 456}
    assert bench.committed_traffic("f32", 2000, launch=good) == pytest.approx(300000)
    assert bench.committed_traffic("f32", 2000, launch={**good, "workload": "compare"}) is None
    assert bench.committed_traffic("f32", 2000, launch={**good, "kernel": "k_step<float, float, 0, 0, 128>"}) is None
    assert bench.committed_traffic("f32", 2000, launch={**good, "grid_blocks": 608}) is None
    assert bench.committed_traffic("f16", 2000, launch=good) is None  # no record for this kernel
    # a second summary for another instantiation is found beside the first
    other = {**good, "kernel": "k_step<float, float, 0, 0, 128>", "block_rows": 38}
    (prof / "k_step_f32_counters_wall_called.txt").write_text(
        f"kernel_source_sha256_16: {h}\nworkload: sweep\n"
        "kernel: k_step<float, float, 0, 0, 128>\nblock_rows: 38\ngrid_blocks: 456\n"
        "nodes_per_launch: 1000\ndram_bytes_per_launch: 160000\n")
    assert bench.committed_traffic("f32", 2000, launch=other) == pytest.approx(320000)
    assert bench.committed_traffic("f32", 2000, launch=good) == pytest.approx(300000)
    assert bench.committed_traffic("f32", 2000, launch={**other, "block_rows": 46}) is None
    # a table of records, one per launch shape, below shared keys
    (prof / "k_step_f16_counters_shapes.txt").write_text(
        f"# table\nkernel_source_sha256_16: {h}\nworkload: sweep\nnodes_per_launch: 1000\n"
        "---\nkernel: k_step<__half, float, 0, 1, 128>\nblock_rows: 42\ngrid_blocks: 608\n"
        "dram_bytes_per_launch: 70000\n"
        "---\nkernel: k_step<__half, float, 0, 1, 128>\nblock_rows: 16\ngrid_blocks: 608\n"
        "dram_bytes_per_launch: 75000\n")
    h16 = {"workload": "sweep", "kernel": "k_step<__half, float, 0, 1, 128>", "grid_blocks": 608}
    assert bench.committed_traffic("f16", 2000, launch={**h16, "block_rows": 42}) == pytest.approx(140000)
    assert bench.committed_traffic("f16", 2000, launch={**h16, "block_rows": 16}) == pytest.approx(150000)
    assert bench.committed_traffic("f16", 2000, launch={**h16, "block_rows": 32}) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda sources=None: "0" * 16)
    assert bench.committed_traffic("f32", 2000, launch=good) is None  # the sources changed
    assert bench.committed_traffic("f32", 2000, launch=other) is None
    assert bench.committed_traffic("f16", 2000, launch={**h16, "block_rows": 42}) is None

