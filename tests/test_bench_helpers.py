"""Host-side helpers of bench.py: the ncu traffic lookup and the roofline arithmetic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_scales_with_the_launch_and_needs_matching_sources(monkeypatch, tmp_path):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.md").write_text(
        "| config | kernel | dram_bytes_per_algorithmic_byte | captured launch | src |\n"
        "|---|---|---|---|---|\n"
        "| c2 | slice_row | 1.25 | one launch | abc123 |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "src_hash", lambda kernel=None: "abc123")
    assert bench.ncu_traffic("slice_row", "c2", 1000.0) == 1250.0
    assert bench.ncu_traffic("slice_col", "c2", 1000.0) is None
    assert bench.ncu_traffic("slice_row", "c4", 1000.0) is None
    monkeypatch.setattr(bench, "src_hash", lambda kernel=None: "changed")
    assert bench.ncu_traffic("slice_row", "c2", 1000.0) is None


def test_src_hash_follows_only_the_kernels_sources():
    """The FFT pass classes hash the files they are compiled from; host-side or time-transform
    files do not enter their hash, and an unlisted class hashes every CUDA source."""
    assert bench.src_hash("slice_row") == bench.src_hash("slice_col")
    assert bench.src_hash("slice_row") != bench.src_hash(None)
    assert "api.cu" not in bench.KERNEL_SOURCES["slice_row"]
    assert "k_slices.cu" in bench.KERNEL_SOURCES["slice_row"]


def test_roofline_picks_the_dominant_kernel_and_its_bound(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 1000.0, "bf16_tflops_sustained": 100.0,
                                                          "sm_max_mhz": 2070.0}, "of measured"))
    monkeypatch.setattr(bench, "ncu_traffic", lambda *a: None)
    # (ms, launches, algorithmic bytes, flops) per step of each class
    prof = {"slice_row": (10.0, 4.0, 4e9, 1e9), "dft_tc_bf16": (1.0, 1.0, 1e6, 5e13)}
    r = bench.roofline(prof, 1, "c2", 2070.0)
    assert r["kernel"] == "slice_row" and r["bound"] == "hbm"
    assert abs(r["achieved"] - 400.0) < 1e-9 and abs(r["frac"] - 0.4) < 1e-12  # 1 GB in 2.5 ms
    prof = {"dft_tc_bf16": (10.0, 1.0, 1e6, 5e11)}  # 5e11 flops in 10 ms
    r = bench.roofline(prof, 1, "c4", 2070.0)
    assert r["bound"] == "tensor" and abs(r["achieved"] - 50.0) < 1e-9 and abs(r["frac"] - 0.5) < 1e-12
