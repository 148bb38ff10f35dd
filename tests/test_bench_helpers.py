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


def _reference_line(env_extra=None):
    import json
    import subprocess
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                        "--steps", "2", "--warmup", "1", "--ref-frames", "2"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return [json.loads(l) for l in lines]


def test_reference_arm_prints_one_contract_line():
    """The reference arm times the FP64 oracle on the host (no GPU) and prints one JSON line
    with the same metric, unit and workload as the CUDA arm."""
    (d,) = _reference_line()
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("c1-") and d["config"]["config"] == "c1"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "2 frame(s) x 1 probe(s) per step" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the oracle and prints; the other ranks exit 0."""
    assert _reference_line({"RANK": "1", "WORLD_SIZE": "2"}) == []
