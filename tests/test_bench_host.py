"""Host-side logic of the benchmark (no GPU): the roofline object of the
dominant sweep kernel, built from the sweep ledger's CUDA-event time and
algorithmic bytes, against the bound that applies to the kernel; the DRAM
traffic taken from a committed profile only while the kernel's sources still
hash to the value recorded with it; and the kernel hash ignoring comments."""
import json
import os

import pytest

import bench

DEV = {"smem_gbs": 40000.0, "fp64_fma_tflops": 1.0, "fp32_fma_tflops": 70.0, "sm_count": 152, "clock_mhz": 2070.0}
PEAKS = {"hbm_gbs": 6800.0}


def _ledger(ms, launches, algo):
    return {kv: (ms, launches, algo) for kv in (1, 2, 3, 4)}


def test_band_kernel_roofline_against_shared_memory():
    # 2 launches of 250 ms moving 5e11 algorithmic bytes each: 2 TB/s
    ms, n, algo = 500.0, 2, 1e12
    obj = bench.roofline_object(2, "heat2d_127", _ledger(ms, n, algo), (ms, n, algo), PEAKS, "measured", DEV, 32)
    assert obj["bound"] == "smem"
    assert obj["achieved"] == pytest.approx(2000.0)
    assert obj["peak"] == DEV["smem_gbs"]
    assert obj["frac"] == pytest.approx(2000.0 / 40000.0)
    assert obj["ms_per_launch"] == pytest.approx(250.0)
    assert obj["algo_bytes_per_launch"] == pytest.approx(5e11)
    # the committed DRAM capture belongs to the current sources: traffic set
    # and reported beside the bound as a fraction of the HBM peak
    prof = json.load(open(bench.profile_summary("fast2d_kernel", "heat2d_127")))
    assert prof["kernel_hash"] == bench.kernel_hash(bench.KERNELS[2][2])
    assert obj["traffic"] == prof["dram_bytes_per_launch_full"]
    side = obj["hbm_side_note"]
    assert side["dram_gbs"] == pytest.approx(obj["traffic"] / 0.25 / 1e9)


def test_generic_kernel_roofline_against_hbm():
    ms, n, algo = 12000.0, 1, 8e12
    obj = bench.roofline_object(1, "heat3d_63", _ledger(ms, n, algo), (ms, n, algo), PEAKS, "measured", DEV, 16)
    assert obj["bound"] == "hbm"
    assert obj["peak"] == PEAKS["hbm_gbs"]
    assert obj["frac"] == pytest.approx((8e12 / 12.0 / 1e9) / 6800.0)
    prof = json.load(open(bench.profile_summary("sweep_kernel", "heat3d_63")))
    assert obj["traffic"] == prof["dram_bytes_per_launch_full"]


def test_stale_profile_gives_no_traffic(tmp_path, monkeypatch):
    # a profile recorded for other sources is not used
    prof = json.load(open(bench.profile_summary("sweep_kernel", "heat3d_63")))
    prof["kernel_hash"] = "0" * 16
    fake = tmp_path / "sweep_kernel_heat3d_63.json"
    fake.write_text(json.dumps(prof))
    monkeypatch.setattr(bench, "profile_summary", lambda name, workload="heat2d_127": str(fake))
    obj = bench.roofline_object(1, "heat3d_63", _ledger(1.0, 1, 1.0), (1.0, 1, 1.0), PEAKS, "measured", DEV, 16)
    assert obj["traffic"] is None


def test_kernel_hash_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1703_05638_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text("int f(int x) { return x + 1; }  // one\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_hash(["a.cuh"])
    (csrc / "a.cuh").write_text("/* header */\nint f(int x)\n{\n  return x + 1;   // two\n}\n")
    assert bench.kernel_hash(["a.cuh"]) == h1
    (csrc / "a.cuh").write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_hash(["a.cuh"]) != h1
