"""Host logic of bench.py's roofline on CPU: the bound of a profiled site,
the achieved rate and fraction, and the DRAM traffic of the committed ncu
data file (measured bytes per algorithmic byte of a few captured launches),
which is reported only while the kernel's source still has the recorded
digest."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6800.0}


def test_site_bounds_and_fractions():
    # 1 GB in 1 ms per launch against 6.8 TB/s: HBM-bound, 1000 GB/s
    r = bench.site_roofline("gmres_update_fp32", dict(ms=2.0, launches=2, bytes=2e9, flops=1e6), PEAKS)
    assert r["bound"] == "hbm" and abs(r["achieved"] - 1000.0) < 1e-9 and abs(r["frac"] - 1000.0 / 6800.0) < 1e-12
    # flops dominate on the FP64 pipe: ALU-bound against the FP64 peak
    r = bench.site_roofline("sai_build", dict(ms=1.0, launches=1, bytes=1e3, flops=1e9), PEAKS)
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_PEAK_TFLOPS and abs(r["achieved"] - 1.0) < 1e-12
    # an FP32 site uses the FP32 peak
    r = bench.site_roofline("gmres_project_fp32", dict(ms=1.0, launches=1, bytes=1e3, flops=1e12), PEAKS)
    assert r["peak"] == bench.FP32_PEAK_TFLOPS
    # a mixed site: 1e9 FP64 and 8e10 FP32 flops in 2 ms need 0.8 + 1.0 ms at the two peaks
    fp64, fp32 = bench.FP64_PEAK_TFLOPS * 1e12, bench.FP32_PEAK_TFLOPS * 1e12
    r = bench.site_roofline("sai_build", dict(ms=2.0, launches=1, bytes=1e3, flops=1e9 + 8.05e10,
                                              flops32=8.05e10), PEAKS)
    t_alu = 1e9 / fp64 + 8.05e10 / fp32
    assert r["bound"] == "alu" and abs(r["frac"] - t_alu / 2e-3) < 1e-12
    assert abs(r["frac_fp64"] - 1e9 / 2e-3 / fp64) < 1e-12 and abs(r["frac_fp32"] - 8.05e10 / 2e-3 / fp32) < 1e-12
    # control kernels carry no algorithmic work
    r = bench.site_roofline("gmres_step", dict(ms=1.0, launches=4, bytes=0.0, flops=0.0), PEAKS)
    assert r["bound"] == "latency" and r["frac"] is None


def test_roofline_picks_the_longest_site_and_can_drop_traffic():
    prof = {"sites": {"krylov_spmm_fp32": dict(ms=5.0, launches=10, timed=10, bytes=1e9, flops=1e8),
                      "gmres_update_fp32": dict(ms=9.0, launches=10, timed=10, bytes=5e9, flops=1e8),
                      "unused": dict(ms=0.0, launches=0, timed=0, bytes=0.0, flops=0.0)}}
    r = bench.roofline(prof, PEAKS, traffic=False)
    assert r["kernel"] == "gmres_update_fp32" and r["traffic"] is None
    assert set(r["sites"]) == {"krylov_spmm_fp32", "gmres_update_fp32"}


def _traffic_file(tmp_path, rel, dig):
    data = {"kernels": [{"site": "site_a", "kernel": "k_a", "source": rel + "::k_a", "sha256_16": dig,
                         "launches": [{"dram_bytes": 1.5e6, "algorithmic_bytes": 1.0e6},
                                      {"dram_bytes": 3.0e6, "algorithmic_bytes": 2.0e6}]}]}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(data))
    return str(path)


def test_traffic_only_while_the_digest_matches(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k_a(int n)\n{\n    (void)n;\n}\n__global__ void k_b(int n)\n{\n}\n")
    rel = os.path.relpath(str(src), ROOT)
    path = _traffic_file(tmp_path, rel, bench.source_digest(rel + "::k_a"))
    # 4.5 MB measured over 3 MB algorithmic: 1.5 measured bytes per algorithmic byte
    assert abs(bench.measured_traffic("site_a", 4.0e6, path) - 6.0e6) < 1e-6
    assert bench.measured_traffic("site_b", 4.0e6, path) is None
    # another kernel of the file changing leaves k_a's figure valid; k_a changing drops it
    src.write_text("__global__ void k_a(int n)\n{\n    (void)n;\n}\n__global__ void k_b(int n)\n{\n    n++;\n}\n")
    assert abs(bench.measured_traffic("site_a", 4.0e6, path) - 6.0e6) < 1e-6
    src.write_text("__global__ void k_a(int n)\n{\n    n += 1;\n}\n")
    assert bench.measured_traffic("site_a", 4.0e6, path) is None


def test_committed_traffic_file_names_existing_kernels():
    """Every entry of the committed traffic file names a source and kernel
    that exist (a renamed kernel would otherwise silently drop its figure)
    and carries launches with both byte counts."""
    if not os.path.exists(bench.TRAFFIC_JSON):
        return
    data = json.load(open(bench.TRAFFIC_JSON))
    for e in data["kernels"]:
        bench.source_digest(e["source"])
        assert e["launches"] and all(l["dram_bytes"] > 0 and l["algorithmic_bytes"] > 0 for l in e["launches"])
