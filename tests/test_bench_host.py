"""Host logic of bench.py's roofline on CPU: the bound of a profiled site,
the achieved rate and fraction, and the DRAM traffic of the committed ncu
table, which is reported only while the kernel's source still has the
recorded digest."""
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


def test_traffic_only_while_the_digest_matches(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k_a(int n)\n{\n    (void)n;\n}\n__global__ void k_b(int n)\n{\n}\n")
    rel = os.path.relpath(str(src), ROOT)
    dig = bench.source_digest(rel + "::k_a")
    table = tmp_path / "traffic.md"
    table.write_text("| site | kernel | launches | DRAM bytes per launch | source | sha256 |\n|---|---|---|---|---|---|\n"
                     "| site_a | `k_a` | 3 | 1.5e+06 | `%s::k_a` | %s |\n" % (rel, dig))
    monkeypatch.setattr(bench, "TRAFFIC_MD", str(table))
    assert bench.measured_traffic("site_a") == 1.5e6
    assert bench.measured_traffic("site_b") is None
    # another kernel of the file changing leaves k_a's figure valid; k_a changing drops it
    src.write_text("__global__ void k_a(int n)\n{\n    (void)n;\n}\n__global__ void k_b(int n)\n{\n    n++;\n}\n")
    assert bench.measured_traffic("site_a") == 1.5e6
    src.write_text("__global__ void k_a(int n)\n{\n    n += 1;\n}\n")
    assert bench.measured_traffic("site_a") is None


def test_committed_traffic_table_names_existing_kernels():
    """Every row of the committed table names a source and kernel that
    exist (a renamed kernel would otherwise silently drop its figure)."""
    rows = 0
    for line in open(bench.TRAFFIC_MD).read().splitlines():
        parts = [q.strip().strip("`") for q in line.strip().strip("|").split("|")]
        if len(parts) >= 6 and "::" in parts[4] or (len(parts) >= 6 and parts[4].endswith(".cu")):
            bench.source_digest(parts[4])
            rows += 1
    assert rows >= 5
