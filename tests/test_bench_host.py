"""Host logic of bench.py's roofline block: the algorithmic bytes per launch,
the achieved bandwidth and fractions from the per-launch CUDA-event average,
the shared-memory pipe fraction from a captured wavefront count, and that
capture figures are used only for the kernel sources they were taken from."""
import pytest

import bench

N_IMG = 1024 * 2048          # the benchmarked B-scan
N_SPEC = 1024 * 2048


def test_algorithmic_bytes_per_launch():
    n = N_IMG
    # fused: eta_hat in, u_hat out (8N each) and half of F s_d (4N): 20N
    assert bench.algorithmic_bytes("ax_fused", N_IMG, N_SPEC) == 20 * n
    # update: u_hat, z^{k-1} in; z^k, eta_hat^{k+1} out: 32N
    assert bench.algorithmic_bytes("lat_update", N_IMG, N_SPEC) == 32 * n
    assert bench.algorithmic_bytes("ax_fwd", N_IMG, N_SPEC) == 16 * n
    assert bench.algorithmic_bytes("misc", N_IMG, N_SPEC) is None


def _kern(ms_total, launches):
    return {"ax_fused": {"ms": ms_total, "launches": launches}}


def test_roofline_arithmetic(monkeypatch):
    sha = bench.kernel_sources_sha("ax_fused")
    monkeypatch.setitem(bench.NCU_CAPTURES, "bscan_test", {
        "ax_fused": {"sha": sha, "dram": 123, "table": 45, "smem_wavefronts": 6_000_000}})
    abytes = 20 * N_IMG
    r = bench.roofline_of(_kern(500.0, 10000), "ax_fused", abytes, "bscan_test", 6787.2,
                          "measured", 2070.0, 152, "note")
    avg_s = 50e-6                                  # 500 ms over 10,000 launches
    assert r["avg_launch_us"] == pytest.approx(50.0)
    assert r["achieved"] == pytest.approx(abytes / avg_s / 1e9)
    assert r["frac"] == pytest.approx(abytes / avg_s / 1e9 / 6787.2)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 123
    assert r["traffic_split"] == {"algorithmic": abytes, "stolt_table": 45, "capture_sha": sha}
    assert r["smem_pipe"]["frac"] == pytest.approx(6_000_000 / (152 * 2070e6 * avg_s))


def test_stale_capture_is_not_reported(monkeypatch):
    monkeypatch.setitem(bench.NCU_CAPTURES, "bscan_test", {
        "ax_fused": {"sha": "0" * 16, "dram": 123, "table": 45, "smem_wavefronts": 1}})
    r = bench.roofline_of(_kern(500.0, 10000), "ax_fused", 20 * N_IMG, "bscan_test", 6787.2,
                          "measured", 2070.0, 152, "note")
    assert r["traffic"] is None and "smem_pipe" not in r and "traffic_note" in r
