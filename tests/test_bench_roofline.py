"""bench.py's roofline arithmetic (no GPU): the committed per-cell ncu counts
belong to the current kernel sources, and a launch's views follow from
them: achieved FP64 flops per second over the measured FP64 peak, split
into pipe busy x lane-and-arithmetic share x FMA mix, the algorithmic HBM
bytes over the copy bandwidth, and the DRAM traffic per launch."""
import pytest

import bench

N = 256 ** 3
PEAKS = {"fp64_tflops": 1.2533, "fp32_tflops": 76.0}
HBM = 6777.6


def test_counts_record_belongs_to_the_kernel_sources():
    """bench.py reports the pipe views only while the record's sources hash
    to the recorded value: a kernel edited without recapturing its counts
    fails here."""
    rec = bench.kernel_counts_record()
    assert rec is not None
    for form in ("fp64", "mixed", "fp64-ppm", "mixed-ppm"):
        for k in ("stage1", "stage2"):
            r = rec["stage_kernels"][form][k]
            assert r["fp64_flop"] > 0 and r["dram_bytes"] > 0
    assert rec["batched"] and rec["adjoint"]


def test_pipe_views_of_the_fp64_stage_kernel():
    rec = bench.kernel_counts_record()["stage_kernels"]["fp64"]["stage1"]
    ms = 46.01
    v = bench.pipe_views(rec, N, ms, PEAKS, HBM, bench.ALG_BYTES[0])
    flops = rec["fp64_flop"] * N / (ms * 1e-3)
    assert v["fp64"]["achieved"] == pytest.approx(flops / 1e12, rel=1e-12)
    assert v["fp64"]["frac"] == pytest.approx(flops / 1e12 / PEAKS["fp64_tflops"], rel=1e-12)
    d = v["fp64"]["decomposition"]
    product = d["fp64_pipe_busy_implied"] * d["lane_arith_share"] * d["fma_mix"]
    assert product == pytest.approx(v["fp64"]["frac"], rel=1e-12)
    assert 0.0 < d["lane_arith_share"] <= 1.0 and 0.5 <= d["fma_mix"] <= 1.0
    # one FP64 warp instruction holds the pipe 16 cycles: the implied busy
    # fraction cannot exceed 1 at the measured clock and time
    assert d["fp64_pipe_busy_implied"] < 1.0
    assert v["hbm"]["achieved"] == pytest.approx(144 * N / (ms * 1e-3) / 1e9, rel=1e-12)
    assert v["hbm"]["frac"] == pytest.approx(v["hbm"]["achieved"] / HBM, rel=1e-12)
    assert v["traffic_per_launch"] == pytest.approx(rec["dram_bytes"] * N, rel=1e-12)
    # the mixed form's transport adds an FP32 view
    recm = bench.kernel_counts_record()["stage_kernels"]["mixed"]["stage1"]
    vm = bench.pipe_views(recm, N, 31.5, PEAKS, HBM, bench.ALG_BYTES[0])
    assert vm["fp32"]["frac"] == pytest.approx(
        recm["fp32_flop"] * N / 31.5e-3 / 1e12 / PEAKS["fp32_tflops"], rel=1e-12)


def test_pipe_views_without_counts_report_hbm_only():
    v = bench.pipe_views(None, N, 46.0, PEAKS, HBM, bench.ALG_BYTES[1])
    assert set(v) == {"hbm"} and v["hbm"]["alg_bytes_per_cell"] == 208


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_rate(N, 20, 1, 1.814) == pytest.approx(N * 20 / 1.814 / 1e6)
    assert bench.whole_job_rate(N, 20, 4, 1.814) == pytest.approx(4 * N * 20 / 1.814 / 1e6)
    assert bench.ALG_BYTES == {0: 144, 1: 208}
