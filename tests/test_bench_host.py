"""bench.py's host-side measurement arithmetic, checked against hand counts:
the algorithmic bytes of the FFT stages (full and reduced grids), the
Legendre flop count, the 16-bit table bytes of the split GEMMs, the roofline
fractions and bounds it reports, and the whole-job throughput."""
import pytest

import bench
from paper_1711_11296_gb300 import workloads as W

T639 = W.WORKLOADS["T639"]
PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def test_fft_bytes_by_hand():
    # FP32 T639 x 256: grid 256 * 1281 * 2560 * 4 B, workspace 640 m x 2
    # parities x 641 northern nodes x 256 fields x 8 B (complex FP32)
    grid = 256 * 1281 * 2560 * 4
    work = 640 * 2 * 641 * 256 * 8
    assert bench.fft_bytes(T639, 256, 4) == grid + work
    assert grid + work == 5_038_407_680   # 5.04 GB
    # a reduced grid counts its own points; the workspace is unchanged
    assert bench.fft_bytes(T639, 256, 4, npts=2_567_936) == 256 * 2_567_936 * 4 + work
    # FP64 doubles both
    assert bench.fft_bytes(T639, 256, 8) == 2 * (grid + work)


def test_legendre_flops_by_hand():
    # 2 flops per (coefficient, northern node, real column)
    ncoef = 640 * 641 // 2
    assert bench.legendre_flops(T639, 256) == 2.0 * ncoef * 641 * 512
    w = W.WORKLOADS["T31"]
    assert bench.legendre_flops(w, 1) == 2.0 * (32 * 33 // 2) * 33 * 2


def test_split_gemm_table_bytes_by_hand():
    # T31, one field: the forward table has rows padded to 8 and K = 33
    # northern nodes padded to 48 (three 16-node slabs), per (m, parity)
    w = W.WORKLOADS["T31"]
    N, Jh, C = 31, 33, 2
    tab = 0
    for m in range(N + 1):
        for q in range(2):
            d = N - m - q
            R = d // 2 + 1 if d >= 0 else 0
            tab += ((R + 7) // 8 * 8) * 48 * 2
    work = (N + 1) * 2 * Jh * C * 4
    spec = (N + 1) * (N + 2) // 2 * C * 4
    assert bench.split_gemm_bytes(w, 1, "bf16x3", False) == work + spec + 3 * tab
    assert bench.split_gemm_bytes(w, 1, "bf16x2", False) == work + spec + 2 * tab


def test_roofline_of_an_fft_stage():
    # 100 launches in 163.0 ms: 1.63 ms each
    r = bench.roofline_for("fft_inverse", 163.0, 100, T639, 256, "bf16x3", PEAKS, "measured")
    want = bench.fft_bytes(T639, 256, 4) / 1.63e-3 / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(want)
    assert r["frac"] == pytest.approx(want / 6800.0)
    assert r["ms_per_launch"] == pytest.approx(1.63)
    # the stored DRAM traffic applies to the regular grid's kernel only
    assert r["traffic"] == pytest.approx(bench.MEASURED_TRAFFIC[("fft_inverse", "bf16x3",
                                                                 "T639", 256)])
    red = bench.roofline_for("fft_inverse", 140.0, 100, T639, 256, "bf16x3", PEAKS,
                             "measured", npts=2_567_936, grid="reduced")
    assert red["traffic"] is None
    assert red["achieved"] == pytest.approx(
        bench.fft_bytes(T639, 256, 4, npts=2_567_936) / 1.4e-3 / 1e9)


def test_roofline_of_the_fp64_and_split_contractions():
    r = bench.roofline_for("legendre_forward", 12060.0, 100, T639, 256, "fp64", PEAKS, "m")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == 1.25
    assert r["achieved"] == pytest.approx(bench.legendre_flops(T639, 256) / 0.1206 / 1e12)
    s = bench.roofline_for("legendre_forward", 123.7, 100, T639, 256, "bf16x3", PEAKS, "m")
    t_frac = 6 * bench.legendre_flops(T639, 256) / 1.237e-3 / 1e12 / 1700.0
    h_frac = bench.split_gemm_bytes(T639, 256, "bf16x3", False) / 1.237e-3 / 1e9 / 6800.0
    # the larger of the two fractions names the bound
    assert s["bound"] == ("hbm" if h_frac >= t_frac else "tensor")
    assert s["frac"] == pytest.approx(max(h_frac, t_frac))


def test_job_throughput_counts_all_ranks():
    # 2 ranks x 256 field-levels x 100 steps in 5600 ms
    assert bench.job_throughput(2, 256, 100, 5600.0) == pytest.approx(2 * 256 * 100 / 5.6)


def test_step_bytes_is_both_ffts_and_both_contractions():
    want = (2 * bench.fft_bytes(T639, 256, 4) + bench.split_gemm_bytes(T639, 256, "bf16x3", False)
            + bench.split_gemm_bytes(T639, 256, "bf16x3", True))
    assert bench.step_bytes(T639, 256, "bf16x3") == want
    # the ensemble's grouped pair is the members' steps
    assert bench.group_pair_bytes(W.ENSEMBLE, "bf16x3") == sum(
        bench.step_bytes(w, w.F, "bf16x3") for w in W.ENSEMBLE)


def test_fp64_roofline_uses_the_measured_pipe_peak():
    pk = dict(PEAKS, fp64_tflops=1.3, dfma_probe=1.3, dgemm=1.1)
    r = bench.roofline_for("legendre_forward", 12060.0, 100, T639, 256, "fp64", pk, "m")
    assert r["peak"] == 1.3 and "measured" in r["peak_source"]
    assert r["frac"] == pytest.approx(r["achieved"] / 1.3)


def test_both_arms_name_the_same_workload():
    args = bench.parse_args([])
    native = bench.workload_config(T639, 256, args, T639.J * T639.I, 4, 1)
    ref = bench.workload_config(T639, 256, args, T639.J * T639.I, 4, args.gpus)
    assert native == ref
    assert native["workload"] == "T639" and native["field_levels_per_gpu"] == 256


def test_oracle_sample_excludes_table_construction():
    # the tables are built by oracle_tables, before and outside the timer;
    # the sample then only transforms
    w = W.WORKLOADS["T31"]
    ms, tables = bench.oracle_tables(w, 4)
    assert ms == list(range(0, 32, 4)) and sorted(tables) == ms
    sec, frac = bench.oracle_sample(w, ms, tables)
    assert sec > 0 and frac == pytest.approx(sum(32 - m for m in ms) / (32 * 33 // 2))


def test_alias_step_bytes_by_hand():
    # three syntheses and two analyses of F fields, plus the U and V grids
    # read and the two product grids written inside W's inverse FFT (in
    # place of W's grid: three grid passes more than the five transforms)
    w = W.ALIAS
    F = 64
    grid = F * w.J * w.I * 4
    inv = bench.fft_bytes(w, F, 4) + bench.split_gemm_bytes(w, F, "bf16x3", True)
    fwd = bench.fft_bytes(w, F, 4) + bench.split_gemm_bytes(w, F, "bf16x3", False)
    assert bench.alias_step_bytes(w, F, "bf16x3") == 3 * inv + 2 * fwd + 3 * grid
