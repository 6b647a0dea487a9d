"""bench.py's roofline model on the host: which kernel and bound each stage reports for each
solver path, the algorithmic work per system, and the rule that a recorded DRAM traffic figure
only describes the kernel source it was captured from."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

N, NT = 1323, 64


def _one(stage, n, mixed, band=0):
    m = bench.stage_model(stage, n, NT, mixed, band)
    assert m is not None and len(m) >= 1
    return m


def test_band_path_chase_is_an_alu_bound_on_the_fp32_units():
    (bnd, work, peak, unit, _, kern), = _one("hetrd", N, True, 63)
    assert (bnd, unit, kern) == ("alu", "TFLOP/s", "k_sbr_chase")
    assert work == 24.0 * 63 * N ** 2  # 6 b^2 complex MACs per step over n^2 / (2b) steps
    assert peak == bench.FP32_ALU_PEAK


def test_dense_reduction_reports_both_bounds():
    m = _one("hetrd", N, True)
    kinds = {b[0]: b for b in m}
    assert set(kinds) == {"alu", "hbm"} and all(b[5] == "k_hetrd" for b in m)
    assert kinds["alu"][1] == 16.0 / 3.0 * N ** 3
    assert kinds["hbm"][1] == 8.0 * N ** 3 / 6.0       # FP32 triangle reads
    assert _one("hetrd", N, False)[1][1] == 16.0 * N ** 3 / 6.0  # FP64


def test_back_transform_kernels_follow_the_path_and_precision():
    def kern(n, mixed, band):
        return [(b[0], b[5]) for b in _one("backtransform", n, mixed, band)]
    assert kern(N, True, 63) == [("tensor", "k_sbr_bt_tc")]      # band, b in 33..64
    assert kern(N, True, 16) == [("alu", "k_sbr_bt_f32")]        # band, narrow
    assert kern(N, False, 63) == [("alu", "k_sbr_bt_f64")]
    assert kern(N, True, 0) == [("tensor", "k_tf3_gemm")]        # dense, n >= 256
    assert kern(200, True, 0) == [("alu", "k_backtransform_f32")]
    assert kern(N, False, 0) == [("alu", "k_backtransform")]
    tc = _one("backtransform", N, True, 63)[0]
    assert tc[1] == 8.0 * N ** 3
    assert abs(tc[2] - bench._peaks().get("bf16_tflops_sustained", bench._peaks()["bf16_tflops"]) * 1e12
               * 1.1 / 2.25) < 1.0


def test_refinement_gram_stage_is_the_band_gram():
    (bnd, work, _, _, _, kern), = _one("refine_gram", N, True)
    assert (bnd, kern) == ("alu", "k_gram_band_df32") and work == 264.0 * N ** 2
    assert bench.stage_model("refine_gram", N, NT, False) is None  # no refinement in FP64


def test_measured_traffic_is_tied_to_the_captured_source():
    assert bench._measured_traffic("no_such_kernel", bench.WORKLOAD, "mixed") is None
    for (kern, wl, prec), (_, path, _) in bench.MEASURED_TRAFFIC.items():
        assert os.path.exists(os.path.join(ROOT, path))
        assert bench._measured_traffic(kern, wl, "fp64" if prec == "mixed" else "mixed") is None
    saved = dict(bench.MEASURED_TRAFFIC)
    try:
        # a record whose hash does not match the source on disk reports nothing
        k = next(iter(saved))
        v, path, _ = saved[k]
        bench.MEASURED_TRAFFIC[k] = (v, path, "0" * 64)
        assert bench._measured_traffic(*k) is None
    finally:
        bench.MEASURED_TRAFFIC.clear()
        bench.MEASURED_TRAFFIC.update(saved)
