"""Host-side logic of bench.py (CPU): the per-stage roofline figures, the
peak selection and the host-link byte count that the JSON line reports."""
import math

import bench

PK = {"hbm_gbs": 6468.0, "bf16_tflops": 1777.7, "bf16_tflops_sustained": 1372.4, "source": "measured"}


def test_stage_rooflines_with_the_assembly_inside_conv1():
    # stage 0 (the separate assembly) holds no kernel when conv1 assembles
    # its own input: no prep entry, conv1..4 and the reconstruction remain
    stages = [0.01, 0.134, 0.240, 0.435, 0.171, 0.129]
    r = bench.stage_rooflines(stages, "bf16", PK, fused_prep=True)
    assert set(r) == {"conv1", "conv2", "conv3", "conv4", "reconstruct"}
    conv3 = r["conv3"]
    flops = 2.0 * 48 * 64 * 25 * 1080 * 1920
    assert math.isclose(conv3["achieved"], flops / (0.435e-3) / 1e12, rel_tol=1e-12)
    assert math.isclose(conv3["frac"], conv3["achieved"] / PK["bf16_tflops"], rel_tol=1e-12)
    rec = r["reconstruct"]
    assert rec["bound"] == "hbm" and rec["unit"] == "GB/s"
    assert math.isclose(rec["achieved"], 84 * 1080 * 1920 / 0.129e-3 / 1e9, rel_tol=1e-12)


def test_stage_rooflines_with_a_separate_assembly_kernel():
    stages = [0.064, 0.123, 0.240, 0.435, 0.171, 0.129]
    r = bench.stage_rooflines(stages, "bf16", PK, fused_prep=False)
    assert "prep" in r and r["prep"]["bound"] == "hbm"
    # 40 B/px of FP32 frames in, 64 B/px of BF16 hi/lo out
    assert math.isclose(r["prep"]["achieved"], 104 * 1080 * 1920 / 0.064e-3 / 1e9, rel_tol=1e-12)


def test_fp8_and_fp32_peaks():
    stages = [0.0, 0.138, 0.204, 0.364, 0.147, 0.127]
    r8 = bench.stage_rooflines(stages, "fp8", PK, fused_prep=True)
    assert math.isclose(r8["conv3"]["frac"], r8["conv3"]["achieved"] / (2 * PK["bf16_tflops"]), rel_tol=1e-12)
    r32 = bench.stage_rooflines([0.06, 0.8, 3.3, 7.2, 2.4, 0.13], "fp32", PK)
    peak = 148 * 128 * 2 * 2032e6 / 1e12
    assert r32["conv3"]["bound"] == "alu"
    assert math.isclose(r32["conv3"]["frac"], r32["conv3"]["achieved"] / peak, rel_tol=1e-12)


def test_tensor_peak_follows_the_power_cap():
    assert bench.tensor_peak(PK, {"reasons": ["sw_power_cap"], "window_ms": 300.0}) == (1372.4, "sustained")
    assert bench.tensor_peak(PK, {"reasons": [], "window_ms": 1500.0}) == (1372.4, "sustained")
    assert bench.tensor_peak(PK, {"reasons": [], "window_ms": 200.0}) == (1777.7, "burst")


def test_host_upload_bytes_are_the_frame_inputs_once():
    # 10 float32 channels per pixel cross the host link once per frame
    assert bench.host_upload_bytes(1080, 1920) == 82_944_000
