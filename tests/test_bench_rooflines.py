"""The per-phase roofline fractions of the bench line rate each phase against the unit it runs on:
the FP64 mode's FMM passes run in double-FP32 on the FP32 pipe (15 FP32 operations per
multiply-add) and its nearfield as products of 16 residues on the tensor cores (32 B per stored
element); the mixed mode's passes on the FP32 pipe and its nearfield as 3 FP16 products (4 B per
element).  Inputs: the 12288-triangle x 256-step workload's tree and phase times as measured."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

NT, ET, MX, MT = 12288, 256, 6, 4
INFO = {"p": 7, "nbox": [1, 1, 1, 1, 8, 8, 56, 56], "m2l_flops": 3.136014e9,
        "nearfield_v_elements": 603979776, "nf_tensor_cores": 3}
PEAKS = {"hbm_gbs": 6653.7, "fp16_tflops": 1899.0, "fp64_tflops": 1.0556, "fp32_tflops": 75.40}
FP64_PHASES = {"nearfield": 4.3805, "s2m": 0.2696, "m2l": 1.9429, "l2t": 0.2059}
MIXED_PHASES = {"nearfield": 0.8503, "s2m": 0.0845, "m2l": 0.631, "l2t": 0.0644}


def test_fp64_mode_phases_against_the_units_they_run_on():
    rl = bench.phase_rooflines(FP64_PHASES, INFO, 8, NT, ET, MX, MT, PEAKS, arith="df64")
    df = PEAKS["fp32_tflops"] / bench.DF64_FP32_OPS_PER_MAC
    m2l = INFO["m2l_flops"] / (FP64_PHASES["m2l"] * 1e-3) / 1e12
    assert rl["m2l"]["fp_peak_tflops"] == pytest.approx(df)
    assert rl["m2l"]["frac_fp"] == pytest.approx(m2l / df)
    nel, dof = INFO["nearfield_v_elements"], NT * ET
    nf = rl["nearfield"]
    assert nf["bytes"] == pytest.approx(32.0 * nel + 48.0 * dof)
    assert nf["frac_hbm"] == pytest.approx(nf["bytes"] / (FP64_PHASES["nearfield"] * 1e-3) / 1e9 / PEAKS["hbm_gbs"])
    assert nf["fp_peak_tflops"] == pytest.approx(PEAKS["fp16_tflops"] / 16)
    assert nf["bound"] == "hbm"
    for ph in ("s2m", "l2t", "m2l", "nearfield"):  # measured phases cannot exceed their unit's peak
        assert 0.0 < rl[ph]["frac_fp"] < 1.0 and 0.0 < rl[ph]["frac_hbm"] < 1.0, (ph, rl[ph])


def test_mixed_mode_phases():
    rl = bench.phase_rooflines(MIXED_PHASES, INFO, 4, NT, ET, MX, MT, PEAKS, arith="fp32")
    assert rl["m2l"]["fp_peak_tflops"] == PEAKS["fp32_tflops"]
    nf = rl["nearfield"]
    assert nf["bytes"] == pytest.approx(4.0 * INFO["nearfield_v_elements"] + 16.0 * NT * ET)
    assert nf["fp_peak_tflops"] == pytest.approx(PEAKS["fp16_tflops"] / 3)
    for ph in ("s2m", "l2t", "m2l", "nearfield"):
        assert 0.0 < rl[ph]["frac_fp"] < 1.0 and 0.0 < rl[ph]["frac_hbm"] < 1.0, (ph, rl[ph])


def test_native_fp64_and_cuda_core_nearfield_use_the_fp64_pipe():
    info = dict(INFO, nf_tensor_cores=0)
    rl = bench.phase_rooflines({"nearfield": 246.0, "m2l": 7.8}, info, 8, NT, ET, MX, MT, PEAKS)
    assert rl["m2l"]["fp_peak_tflops"] == PEAKS["fp64_tflops"]
    assert rl["nearfield"]["fp_peak_tflops"] == PEAKS["fp64_tflops"]
    assert rl["nearfield"]["bytes"] == pytest.approx(8.0 * INFO["nearfield_v_elements"] + 16.0 * NT * ET)
    assert "s2m" not in rl  # phases without a time are left out
