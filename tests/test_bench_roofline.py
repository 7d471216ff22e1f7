"""bench.py's roofline arithmetic against the per-unit work stated for each kernel:
the Jacobian's basis contraction (332.8 kFLOP per element at p = 3), the folded FP64
stage operator (3 nb^2 FMAs per element, FP64-ALU bound) and its FP32 twin (3 nb^2 + 5 nb
words per element, HBM bound)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

C1 = dict(p=3)
PEAKS = {"hbm_gbs": 6700.0}


def _res(kern_ms, launches=10, ne=2048, config="c1"):
    return dict(ne=ne, kern_launches=launches, kern_ms=kern_ms, config=config)


def test_jacobian_contraction_flops():
    r = bench.roofline_for("jacobian", _res(kern_ms=10.0), PEAKS, 1.0, C1)   # 1 ms per launch
    assert abs(r["achieved"] - 2048 * 332.8e3 / 1e-3 / 1e12) < 1e-9
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"


def test_folded_fp64_operator_flops_and_traffic():
    nb = 40
    r = bench.roofline_for("stage_op", _res(kern_ms=0.3), PEAKS, 1.0, C1)   # 30 us per launch
    assert abs(r["achieved"] - 2.0 * 2048 * 3 * nb * nb / 30e-6 / 1e12) < 1e-9
    assert r["bound"] == "alu" and r["frac"] == r["achieved"]
    assert r["traffic"] == bench.MEASURED_TRAFFIC[("stage_op", "c1")]
    assert abs(r["hbm_gbs_equiv"] - 2048 * (3 * nb * nb + 5 * nb) * 8 / 30e-6 / 1e9) < 1e-6


def test_folded_fp32_operator_bytes():
    nb = 40
    r = bench.roofline_for("stage_op32", _res(kern_ms=0.1), PEAKS, 1.0, C1)  # 10 us per launch
    assert r["bound"] == "hbm"
    assert abs(r["achieved"] - 2048 * (3 * nb * nb + 5 * nb) * 4 / 10e-6 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6700.0) < 1e-12
    assert r["traffic"] is None                      # no capture of this class on file


def test_l2_note_flags_small_working_sets():
    from pp_inputs import CONFIGS
    assert "far larger than L2" in bench.l2_note(dict(ne=2048, Nt=100), CONFIGS["c1"], "fp64")
    assert "not a bench value" in bench.l2_note(dict(ne=64, Nt=20), CONFIGS["c0"], "fp64")
