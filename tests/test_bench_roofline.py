"""bench.py's roofline arithmetic against the per-unit work stated for each timed kernel:
the folded FP64 stage operator (3 nb^2 FMAs per element, FP64-ALU bound), its FP32 twin
(3 nb^2 + 5 nb words per element, HBM bound), and the Gram-Schmidt passes of an Arnoldi
step (counted algorithmic bytes over their summed time); and the L2 note."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

C1 = dict(p=3)
PEAKS = {"hbm_gbs": 6700.0}


def _res(kernel, ms, launches=10, counted=0.0, ne=2048, config="c1"):
    return dict(ne=ne, config=config, kern={kernel: (launches, ms, counted)})


def test_folded_fp64_operator_flops():
    nb = 40
    r = bench.roofline_for("stage_op", _res("stage_op", 0.3), PEAKS, 1.0, C1, False)   # 30 us per launch
    assert abs(r["achieved"] - 2.0 * 2048 * 3 * nb * nb / 30e-6 / 1e12) < 1e-9
    assert r["bound"] == "alu" and r["frac"] == r["achieved"]
    assert abs(r["hbm_gbs_equiv"] - 2048 * (3 * nb * nb + 5 * nb) * 8 / 30e-6 / 1e9) < 1e-6


def test_folded_fp32_operator_bytes():
    nb = 40
    r = bench.roofline_for("stage_op32", _res("stage_op32", 0.1), PEAKS, 1.0, C1, False)  # 10 us per launch
    assert r["bound"] == "hbm"
    assert abs(r["achieved"] - 2048 * (3 * nb * nb + 5 * nb) * 4 / 10e-6 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6700.0) < 1e-12


def test_arnoldi_bytes_over_time():
    # 40 launches of an Arnoldi step family taking 1 ms in total, 3.3e9 counted bytes
    r = bench.roofline_for("arnoldi", _res("arnoldi", 1.0, launches=40, counted=3.3e9), PEAKS, 1.0, C1, False)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 3.3e9 / 1e-3 / 1e9) < 1e-9
    assert abs(r["avg_us"] - 25.0) < 1e-9


def test_l2_note_states_the_per_stage_working_set():
    from pp_inputs import CONFIGS
    note = bench.l2_note(dict(ne=2048, Nt=100, nu=81920), CONFIGS["c1"], "fp64")
    assert "L2" in note and "no flush" in note
    assert "105 MB" in note         # 4 nb^2 FP64 words per element: folded operator + inverse
