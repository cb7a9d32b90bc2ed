"""The bench's ALU roofline for the binary64 Stage 1 (CPU only)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_stage1_op_count_against_the_executed_instructions():
    """Per block of 16 rows the kernel executes 73 DMUL and 106 DFMA (ncu,
    profiles/stage1_keep_f64_N2e23_full.md): the algorithmic count has exactly
    those MULs and no more FMAs than were executed."""
    import bench

    fma, mul = bench.stage1_f64_ops(16)
    assert mul == 73
    assert fma == 101 and fma <= 106
    # per row: 12 - 18/s operations, 19 - 29/s flops, for every block size
    for s in (4, 8, 16, 32, 64):
        f, m = bench.stage1_f64_ops(s)
        assert f + m == 12 * s - 18
        assert 2 * f + m == 19 * s - 29


def test_stage1_roofline_fields():
    import bench

    r = bench.stage1_f64_roofline(1.368, 1 << 26, 16, 6681.8, None)
    assert r["bound"] == "alu" and r["unit"] == "Gop/s"
    assert abs(r["peak"] - 152 * 2.07 * 2) < 1e-9
    assert abs(r["achieved"] - 10.875 * (1 << 26) / 1.368e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert 0.84 < r["frac"] < 0.86 and 0.66 < r["frac_flops"] < 0.68
    assert r["algorithmic_bytes_per_row"] == 60.0
