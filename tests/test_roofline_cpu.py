"""Algorithmic byte counts of the benchmark step (roofline.step_bytes), from
the data each kernel must touch: FP64 state rows (5 N x 8 B per cell), the
FP32 shadow (5 N x 4 B), face fluxes (15 Q^2 per cell, 4 or 8 B), the cached
driving field (3 Q^3), and bench.py's whole-step roofline entry built on
them."""
import bench
from paper_1602_09079_gb300 import roofline as rl


def dims(k):
    return (k + 1) * (k + 2) * (k + 3) // 6, (k + 1) ** 2, (k + 1) ** 3


def test_mixed_step_bytes_by_hand():
    for k in (1, 2, 3):
        N, Q2, Q3 = dims(k)
        state, shadow, flux32, field32 = 5 * N * 8, 5 * N * 4, 15 * Q2 * 4, 3 * Q3 * 4
        faces = 3 * (shadow + flux32)  # read the shadow, write the fluxes
        # stage 1 reads y_s (not y_0); every stage reads the fluxes, the
        # field and the shadow, writes y_{s+1} and its shadow
        v1 = 2 * state + flux32 + field32 + 2 * shadow
        v23 = 3 * state + flux32 + field32 + 2 * shadow
        reset = 4 * 8 + 4 * (N - 1) * 4 + 8 + N * 12
        assert rl.step_bytes(k, True) == 40 + faces + v1 + 2 * v23 + reset
    assert rl.step_bytes(2, True) == 9556


def test_fp64_step_bytes_by_hand():
    for k in (1, 2, 3):
        N, Q2, Q3 = dims(k)
        state, flux64, field64 = 5 * N * 8, 15 * Q2 * 8, 3 * Q3 * 8
        faces = 3 * (state + flux64)
        vol = 3 * (3 * state + flux64 + field64)
        reset = 4 * N * 8 + 8 + N * 8
        assert rl.step_bytes(k, False) == 40 + faces + vol + reset


def test_stage_algorithmic_counts_by_hand():
    """Algorithmic bytes of a stage: read y_s, y_0 (stages 2-3), write y_{s+1} in FP64, i.e.
    8/3 x 5 N x 8 bytes per cell per stage; flops: the sum-factorised volume
    integral with the source and three owned faces."""
    for k in (1, 2, 3):
        N = dims(k)[0]
        assert abs(rl.stage_min_bytes(k) - 8 / 3 * 5 * N * 8) <= 1e-9
        assert rl.stage_flops(k, True) == rl.volume_sf_flops(k, True) + rl.face_sf_flops(k)
    assert round(rl.stage_min_bytes(2)) == 1067
    assert rl.stage_flops(2, True) == 13046 + 6540
    # the fused kernel's own traffic: y_s, field, y_{s+1} every stage; d
    # written in stages 1-2 and read in 2-3; the shadow written in stage 3
    N, Q2, Q3 = dims(2)
    st, f32, fld = 5 * N * 8, 5 * N * 4, 3 * Q3 * 4
    assert abs(rl.fused_impl_bytes(2, True) - (3 * (2 * st + fld) + 4 * f32 + f32) / 3) <= 1e-9


def test_stage_roofline_entry():
    nc = 128 ** 3
    e = rl.stage_roofline(2, True, nc, 2.0, 6791.7, rl.FP32_PEAK)
    t_alu = rl.stage_flops(2, True) * nc / rl.FP32_PEAK
    t_hbm = rl.stage_min_bytes(2) * nc / 6791.7e9
    assert t_alu > t_hbm and e["bound"] == "alu" and e["unit"] == "TFLOP/s"
    assert abs(e["frac"] - t_alu / 2e-3) <= 1e-12
    assert abs(e["achieved"] / e["peak"] - e["frac"]) <= 1e-12
    assert abs(rl.FP32_PEAK - 80.54784e12) <= 1.0
    # FP64: the ALU time dominates too
    f = rl.stage_roofline(2, True, nc, 50.0, 6791.7, rl.FP64_PEAK)
    assert f["bound"] == "alu" and abs(f["frac"] - rl.stage_flops(2, True) * nc / 1.25e12 / 0.05) <= 1e-12


def test_step_roofline_entry():
    nc = 128 ** 3
    N = dims(2)[0]
    byts = (3200 + (5 * N + 1) * 8 + 40) * nc
    flops = 3 * rl.stage_flops(2, True) * nc
    r = bench.step_roofline(2, True, nc, 8.0, 6780.0)
    assert r["bytes_per_step"] == byts and r["flops_per_step"] == flops
    assert r["bound"] == "alu" and abs(r["frac"] - flops / rl.FP32_PEAK / 8e-3) <= 1e-12
    f = bench.step_roofline(2, False, nc, 173.0, 6780.0)
    assert f["bound"] == "alu" and abs(f["frac"] - flops / 0.173 / 1.25e12) <= 1e-12
    assert bench.step_roofline(1, True, 512, 1.0, None)["frac"] is None
