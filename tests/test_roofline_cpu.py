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


def test_step_roofline_entry():
    nc = 128 ** 3
    r = bench.step_roofline(2, True, nc, 12.4, 6780.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 9556 * nc / 12.4e-3 / 1e9) <= 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 6780.0) <= 1e-15
    f = bench.step_roofline(2, False, nc, 173.0, 6780.0)
    flops = 3 * (rl.face_sf_flops(2) + rl.volume_sf_flops(2, True)) * nc
    assert f["bound"] == "alu" and f["flops_per_step"] == flops
    assert abs(f["frac"] - flops / 0.173 / 1.25e12) <= 1e-12
    assert bench.step_roofline(1, True, 512, 1.0, None)["frac"] is None
