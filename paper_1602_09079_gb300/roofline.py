"""Algorithmic work of the DG kernels, counted from their loop bounds.

Per cell and per RK stage (k = degree, N = N(k), Q = k+1, Q2 = Q^2,
Q3 = Q^3; FMA = 2 flops; sqrt and division count as one flop each):

faces, dense count (3 faces per cell, Q2 points each; face_flops)
    traces of both sides  2 x 5 x N FMA           -> 20 N
    HLLC flux                                      -> HLLC_FLOPS
face_sf64_kernel (sum-factorised traces; face_sf_flops)
    normal contraction    2 x 5 N FMA per face
    tangential expansion  2 x 5 (Q T + Q2 (k+1)) FMA per face, then HLLC
volume_sf_kernel (sum factorisation; T = (k+1)(k+2)/2, KP = k+1)
    point values          5 (Q N + Q2 T + Q3 KP) FMA
    Euler fluxes, scaling Q3 x 46;   source  Q3 x 12 (forcing only)
    gradient projection   15 KP Q3 + 5 T Q (2Q + Q) + 5 N 2Q FMA
    source projection     4 (KP Q3 + T Q2 + N Q) FMA (forcing only)
    face projection       30 (Q2 KP + T Q) FMA + 30 T + 5 N x 6 FMA
    stage combination     5 N x 5;  limiter screen ~ 10 N + 30 (RK stage only)
volume_kernel (dense quadrature; the FP32 tiled kernel follows the same counts)
    point values          Q3 x 5 N FMA            -> 10 N Q3
    Euler fluxes, scaling Q3 x 46                  (1 div, velocity,
                                                    pressure, 3 fluxes, 1/dx)
    source                Q3 x 8                   (forcing only)
    volume projection     5 x 3 Q3 N FMA           -> 30 Q3 N
    source projection     4 x Q3 N FMA             -> 8 Q3 N (forcing only)
    face projection       5 x 3 Q2 (2 + 2 N FMA)   -> 15 Q2 (2 + 4 N)
    stage combination     5 N x 5                  (RK stage only)
    limiter screen        ~ 10 N + 30              (RK stage only)

Algorithmic roofline of one RK stage (the method's own work, whatever
form a kernel takes): read y_s, read y_0 (stages 2-3), write y_{s+1}, FP64,
on average 8/3 x 5 N x 8 bytes per cell (stage_min_bytes); the
sum-factorised volume and face flop counts (stage_flops). The fused
FP32-mixed stage kernel's own traffic (fused_impl_bytes) reads y_s and the
FP32 increment d instead of y_0, and the cached driving field.

Peaks: HBM from MEASURED_PEAKS.json; FP32 152 SMs x 128 FMA lanes x 2
flops x 2.07 GHz (unit counts and maximum clock of the GB300); FP64 the
GB300's nominal 1.25 TFLOP/s.

Kernel bytes (unique data each launch must touch):
    face:   read y_s (5 N x 8) + write face fluxes (15 Q2 x sizeof(T))
    volume: read y_s, y_0 (stages 2-3), face fluxes, forcing field
            (3 Q3 x sizeof(T)), write y_{s+1} (5 N x 8 each); the FP32 stage
            kernels also read and write the FP32 shadow (5 N x 4 each)
"""
from __future__ import annotations

HLLC_FLOPS = 120


def _dims(k):
    N = (k + 1) * (k + 2) * (k + 3) // 6
    Q = k + 1
    return N, Q, Q * Q, Q * Q * Q


def face_flops(k):
    N, Q, Q2, Q3 = _dims(k)
    return 3 * Q2 * (20 * N + HLLC_FLOPS)


def face_sf_flops(k):
    """face_sf64_kernel: per face, 2 x 5 N FMA along the normal, then per
    side 5 (Q T + Q^2 (k+1)) FMA for the Q^2 points, and the flux."""
    N, Q, Q2, Q3 = _dims(k)
    T = (k + 1) * (k + 2) // 2
    return 3 * (2 * (2 * 5 * N) + 2 * 2 * 5 * (Q * T + Q2 * (k + 1)) + Q2 * HLLC_FLOPS)


def volume_flops(k, forcing, stage=True):
    N, Q, Q2, Q3 = _dims(k)
    f = 10 * N * Q3 + 46 * Q3 + 30 * Q3 * N + 15 * Q2 * (2 + 4 * N)
    if forcing:
        f += 8 * Q3 + 8 * Q3 * N
    if stage:
        f += 25 * N + 10 * N + 30
    return f


def volume_sf_flops(k, forcing, stage=True):
    N, Q, Q2, Q3 = _dims(k)
    T, KP = (k + 1) * (k + 2) // 2, k + 1
    fma = 5 * (Q * N + Q2 * T + Q3 * KP)
    fma += 15 * KP * Q3 + 5 * T * Q * 3 * Q + 5 * N * 2 * Q
    fma += 30 * (Q2 * KP + T * Q) + 5 * N * 6
    f = 2 * fma + 46 * Q3 + 30 * T
    if forcing:
        f += 12 * Q3 + 2 * 4 * (KP * Q3 + T * Q2 + N * Q)
    if stage:
        f += 25 * N + 10 * N + 30
    return f


def face_bytes(k, tsize):
    N, Q, Q2, Q3 = _dims(k)
    return 5 * N * 8 + 15 * Q2 * tsize


def volume_bytes(k, tsize, forcing, reads_y0=True, shadow=False):
    """shadow: the FP32 stage kernels also read the stage input's FP32
    shadow and write the output's (5 N x 4 bytes each way)."""
    N, Q, Q2, Q3 = _dims(k)
    b = 5 * N * 8 * (3 if reads_y0 else 2) + 15 * Q2 * tsize
    if forcing:
        b += 3 * Q3 * tsize
    if shadow:
        b += 2 * 5 * N * 4
    return b


def reset_bytes(k, mixed):
    """energy_reset_kernel: reads the four FP64 means and the other density
    and momentum coefficients (FP32 shadow on the mixed path, FP64
    otherwise) and the old energy mean; writes the N energy modes (FP64,
    plus their FP32 shadow on the mixed path)."""
    N = (k + 1) * (k + 2) * (k + 3) // 6
    if mixed:
        return 4 * 8 + 4 * (N - 1) * 4 + 8 + N * (8 + 4)
    return 4 * N * 8 + 8 + N * 8


def cfl_bytes():
    """cfl_kernel: the five means of each cell."""
    return 5 * 8


def step_bytes(k, mixed, forcing=True):
    """Algorithmic HBM bytes per cell of one benchmark step: the CFL
    reduction, three stages of face fluxes and volume kernel, and the energy
    reset. Mixed path: the face kernel reads the FP32 shadow and writes FP32
    fluxes; the first stage's volume kernel skips y_0."""
    N, Q, Q2, Q3 = _dims(k)
    if mixed:
        faces = 3 * (5 * N * 4 + 15 * Q2 * 4)
        vol = (volume_bytes(k, 4, forcing, reads_y0=False, shadow=True)
               + 2 * volume_bytes(k, 4, forcing, shadow=True))
    else:
        faces = 3 * face_bytes(k, 8)
        vol = 3 * volume_bytes(k, 8, forcing)
    return cfl_bytes() + faces + vol + reset_bytes(k, mixed)


def step_flops(k, forcing):
    """Per cell per SSP-RK3 step (3 stages), both RHS kernels."""
    return 3 * (face_flops(k) + volume_flops(k, forcing))


def step_min_bytes(k):
    """Minimum HBM traffic per cell per step of a fully fused stage: read
    y_s, read y_0 on stages 2-3, write y_{s+1} (FP64 state)."""
    N = (k + 1) * (k + 2) * (k + 3) // 6
    return (3 + 2 + 3) * 5 * N * 8


FP32_PEAK = 152 * 128 * 2 * 2.07e9
FP64_PEAK = 1.25e12
PEAK_SOURCE = ("HBM: MEASURED_PEAKS.json hbm_gbs (measured copy); FP32: 152 SM x 128 lanes x 2 flops x "
               "2.07 GHz (unit counts, maximum clock); FP64: nominal 1.25 TFLOP/s of the GB300")


def stage_min_bytes(k):
    """Algorithmic HBM bytes per cell of one RK stage, averaged over the
    three stages: read y_s, y_0 (stages 2-3), write y_{s+1} in FP64."""
    return step_min_bytes(k) / 3


def stage_flops(k, forcing):
    """Algorithmic flops per cell of one RK stage: the sum-factorised volume
    integral (with the driving source when forcing) and the three faces a
    cell owns, traces and numerical flux included."""
    return volume_sf_flops(k, forcing) + face_sf_flops(k)


def fused_impl_bytes(k, forcing):
    """HBM bytes per cell the fused FP32-mixed stage kernel moves, averaged
    over the three stages: every stage reads y_s (FP64) and the driving
    field (FP32) and writes y_{s+1} (FP64); stages 1-2 write the FP32
    increment d, stages 2-3 read it; stage 3 writes the FP32 shadow.
    Neighbour coefficients are re-read from L2 and not counted."""
    N, Q, Q2, Q3 = _dims(k)
    st, f32 = 5 * N * 8, 5 * N * 4
    fld = 3 * Q3 * 4 if forcing else 0
    s1 = st + fld + st + f32
    s2 = st + f32 + fld + st + f32
    s3 = st + f32 + fld + st + f32
    return (s1 + s2 + s3) / 3


def stage_roofline(k, forcing, nc, stage_ms, hbm_gbs, fp_peak):
    """Roofline entry of one RK stage: the larger of the algorithmic flops
    over the ALU peak and the algorithmic bytes over the HBM peak is the
    bound; achieved = that quantity over the measured stage time."""
    sec = stage_ms * 1e-3
    flops = stage_flops(k, forcing) * nc
    byts = stage_min_bytes(k) * nc
    t_alu = flops / fp_peak
    t_hbm = byts / (hbm_gbs * 1e9) if hbm_gbs else 0.0
    out = {"flops_per_launch": flops, "bytes_per_launch": byts, "ms_per_launch": stage_ms,
           "achieved_tflops": flops / sec / 1e12, "achieved_gbs": byts / sec / 1e9,
           "roofline_ms": max(t_alu, t_hbm) * 1e3}
    if t_alu >= t_hbm:
        out.update({"bound": "alu", "achieved": flops / sec / 1e12, "peak": fp_peak / 1e12, "unit": "TFLOP/s",
                    "frac": t_alu / sec})
    else:
        out.update({"bound": "hbm", "achieved": byts / sec / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                    "frac": t_hbm / sec})
    return out
