"""Driven isothermal-like turbulence runs through the library (arXiv:1602.09079,
Sect. 3-4): the setting of the paper's subsonic simulations, with its
diagnostics recorded over time.

Start from rest (rho = 1, p = 1/gamma, so c = 1), OU driving on the modes
1 <= |n| <= 2 (Sect. 3.1) updated every 0.1 t_s with t_s = L / (2 M c), the
energy reset to the isothermal internal energy after every step (Sect. 3.2,
gamma = 1.01 by default as in the paper), and per step: the injected work of
the driving force (trapezoidal in time over the step, from dg_diagnostics'
power), the dissipated energy the reset reports, and at record times the rms
Mach number and kinetic energy of the cell means (Sect. 4.1-4.2). The energy
budget closes: total energy change = injected work - dissipated energy.

    python -m paper_1602_09079_gb300.turbulence --n 64 --order 3 --t-end 12 --out run.json

--checkpoint F --checkpoint-every T writes the state, the OU amplitudes and
the run's counters to F ("{steps}" in F keeps one file per checkpoint);
--resume F continues such a run, bit for bit if F was taken before t_end. With --spectrum-sub S the final state's velocity power spectrum and density
PDF (Sect. 4.3-4.4) on S^3 samples per cell are added to the output.

The driving amplitude is scaled once so that the box rms of the acceleration
starts at M c / t_s (the paper rescales its amplitude until the target Mach
number is reached); the reached rms Mach number is an output.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import DG_PREC_FP64, DG_PREC_MIXED, Solver
from .forcing import OUDriving, half_space_modes


def save_checkpoint(path, state, theta, meta):
    """One .npz file: the canonical state [nz][ny][nx][5][N] (FP64), the OU
    amplitudes theta and the run's counters and records as JSON (floats
    round-trip exactly). Written to a temporary file first, then renamed."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, state=np.asarray(state, dtype=np.float64), theta=np.asarray(theta, dtype=np.float64),
             meta=np.array(json.dumps(meta)))
    os.replace(tmp, path)


def load_checkpoint(path):
    with np.load(path) as f:
        return f["state"].copy(), f["theta"].copy(), json.loads(str(f["meta"]))


# run parameters a resumed run must share with the checkpointed one
_RESUME_KEYS = ("n", "order", "gamma", "target_mach", "precision", "seed", "courant", "record_every")


def run(n=64, order=3, gamma=1.01, t_end=12.0, mach=0.3, precision="mixed", seed=1234, courant=0.3,
        record_every=0.1, max_steps=10_000_000, spectrum_sub=0, pdf_range=(-0.5, 0.5), pdf_bins=100,
        checkpoint=None, checkpoint_every=None, resume=None, solver=None):
    """checkpoint: .npz path written every checkpoint_every time units and
    when the run stops ("{steps}" in it is replaced by the step count, which
    keeps one file per checkpoint); resume: a checkpoint to continue from
    (same parameters; the OU draws come from the same seeded stream). A run
    resumed from a checkpoint taken before t_end (periodic, or where
    max_steps stopped the run) reproduces the uninterrupted run bit for bit;
    a run that reached t_end ended on a step shortened to land there, so
    extending it to a later t_end is a slightly different trajectory.
    solver: the Solver class (a stand-in for tests of the driver's host
    logic)."""
    Solver_ = Solver if solver is None else solver
    s = Solver_((n, n, n), order, gamma, forcing=True)
    s.set_precision(DG_PREC_MIXED if precision == "mixed" else DG_PREC_FP64)
    rho0, p0 = 1.0, 1.0 / gamma
    c = math.sqrt(gamma * p0 / rho0)
    w = np.zeros(s.state_shape)
    w[..., 0, 0] = rho0
    w[..., 4, 0] = p0 / (gamma - 1.0)
    s.set_state(w)
    c_iso = math.sqrt(p0 / rho0)

    t_s = 1.0 / (2.0 * mach * c)
    dt_update = 0.1 * t_s
    nv = half_space_modes(1.0, 2.0)
    n_updates = int(t_end / dt_update) + 3
    z = np.random.default_rng(seed).standard_normal((n_updates, len(nv), 6))
    # the box rms of a(x) = sum_j Re(a_j e^{i k_j . x}) over distinct modes is
    # sqrt(sum_j |a_j|^2 / 2): scale the amplitudes once so that it starts at
    # M c / t_s (the acceleration that builds the target velocity M c within
    # one correlation time; the OU process keeps it stationary on average)
    target = mach * c / t_s
    drv = OUDriving(nv, t_s, dt_update, 1.0, z[0])
    rms1 = math.sqrt(0.5 * float(np.sum(drv.ahat() ** 2)))
    amp = target / rms1
    drv.amplitude = amp
    k_upd = 1
    s.set_forcing(drv.nvec, drv.ahat())
    next_update = dt_update

    E0 = s.totals()[4]
    work = diss = 0.0
    t, steps = 0.0, 0
    P = s.diagnostics()[2]
    series = []
    next_record = 0.0
    cfg = {"n": n, "order": order, "gamma": gamma, "target_mach": mach, "precision": precision, "seed": seed,
           "courant": courant, "record_every": record_every}
    if resume:
        state, theta, meta = load_checkpoint(resume)
        for key in _RESUME_KEYS:
            if meta["config"][key] != cfg[key]:
                raise ValueError(f"checkpoint {resume}: {key} = {meta['config'][key]!r}, run asks {cfg[key]!r}")
        s.set_state(state)
        drv.theta = theta
        drv.n_updates = meta["drv_updates"]
        k_upd, next_update = meta["k_upd"], meta["next_update"]
        s.set_forcing(drv.nvec, drv.ahat())
        E0, work, diss, P = meta["E0"], meta["work"], meta["diss"], meta["P"]
        t, steps, next_record = meta["t"], meta["steps"], meta["next_record"]
        series = [r for r in meta["series"] if not r.get("end_only")]

    def write_checkpoint():
        meta = {"config": cfg, "t": t, "steps": steps, "k_upd": k_upd, "next_update": next_update,
                "drv_updates": drv.n_updates, "E0": E0, "work": work, "diss": diss, "P": P,
                "next_record": next_record, "series": series}
        save_checkpoint(checkpoint.format(steps=steps), s.get_state(), drv.theta, meta)

    next_ckpt = t + checkpoint_every if (checkpoint and checkpoint_every) else math.inf
    t_wall = time.perf_counter()
    while t < t_end - 1e-12 and steps < max_steps:
        dt = min(s.cfl_dt(courant), t_end - t)
        s.step(dt)
        t += dt
        steps += 1
        P1 = s.diagnostics()[2]
        work += 0.5 * (P + P1) * dt
        diss += s.energy_reset(c_iso, rho0, want_dissipated=True)
        P = P1
        if t >= next_update - 1e-12 and k_upd < n_updates:
            drv.update(z[k_upd])
            k_upd += 1
            s.set_forcing(drv.nvec, drv.ahat())
            next_update += dt_update
            P = s.diagnostics()[2]
        at_record = t >= next_record - 1e-12
        if at_record or t >= t_end - 1e-12:
            d = s.diagnostics()
            series.append({"t": t, "steps": steps, "rms_mach": d[0], "kinetic": d[1], "power": d[2],
                           "injected": work, "dissipated": diss, "total_energy_change": s.totals()[4] - E0})
            if at_record:
                next_record += record_every
            else:
                series[-1]["end_only"] = True  # taken because the run ends here
        if t >= next_ckpt - 1e-12:
            write_checkpoint()
            next_ckpt += checkpoint_every
    s.check()
    if checkpoint:
        write_checkpoint()
    wall = time.perf_counter() - t_wall
    analysis = {}
    if spectrum_sub > 0:
        # final state (Sect. 4.3-4.4): velocity power spectrum and volume-weighted
        # PDF of ln(rho), both on spectrum_sub^3 samples per cell
        analysis["velocity_spectrum"] = {"sub": spectrum_sub,
                                         "shells": [float(x) for x in s.velocity_spectrum(spectrum_sub)]}
        lo, hi = pdf_range
        counts = s.density_pdf(spectrum_sub, lo, hi, pdf_bins)
        analysis["density_pdf"] = {"sub": spectrum_sub, "lo": lo, "hi": hi, "bins": pdf_bins,
                                   "counts": [int(x) for x in counts]}
    late = [r for r in series if r["t"] >= 0.5 * t_end]
    return {
        "config": {"n": n, "order": order, "gamma": gamma, "t_end": t_end, "target_mach": mach,
                   "precision": precision, "seed": seed, "courant": courant, "t_s": t_s,
                   "driving_amplitude": amp, "modes": int(len(drv.nvec))},
        "steps": steps, "wall_s": wall,
        "summary": {
            "rms_mach_final": series[-1]["rms_mach"],
            "rms_mach_mean_second_half": float(np.mean([r["rms_mach"] for r in late])) if late else None,
            "injected": work, "dissipated": diss, "total_energy_change": series[-1]["total_energy_change"],
            "budget_residual": series[-1]["total_energy_change"] - (work - diss),
        },
        "series": series,
        **analysis,
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--gamma", type=float, default=1.01)
    ap.add_argument("--t-end", type=float, default=12.0)
    ap.add_argument("--mach", type=float, default=0.3)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--seed", type=int, default=1234)
    ap.add_argument("--courant", type=float, default=0.3)
    ap.add_argument("--record-every", type=float, default=0.1)
    ap.add_argument("--spectrum-sub", type=int, default=0,
                    help="if > 0, record the final velocity spectrum and density PDF on sub^3 samples per cell")
    ap.add_argument("--pdf-lo", type=float, default=-0.5)
    ap.add_argument("--pdf-hi", type=float, default=0.5)
    ap.add_argument("--pdf-bins", type=int, default=100)
    ap.add_argument("--checkpoint", default=None, help=".npz file written every --checkpoint-every and at the end")
    ap.add_argument("--checkpoint-every", type=float, default=None)
    ap.add_argument("--resume", default=None, help="continue from this checkpoint (same run parameters)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run(a.n, a.order, a.gamma, a.t_end, a.mach, a.precision, a.seed, a.courant, a.record_every,
              spectrum_sub=a.spectrum_sub, pdf_range=(a.pdf_lo, a.pdf_hi), pdf_bins=a.pdf_bins,
              checkpoint=a.checkpoint, checkpoint_every=a.checkpoint_every, resume=a.resume)
    txt = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    print(json.dumps({k: res[k] for k in ("config", "steps", "wall_s", "summary")}))


if __name__ == "__main__":
    main()
