"""Host logic of the driven-run driver (paper_1602_09079_gb300.turbulence) on
the CPU, with a deterministic stand-in for the GPU Solver: OU updates every
0.1 t_s, records every record_every and at the end, the final analysis hook,
and checkpoint/resume reproducing the uninterrupted run bit for bit (the
real solver is deterministic too: no value depends on the order of atomic
operations)."""
import math

import numpy as np
import pytest

from paper_1602_09079_gb300 import turbulence


class StandIn:
    """Toy dynamics on the canonical state: the momentum means are pushed by
    the mean driving acceleration, the first momentum modes decay, the energy
    mean takes the work; deterministic in the state and the forcing."""

    instances = []

    def __init__(self, n, order, gamma, forcing=True):
        self.n, self.N = n, order * (order + 1) * (order + 2) // 6
        self.w = np.zeros(self.state_shape)
        self.acc = np.zeros(3)
        self.forcing_calls = 0
        StandIn.instances.append(self)

    @property
    def state_shape(self):
        return (self.n[2], self.n[1], self.n[0], 5, self.N)

    def set_precision(self, mode):
        self.prec = mode

    def set_state(self, w):
        self.w = np.array(w, dtype=np.float64, copy=True)

    def get_state(self):
        return self.w.copy()

    def set_forcing(self, nvec, ahat):
        a = np.asarray(ahat)
        self.acc = a[:, :3].sum(axis=0) * 0.1 + a[:, 3:].sum(axis=0) * 0.05
        self.forcing_calls += 1

    def cfl_dt(self, courant):
        m = np.abs(self.w[..., 1:4, 0]).max()
        return courant * 0.02 / (1.0 + m)

    def step(self, dt):
        rho = self.w[..., 0:1, 0]
        m = self.w[..., 1:4, 0]
        self.w[..., 4, 0] += dt * np.sum(m * self.acc, axis=-1)
        self.w[..., 1:4, 0] = m + dt * rho * self.acc * (1 + 0.01 * np.arange(self.w.shape[2]))[None, None, :, None]
        self.w[..., 1:4, 1] = self.w[..., 1:4, 1] * (1 - 0.1 * dt) + 0.01 * dt

    def diagnostics(self):
        rho = self.w[..., 0, 0]
        m = self.w[..., 1:4, 0]
        v2 = np.sum(m * m, axis=-1) / rho ** 2
        vol = 1.0 / rho.size
        return (float(np.sqrt(np.mean(v2))), float(np.sum(0.5 * rho * v2) * vol),
                float(np.sum(m * self.acc) * vol))

    def energy_reset(self, c_iso, rho0=1.0, want_dissipated=False):
        d = 1e-3 * self.w[..., 1:4, 1].sum(axis=-1)
        self.w[..., 4, 0] -= d
        return float(np.sum(d) / d.size)

    def totals(self):
        return self.w[..., :, 0].sum(axis=(0, 1, 2)) / self.w[..., 0, 0].size

    def check(self):
        assert np.all(np.isfinite(self.w))

    def velocity_spectrum(self, sub):
        return np.arange(5, dtype=float) * sub

    def density_pdf(self, sub, lo, hi, n_bins):
        return np.full(n_bins + 2, sub, dtype=np.int64)


KW = dict(n=4, order=2, gamma=1.01, mach=0.3, precision="mixed", seed=5, courant=0.3, record_every=0.1,
          solver=StandIn)


def test_records_updates_and_analysis():
    StandIn.instances.clear()
    r = turbulence.run(t_end=0.45, spectrum_sub=2, pdf_bins=8, **KW)
    s = StandIn.instances[-1]
    ts = [e["t"] for e in r["series"]]
    # records at the first step (t ~ 0), near 0.1, 0.2, 0.3, 0.4, and the
    # end-of-run record at 0.45
    assert len(ts) == 6 and abs(ts[-1] - 0.45) <= 1e-12 and r["series"][-1].get("end_only")
    assert not any(e.get("end_only") for e in r["series"][:-1])
    for j, t in enumerate(ts[:-1]):
        assert 0.1 * j - 1e-12 <= t <= 0.1 * j + 0.02  # the first step at or after the record time
    t_s = 1.0 / (2.0 * 0.3 * 1.0)  # c = 1 at the start state
    assert s.forcing_calls == 1 + int(0.45 / (0.1 * t_s))
    assert r["velocity_spectrum"]["shells"] == [0.0, 2.0, 4.0, 6.0, 8.0]
    assert r["density_pdf"]["counts"] == [2] * 10
    assert r["steps"] == r["series"][-1]["steps"]


@pytest.mark.parametrize("stop_steps", [37, 60])
def test_interrupted_run_resumes_bitwise(tmp_path, stop_steps):
    """A run stopped after stop_steps steps (as by a time limit; its last
    checkpoint is written there) and resumed to t_end gives the records,
    totals and final state of the uninterrupted run, bit for bit."""
    ck = str(tmp_path / "run.npz")
    StandIn.instances.clear()
    full = turbulence.run(t_end=1.0, **KW)
    w_full = StandIn.instances[-1].get_state()
    part = turbulence.run(t_end=1.0, checkpoint=ck, checkpoint_every=0.25, max_steps=stop_steps, **KW)
    assert part["steps"] == stop_steps
    state, theta, meta = turbulence.load_checkpoint(ck)
    assert meta["steps"] == stop_steps and np.array_equal(state, StandIn.instances[-1].get_state())
    rest = turbulence.run(t_end=1.0, resume=ck, **KW)
    assert rest["series"] == full["series"]
    assert rest["steps"] == full["steps"]
    for key in ("injected", "dissipated", "total_energy_change", "budget_residual", "rms_mach_final"):
        assert rest["summary"][key] == full["summary"][key]
    assert np.array_equal(StandIn.instances[-1].get_state(), w_full)


def test_periodic_checkpoint_resumes_bitwise(tmp_path):
    """With "{steps}" in the path every periodic checkpoint keeps its own
    file; resuming from the one near t = 0.3 reproduces the uninterrupted
    run."""
    pattern = str(tmp_path / "c_{steps}.npz")
    StandIn.instances.clear()
    full = turbulence.run(t_end=0.8, checkpoint=pattern, checkpoint_every=0.3, **KW)
    files = sorted(tmp_path.glob("c_*.npz"), key=lambda f: int(f.stem[2:]))
    ts = [turbulence.load_checkpoint(str(f))[2]["t"] for f in files]
    assert len(files) == 3 and 0.3 <= ts[0] < 0.32 and 0.6 <= ts[1] < 0.62 and abs(ts[2] - 0.8) <= 1e-12
    rest = turbulence.run(t_end=0.8, resume=str(files[0]), **KW)
    assert rest["series"] == full["series"] and rest["steps"] == full["steps"]


def test_resume_rejects_other_parameters(tmp_path):
    ck = str(tmp_path / "b.npz")
    turbulence.run(t_end=0.2, checkpoint=ck, max_steps=20, **KW)
    with pytest.raises(ValueError, match="seed"):
        turbulence.run(t_end=0.4, resume=ck, **dict(KW, seed=6))
    with pytest.raises(ValueError, match="order"):
        turbulence.run(t_end=0.4, resume=ck, **dict(KW, order=3))
    assert math.isfinite(turbulence.load_checkpoint(ck)[2]["E0"])
