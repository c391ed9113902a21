"""Turbulence diagnostics on the GPU (Sect. 4.1 rms Mach number, Sect. 4.2
injected energy) through the C ABI: against the oracle on the same seeded
states, and the energy budget of driven steps with the energy reset at the
paper's gamma = 1.01: the change of the total energy equals the work of the
driving force (trapezoidal in time) minus the dissipated energy the reset
reports."""
import math

import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1602_09079_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("prec,tol_pow", [(0, 1e-11), (1, 1e-6)])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_diagnostics_match_oracle(dg, order, prec, tol_pow):
    n, g = (7, 6, 5), syn.GAMMA
    s = dg.Solver(n, order, g, forcing=True)
    s.set_precision(prec)
    o = oracle.Oracle(n, order - 1, g)
    nv = syn.driving_modes(1.0, 2.0)
    ah = np.random.default_rng(11).normal(size=(len(nv), 6))
    s.set_forcing(nv, ah)
    o.set_forcing(nv, ah)
    w = syn.random_state(n, s.N, g, seed=900 + order, high=0.01)
    s.set_state(w)
    d, do = s.diagnostics(), o.diagnostics(w)
    assert abs(d[0] - do[0]) <= 1e-13 * do[0]
    assert abs(d[1] - do[1]) <= 1e-13 * do[1]
    # the power is a sum of products of both signs: bound its error by the
    # sum of their magnitudes (the kinetic energy times the force scale)
    scale = abs(do[2]) + np.abs(ah).sum() * math.sqrt(2 * do[1])
    assert abs(d[2] - do[2]) <= tol_pow * scale, (d, do)
    s.set_forcing(nv[:0], ah[:0])
    assert s.diagnostics()[2] == 0.0


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_budget_of_driven_steps(dg, prec):
    """gamma = 1.01, warm subsonic turbulence on 24^3 at degree 2, fixed
    driving modes, 12 steps with the energy reset after each: total energy
    change = sum of (P_start + P_end)/2 dt - sum of dissipated energies."""
    n, g = (24, 24, 24), 1.01
    s = dg.Solver(n, 3, g, forcing=True)
    s.set_precision(prec)
    s.project_fn(syn.solenoidal_velocity(seed=1234, mach=0.3, gamma=g))
    nv = syn.driving_modes(1.0, 2.0)
    ah = np.random.default_rng(5).normal(size=(len(nv), 6)) * 2.0
    s.set_forcing(nv, ah)
    c_iso = math.sqrt(1.0 / g)
    s.energy_reset(c_iso, 1.0)
    E0 = s.totals()[4]
    work = diss = 0.0
    P = s.diagnostics()[2]
    for _ in range(12):
        dt = s.cfl_dt(0.3)
        s.step(dt)
        P1 = s.diagnostics()[2]
        work += 0.5 * (P + P1) * dt
        diss += s.energy_reset(c_iso, 1.0, want_dissipated=True)
        P = P1
    dE = s.totals()[4] - E0
    assert abs(work) > 1e-6  # the driving does work
    assert abs(dE - (work - diss)) <= 1e-3 * (abs(work) + abs(diss)), (dE, work, diss)
