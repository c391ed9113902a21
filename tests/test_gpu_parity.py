"""CUDA path vs the FP64 CPU oracle, element by element on the same seeded
inputs, through the C ABI (Python binding with the same names).

Bar (normwise per conserved variable, because high modes close to zero make
element-wise relative error meaningless):
  FP64 path:  max|gpu - oracle| / max|oracle| <= 1e-12
  mixed path: max|gpu - oracle| / max|oracle| <= 2e-5 (FP32 quadrature of
              O(10^2) terms; see the tolerance derivation in the design notes)
Integer outputs (limiter flags) must match exactly.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 2e-5


@pytest.fixture(scope="module")
def dg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1602_09079_gb300 as m
    m.load()
    return m


def normwise(got, ref):
    got = np.asarray(got).reshape(-1, 5, got.shape[-1]) if got.ndim > 2 else got
    ref = np.asarray(ref).reshape(got.shape)
    errs = []
    for i in range(5):
        den = np.max(np.abs(ref[:, i, :]))
        errs.append(np.max(np.abs(got[:, i, :] - ref[:, i, :])) / max(den, 1e-300))
    return max(errs)


MESHES = [(1, 1, 1), (2, 2, 2), (5, 7, 3), (8, 8, 8), (16, 12, 10)]


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("n", MESHES)
def test_rhs_fp64_matches_oracle(dg, order, n):
    g = 1.4
    s = dg.Solver(n, order, g, length=(1.0, 0.8, 1.3))
    o = oracle.Oracle(n, order - 1, g, L=(1.0, 0.8, 1.3))
    w = syn.random_state(n, s.N, g, seed=100 + order, high=0.01)
    s.set_state(w)
    R = s.rhs()
    Ro = o.rhs(w)
    assert np.all(np.isfinite(Ro))
    assert normwise(R, Ro) <= TOL64


@pytest.mark.parametrize("order", [2, 3, 4])
def test_rhs_mixed_matches_oracle(dg, order):
    n, g = (9, 8, 7), syn.GAMMA
    s = dg.Solver(n, order, g)
    s.set_precision(dg.DG_PREC_MIXED)
    o = oracle.Oracle(n, order - 1, g)
    w = syn.random_state(n, s.N, g, seed=200 + order, high=0.01)
    s.set_state(w)
    assert normwise(s.rhs(), o.rhs(w)) <= TOLMIX


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOLMIX)])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_rhs_with_forcing_matches_oracle(dg, order, prec, tol):
    n, g = (6, 5, 7), syn.GAMMA
    s = dg.Solver(n, order, g, forcing=True)
    s.set_precision(prec)
    o = oracle.Oracle(n, order - 1, g)
    nv = syn.driving_modes(1.0, 2.0)
    ah = np.random.default_rng(7).normal(size=(len(nv), 6))
    s.set_forcing(nv, ah)
    o.set_forcing(nv, ah)
    w = syn.random_state(n, s.N, g, seed=300 + order, high=0.01)
    s.set_state(w)
    assert normwise(s.rhs(), o.rhs(w)) <= tol


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_step_fp64_matches_oracle(dg, order):
    n, g = (7, 6, 5), syn.GAMMA
    s = dg.Solver(n, order, g)
    o = oracle.Oracle(n, order - 1, g)
    w = syn.random_state(n, s.N, g, seed=400 + order, high=0.01)
    s.set_state(w)
    for _ in range(3):
        dt = s.cfl_dt(0.3)
        st, dto = o.cfl_dt(w, 0.3)
        assert st == 0 and abs(dt - dto) <= 1e-14 * dto
        s.step(dt)
        st, w = o.step(w, dt)
        assert st == 0
        assert normwise(s.get_state(), w) <= TOL64
    s.check()


@pytest.mark.parametrize("order", [2, 3, 4])
def test_step_with_limiter_active_matches_oracle(dg, order):
    """States whose polynomials leave the positive set: the limiter fires in
    every stage; results still within the FP64 bar."""
    n, g, eps = (6, 6, 6), syn.GAMMA, 1e-2
    s = dg.Solver(n, order, g)
    s.set_eps(eps, eps)
    o = oracle.Oracle(n, order - 1, g, eps_rho=eps, eps_p=eps)
    w = syn.random_state(n, s.N, g, seed=500 + order, high=0.4)
    st, wl, fl, nl = o.limit(w)
    assert st == 0 and nl > 0
    s.set_state(w)
    dt = s.cfl_dt(0.2)
    s.step(dt)
    st, ref = o.step(w, dt)
    assert st == 0
    assert normwise(s.get_state(), ref) <= TOL64


@pytest.mark.parametrize("order", [2, 3, 4])
def test_step_mixed_close_to_oracle(dg, order):
    n, g = (8, 7, 6), syn.GAMMA
    s = dg.Solver(n, order, g)
    s.set_precision(dg.DG_PREC_MIXED)
    o = oracle.Oracle(n, order - 1, g)
    w = syn.random_state(n, s.N, g, seed=600 + order, high=0.01)
    s.set_state(w)
    for _ in range(2):
        dt = s.cfl_dt(0.3)
        s.step(dt)
        st, w = o.step(w, dt)
    # an FP32 increment dt R on an O(1) FP64 state: error ~ 1e-7 dt |R|
    assert normwise(s.get_state(), w) <= 1e-7


@pytest.mark.parametrize("order", [2, 3, 4])
def test_limiter_matches_oracle(dg, order):
    n, g, eps = (9, 7, 5), 1.4, 1e-2
    s = dg.Solver(n, order, g)
    s.set_eps(eps, eps)
    o = oracle.Oracle(n, order - 1, g, eps_rho=eps, eps_p=eps)
    w = syn.random_state(n, s.N, g, seed=700 + order, high=0.5)
    s.set_state(w)
    nl, flags = s.limit(want_flags=True)
    st, ref, fref, nref = o.limit(w)
    assert st == 0
    assert nl == nref and nl > 10
    assert np.array_equal(flags, fref)
    assert normwise(s.get_state(), ref) <= TOL64


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_projection_matches_oracle(dg, order):
    n, g = (5, 4, 6), syn.GAMMA
    s = dg.Solver(n, order, g, length=(1.0, 1.0, 2.0))
    o = oracle.Oracle(n, order - 1, g, L=(1.0, 1.0, 2.0))
    fn = syn.solenoidal_velocity(seed=3, mach=0.5, gamma=g)
    assert np.allclose(s.quadrature_points(), o.volume_points(), rtol=0, atol=1e-15)
    s.project_fn(fn)
    assert normwise(s.get_state(), o.project_fn(fn)) <= 1e-14


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, 1e-6)])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_energy_reset_matches_oracle(dg, order, prec, tol):
    n, g = (7, 5, 6), syn.GAMMA
    s = dg.Solver(n, order, g)
    s.set_precision(prec)
    o = oracle.Oracle(n, order - 1, g)
    w = syn.random_state(n, s.N, g, seed=800 + order, high=0.01, v_mean=(-0.2, 0.2))
    s.set_state(w)
    d = s.energy_reset(0.7, 1.0, want_dissipated=True)
    st, ref, dref = o.energy_reset(w, 0.7, 1.0)
    assert st == 0
    assert normwise(s.get_state(), ref) <= tol
    assert abs(d - dref) <= tol * max(abs(dref), 1e-3)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_mixed_step_then_energy_reset_close_to_oracle(dg, order):
    """Mixed path: a step leaves a valid FP32 shadow, so the reset reads its
    point values from the shadow and screens in FP32; the state and the
    dissipated energy stay within the mixed tolerances of the oracle."""
    n, g = (7, 5, 6), syn.GAMMA
    s = dg.Solver(n, order, g)
    s.set_precision(dg.DG_PREC_MIXED)
    o = oracle.Oracle(n, order - 1, g)
    w = syn.random_state(n, s.N, g, seed=850 + order, high=0.01, v_mean=(-0.2, 0.2))
    s.set_state(w)
    for _ in range(2):
        dt = s.cfl_dt(0.3)
        s.step(dt)
        d = s.energy_reset(0.7, 1.0, want_dissipated=True)
        st, w = o.step(w, dt)
        assert st == 0
        st, w, dref = o.energy_reset(w, 0.7, 1.0)
        assert st == 0
        assert normwise(s.get_state(), w) <= 1e-6
        # the dissipated energy is a small difference of internal energies
        # whose new values the mixed path forms in FP32: on a smooth state
        # every cell rounds alike, so the cells' errors add up coherently;
        # bound it by the mixed reset's state-level tolerance (1e-6) times
        # the total energy
        assert abs(d - dref) <= 1e-6 * abs(o.totals(w)[4])
        w = s.get_state()  # continue both from the GPU state


def test_totals_and_conservation(dg):
    n, g = (12, 10, 9), syn.GAMMA
    s = dg.Solver(n, 3, g)
    o = oracle.Oracle(n, 2, g)
    w = syn.random_state(n, s.N, g, seed=900, high=0.01)
    s.set_state(w)
    t0 = s.totals()
    assert np.max(np.abs(t0 - o.totals(w)) / np.abs(o.totals(w)).clip(1e-3)) <= 1e-14
    for _ in range(5):
        s.step(s.cfl_dt(0.3))
    t1 = s.totals()
    assert np.max(np.abs(t1 - t0) / np.abs(t0).clip(1e-3)) <= 1e-13


def test_config4_size_sampled(dg):
    """256^3 cells, order 4 (degree 3), with the driving source: the size and
    launch configuration of the degree-3 benchmark. The state is a random
    smooth state of 32^3 cells tiled periodically to 256^3 (cheap to build on
    the host, every cell's neighbours a different random cell). R at sampled
    cells against the oracle in both precisions, then one mixed SSP-RK3 step
    with the energy reset conserves mass to round-off."""
    import torch
    n, order, g = (256, 256, 256), 4, syn.GAMMA
    s = dg.Solver(n, order, g, forcing=True)
    w = np.tile(syn.random_state((32, 32, 32), s.N, g, seed=44, high=0.01), (8, 8, 8, 1, 1))
    s.set_state(w)
    nv = syn.driving_modes(1.0, 2.0)
    ah = np.random.default_rng(1234).normal(size=(len(nv), 6)) * 0.5
    s.set_forcing(nv, ah)
    o = oracle.Oracle(n, order - 1, g)
    o.set_forcing(nv, ah)
    cells = syn.sample_cells(s.ncells, 200, seed=6)
    Ro = o.rhs_cells(w, cells)
    st, dt1 = o.cfl_dt(w, 1.0)
    assert st == 0
    w0max = np.abs(w.reshape(-1, 5, s.N)[:, :, 0]).max(axis=0)
    del w
    for prec, tol in ((dg.DG_PREC_FP64, TOL64), (dg.DG_PREC_MIXED, TOLMIX)):
        s.set_precision(prec)
        R = s.rhs().reshape(-1, 5, s.N)[cells]
        for i in range(5):
            scale = max(np.abs(Ro[:, i, :]).max(), w0max[i] / dt1)
            assert np.abs(R[:, i, :] - Ro[:, i, :]).max() <= tol * scale, (prec, i)
        del R
    s.set_precision(dg.DG_PREC_MIXED)
    t0 = s.totals()
    s.step(s.cfl_dt(0.3))
    s.energy_reset(math.sqrt(1.0 / g), 1.0)
    s.check()
    assert abs(s.totals()[0] - t0[0]) <= 1e-13 * abs(t0[0])
    torch.cuda.synchronize()


def test_error_codes(dg):
    g = syn.GAMMA
    s = dg.Solver((4, 4, 4), 3, g)
    w = syn.random_state((4, 4, 4), s.N, g, seed=1, high=0.01)
    s.set_state(w)
    with pytest.raises(dg.DGError) as e:
        s.step(-1.0)
    assert e.value.code == dg.DG_ERR_ARG
    bad = w.copy()
    bad[1, 2, 3, 0, 0] = -0.5  # negative mean density: the limiter cannot fix it
    s.set_state(bad)
    with pytest.raises(dg.DGError) as e:
        s.limit()
    assert e.value.code == dg.DG_ERR_POSITIVITY
    bad = w.copy()
    bad[0, 0, 0, 4, 3] = np.nan
    s.set_state(bad)
    with pytest.raises(dg.DGError) as e:
        s.limit()
    assert e.value.code == dg.DG_ERR_NONFINITE
    # the context stays usable after a reported device error
    s.set_state(w)
    assert s.limit() == 0
    with pytest.raises(dg.DGError) as e:
        s.set_forcing(syn.driving_modes(), np.zeros((10, 6)))  # scratch not sized for it
    assert e.value.code == dg.DG_ERR_ARG
    ctx = dg.dg_init((2, 2, 2), 2, g)
    with pytest.raises(dg.DGError) as e:
        dg.dg_step(ctx, 0.1)
    assert e.value.code == dg.DG_ERR_NOT_BOUND
    dg.dg_destroy(ctx)
    with pytest.raises(dg.DGError):
        dg.dg_init((2, 2, 2), 5, g)
    with pytest.raises(dg.DGError):
        dg.dg_init((2, 0, 2), 2, g)


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOLMIX)])
def test_full_size_turbulence_sampled(dg, prec, tol):
    """128^3 cells, order 3 (degree 2), driven subsonic turbulence, the
    workload the benchmark times: R at sampled cells (incl. the periodic
    corners) against the oracle, evaluated one cell at a time; and one full
    SSP-RK3 step with the energy reset conserves mass to round-off."""
    import torch
    n, order, g = (128, 128, 128), 3, syn.GAMMA
    s = dg.Solver(n, order, g, forcing=True)
    s.set_precision(prec)
    fn = syn.solenoidal_velocity(seed=1234, mach=0.3, gamma=g)
    s.project_fn(fn)
    nv = syn.driving_modes(1.0, 2.0)
    ah = np.random.default_rng(1234).normal(size=(len(nv), 6)) * 0.5
    s.set_forcing(nv, ah)
    w = s.get_state()
    o = oracle.Oracle(n, order - 1, g)
    o.set_forcing(nv, ah)
    cells = syn.sample_cells(s.ncells, 300, seed=5)
    Ro = o.rhs_cells(w, cells)
    R = s.rhs().reshape(-1, 5, s.N)[cells]
    # For a solenoidal start d(rho)/dt = -div(rho v) nearly cancels, so R_rho
    # is far below the flux terms it is summed from; the error of each
    # variable is measured against the change its state can undergo over one
    # Courant-1 time step (max|w_i0| / dt_1), or max|R_i| if larger.
    st, dt1 = o.cfl_dt(w, 1.0)
    assert st == 0
    w0max = np.abs(w.reshape(-1, 5, s.N)[:, :, 0]).max(axis=0)
    for i in range(5):
        scale = max(np.abs(Ro[:, i, :]).max(), w0max[i] / dt1)
        assert np.abs(R[:, i, :] - Ro[:, i, :]).max() <= tol * scale, i
    t0 = s.totals()
    dt = s.cfl_dt(0.3)
    s.step(dt)
    s.energy_reset(math.sqrt(1.0 / g), 1.0)
    s.check()
    t1 = s.totals()
    assert abs(t1[0] - t0[0]) <= 1e-13 * abs(t0[0])
    torch.cuda.synchronize()
