"""The exact-Riemann-solver flux option (Sect. 2.3, next to HLLC) on the
GPU against the oracle's exact solver, through the C ABI: R(y) in FP64
(<= 1e-12 normwise) and in the mixed path (<= 2e-5), on mild states and on
states whose neighbouring cell means jump strongly (shocks, rarefactions,
supersonic faces and vacuum-opening expansions), and full SSP-RK3 steps."""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 2e-5
STRONG = dict(rho_mean=(0.2, 2.0), v_mean=(-2.0, 2.0), p_mean=(0.1, 2.0))


@pytest.fixture(scope="module")
def dg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1602_09079_gb300 as m
    m.load()
    return m


def normwise(got, ref):
    got = np.asarray(got).reshape(-1, 5, got.shape[-1])
    ref = np.asarray(ref).reshape(got.shape)
    return max(np.max(np.abs(got[:, i] - ref[:, i])) / max(np.max(np.abs(ref[:, i])), 1e-300) for i in range(5))


def strong_state(o, n, N, g, seed):
    """Strong jumps between neighbouring cell means, then the oracle's
    positivity limiter so that every face trace is a physical state (the
    step applies the limiter before each R evaluation the same way)."""
    w = syn.random_state(n, N, g, seed=seed, high=0.01, **STRONG)
    st, w, _, _ = o.limit(w)
    assert st == 0
    return w


def exact_pair(dg, n, order, g, prec=0, **kw):
    s = dg.Solver(n, order, g, **kw)
    s.set_precision(prec)
    s.set_flux(dg.DG_FLUX_EXACT)
    o = oracle.Oracle(n, order - 1, g, flux=oracle.FLUX_EXACT)
    return s, o


@pytest.mark.parametrize("strong", [False, True])
@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_rhs_exact_fp64_matches_oracle(dg, order, strong):
    n, g = (6, 5, 7), 1.4
    s, o = exact_pair(dg, n, order, g)
    w = (strong_state(o, n, s.N, g, 500 + order) if strong else
         syn.random_state(n, s.N, g, seed=500 + order, high=0.01))
    s.set_state(w)
    Ro = o.rhs(w)
    assert np.all(np.isfinite(Ro))
    assert normwise(s.rhs(), Ro) <= TOL64
    s.check()


def test_exact_and_hllc_fluxes_differ(dg):
    """The switch selects a different flux: on strong jumps R differs from
    the HLLC one (and the HLLC one is restored by switching back)."""
    n, g = (5, 4, 6), 1.4
    s = dg.Solver(n, 3, g)
    w = strong_state(oracle.Oracle(n, 2, g), n, s.N, g, 9)
    s.set_state(w)
    R_h = s.rhs()
    s.set_flux(dg.DG_FLUX_EXACT)
    R_e = s.rhs()
    s.set_flux(dg.DG_FLUX_HLLC)
    assert np.abs(R_e - R_h).max() > 1e-4 * np.abs(R_h).max()
    assert np.array_equal(s.rhs(), R_h)
    with pytest.raises(dg.DGError) as e:
        s.set_flux(2)
    assert e.value.code == dg.DG_ERR_ARG


@pytest.mark.parametrize("strong", [False, True])
@pytest.mark.parametrize("order", [2, 3, 4])
def test_rhs_exact_mixed_close_to_oracle(dg, order, strong):
    n, g = (9, 8, 7), syn.GAMMA
    s, o = exact_pair(dg, n, order, g, prec=dg.DG_PREC_MIXED)
    w = (strong_state(o, n, s.N, g, 600 + order) if strong else
         syn.random_state(n, s.N, g, seed=600 + order, high=0.01))
    s.set_state(w)
    assert normwise(s.rhs(), o.rhs(w)) <= TOLMIX
    s.check()


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_step_exact_fp64_matches_oracle(dg, order):
    """Three SSP-RK3 steps with the exact flux and the positivity limiter,
    step by step against the oracle."""
    n, g = (7, 6, 5), syn.GAMMA
    s, o = exact_pair(dg, n, order, g)
    w = syn.random_state(n, s.N, g, seed=700 + order, high=0.01, v_mean=(-1.5, 1.5))
    s.set_state(w)
    for _ in range(3):
        dt = s.cfl_dt(0.3)
        st, dto = o.cfl_dt(w, 0.3)
        assert st == 0 and abs(dt - dto) <= 1e-14 * dto
        s.step(dt)
        st, w = o.step(w, dt)
        assert st == 0
        assert normwise(s.get_state(), w) <= TOL64
