"""The optional limiter point set S u (volume Gauss points) on the GPU
against the oracle with the same option: limiter flags bit-exact and state
to 1e-12, SSP-RK3 steps to 1e-12, and the interior-dip cell that only the
union catches."""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


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


@pytest.mark.parametrize("order", [2, 3, 4])
def test_union_limiter_matches_oracle(dg, order):
    n, g, eps = (9, 7, 5), 1.4, 1e-2
    s = dg.Solver(n, order, g)
    s.set_eps(eps, eps)
    s.set_limiter_points(dg.DG_LIMIT_S_VOLUME)
    o = oracle.Oracle(n, order - 1, g, eps_rho=eps, eps_p=eps, limiter_points=oracle.LIMIT_S_VOLUME)
    w = syn.random_state(n, s.N, g, seed=720 + order, high=0.5)
    s.set_state(w)
    nl, flags = s.limit(want_flags=True)
    st, ref, fref, nref = o.limit(w)
    assert st == 0
    assert nl == nref and nl > 10
    assert np.array_equal(flags, fref)
    assert normwise(s.get_state(), ref) <= TOL64


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("order", [2, 3])
def test_union_limiter_steps_match_oracle(dg, order, prec):
    """Floors at 1e-2 as in the S-limiter step test (floors near zero make
    the theta2 root ill-conditioned in both implementations); the limiter
    fires in every stage."""
    n, g, eps = (7, 6, 5), syn.GAMMA, 1e-2
    s = dg.Solver(n, order, g)
    s.set_precision(prec)
    s.set_eps(eps, eps)
    s.set_limiter_points(dg.DG_LIMIT_S_VOLUME)
    o = oracle.Oracle(n, order - 1, g, eps_rho=eps, eps_p=eps, limiter_points=oracle.LIMIT_S_VOLUME)
    w = syn.random_state(n, s.N, g, seed=740 + order, high=0.4)
    s.set_state(w)
    for _ in range(3):
        dt = s.cfl_dt(0.2)
        s.step(dt)
        st, w = o.step(w, dt)
        assert st == 0
        assert normwise(s.get_state(), w) <= (TOL64 if prec == 0 else 1e-6)
        w = s.get_state()


def test_interior_dip_cell(dg):
    k = 2
    idx = {tuple(x): i for i, x in enumerate(oracle.mode_exponents(k))}
    probe = oracle.Oracle((1, 1, 1), k, syn.GAMMA)
    w = np.zeros(probe.state_shape)
    w[..., 0, 0] = 1.0
    w[..., 4, 0] = 50.0
    for m in ((1, 1, 0), (1, 0, 1), (0, 1, 1)):
        w[..., 0, idx[m]] = -0.3
    for m in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
        w[..., 0, idx[m]] = 0.26
    eps = 0.095  # between the minimum over S (0.112) and over the Gauss points (0.078)
    s = dg.Solver((1, 1, 1), k + 1, syn.GAMMA)
    s.set_eps(eps, 1e-6)
    s.set_state(w)
    nl, flags = s.limit(want_flags=True)
    assert nl == 0 and np.array_equal(s.get_state(), w)
    s.set_limiter_points(dg.DG_LIMIT_S_VOLUME)
    nl, flags = s.limit(want_flags=True)
    assert nl == 1 and flags[0] & 1
    o = oracle.Oracle((1, 1, 1), k, syn.GAMMA, eps_rho=eps, eps_p=1e-6, limiter_points=oracle.LIMIT_S_VOLUME)
    st, ref, _, _ = o.limit(w)
    assert st == 0 and normwise(s.get_state(), ref) <= TOL64
    with pytest.raises(dg.DGError) as e:
        s.set_limiter_points(2)
    assert e.value.code == dg.DG_ERR_ARG
