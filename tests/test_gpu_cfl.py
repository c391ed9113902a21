"""dg_cfl_dt against the FP64 oracle on cell means built to stress the
kernel's FP32 pre-selection of candidate cells (Sect. 2.4: the time step
from the largest wave-speed sum over the cells' means).

The kernel evaluates every cell in FP32 and re-evaluates in FP64 only the
cells near its block's FP32 maximum and the cells whose FP32 value it cannot
trust; the result must still be the FP64 maximum. The cases: near ties of the
wave-speed sum that FP32 cannot tell apart, hypersonic cells (kinetic energy
above 0.99 of E: the FP32 pressure is a cancellation), densities below the
FP32 normal range, maxima in different thread blocks, on a ragged mesh of
many blocks. Bar: 1e-14 relative to the oracle (the same FP64 formula, up to
rounding order)."""
import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

MESH = (37, 33, 29)  # 35,409 cells: 35 blocks of 1024, the last one ragged


@pytest.fixture(scope="module")
def dg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1602_09079_gb300 as m
    m.load()
    return m


def state_from_means(rho, v, p, N, gamma=syn.GAMMA):
    """Canonical state [nz][ny][nx][5][N] with the given primitive means and
    zero higher modes."""
    means = syn.conserved(rho, v[0], v[1], v[2], p, gamma)
    w = np.zeros(rho.shape + (5, N))
    w[..., 0] = np.moveaxis(means, 0, -1)
    return w


def check(dg, w, order=3):
    s = dg.Solver(MESH, order, syn.GAMMA)
    o = oracle.Oracle(MESH, order - 1, syn.GAMMA)
    s.set_state(w)
    dt = s.cfl_dt(0.3)
    st, dto = o.cfl_dt(w, 0.3)
    assert st == 0
    assert abs(dt - dto) <= 1e-14 * dto, (dt, dto)
    return dt


def base(seed):
    rng = np.random.default_rng(seed)
    shp = MESH[::-1]
    rho = rng.uniform(0.5, 2.0, size=shp)
    v = rng.uniform(-0.5, 0.5, size=(3,) + shp)
    p = rng.uniform(0.5, 1.5, size=shp)
    return rng, rho, v, p


@pytest.mark.parametrize("where", [0, 35408, 17 * 1024 + 3])
def test_cfl_near_ties(dg, where):
    """Every cell has the same means up to relative 1e-9 perturbations of the
    velocity; the unique FP64 maximum sits in the first, the last (ragged) or
    a middle block."""
    shp = MESH[::-1]
    rng = np.random.default_rng(11)
    rho = np.ones(shp)
    p = np.ones(shp)
    v = np.zeros((3,) + shp)
    v[0] = 0.5 * (1.0 + 1e-9 * rng.uniform(0.0, 1.0, size=shp))
    v[0].reshape(-1)[where] = 0.5 * (1.0 + 2e-9)
    w = state_from_means(rho, v, p, 10)
    check(dg, w)


def test_cfl_hypersonic_cells(dg):
    """Scattered cells at Mach 40-60 (kinetic energy above 0.99 of E), with
    and without the largest sum, and a hypersonic cell that is not the
    maximum."""
    rng, rho, v, p = base(12)
    flat = v.reshape(3, -1)
    idx = rng.choice(flat.shape[1], size=40, replace=False)
    c = np.sqrt(syn.GAMMA * p.reshape(-1)[idx] / rho.reshape(-1)[idx])
    flat[0, idx] = rng.uniform(40.0, 60.0, size=idx.size) * c
    check(dg, state_from_means(rho, v, p, 10))
    # a hypersonic cell whose sum stays below the maximum of a fast, hot cell
    rng, rho, v, p = base(13)
    rho.reshape(-1)[5] = 1.0
    p.reshape(-1)[5] = 1e-6
    v.reshape(3, -1)[:, 5] = (0.9, 0.0, 0.0)  # Mach ~700, s ~ 0.9 / dx
    p.reshape(-1)[20000] = 50.0                # c ~ 9: the maximum
    check(dg, state_from_means(rho, v, p, 10))


def test_cfl_tiny_densities(dg):
    """Densities below the FP32 normal range (1e-40) and large ones (1e35)
    with pressures that keep the means positive."""
    rng, rho, v, p = base(14)
    rho.reshape(-1)[[7, 300, 35000]] = 1e-40
    p.reshape(-1)[[7, 300, 35000]] = 1e-30
    v.reshape(3, -1)[:, [7, 300, 35000]] = 0.0
    rho.reshape(-1)[[11, 12]] = 1e35
    v.reshape(3, -1)[:, [11, 12]] = 0.0  # no cancellation in the FP64 pressure either
    check(dg, state_from_means(rho, v, p, 10))


@pytest.mark.parametrize("order", [2, 4])
def test_cfl_random_states_other_degrees(dg, order):
    """Random positive states with higher modes (which the bound ignores)
    at degrees 1 and 3."""
    N = order * (order + 1) * (order + 2) // 6
    w = syn.random_state(MESH, N, syn.GAMMA, seed=15 + order, high=0.05)
    check(dg, w, order)
