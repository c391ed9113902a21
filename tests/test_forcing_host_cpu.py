"""Host side of the OU driving (Sect. 3.1), pinned on the CPU: the mode set
by the counts of integer vectors on spheres (r3(1), r3(2), r3(3), r3(4) =
6, 12, 8, 6), the paraboloid weights, the Helmholtz projection (divergence
free, idempotent), the OU process's stationary variance and lag-one
correlation exp(-dt / t_s), and the box rms of the driven field that sets the
driving amplitude, sqrt(sum_j |a_j|^2 / 2), against the oracle's field on a
grid."""
import math

import numpy as np

import oracle
import synthetic as syn
from paper_1602_09079_gb300.forcing import OUDriving, half_space_modes, helmholtz_solenoidal, paraboloid


def test_half_space_modes_counts_and_pairs():
    nv = half_space_modes(1.0, 2.0)
    assert len(nv) == (6 + 12 + 8 + 6) // 2
    sq = np.sum(nv.astype(np.int64) ** 2, axis=1)
    assert sorted(np.unique(sq, return_counts=True)[1].tolist()) == [3, 3, 4, 6]
    pairs = {tuple(v) for v in nv} | {tuple(-v) for v in nv}
    assert len(pairs) == 2 * len(nv)  # no n together with -n
    assert sorted(tuple(v) for v in nv) == [tuple(v) for v in nv]


def test_paraboloid_keeps_the_inner_shells():
    assert paraboloid(1.5) == 1.0 and paraboloid(1.0) == 0.0 and paraboloid(2.0) == 0.0
    assert abs(paraboloid(math.sqrt(2)) - (1 - ((math.sqrt(2) - 1.5) / 0.5) ** 2)) <= 1e-15
    nv = half_space_modes(1.0, 2.0)
    d = OUDriving(nv, 1.0, 0.1, 1.0, np.ones((len(nv), 6)))
    sq = np.sum(d.nvec.astype(np.int64) ** 2, axis=1)
    assert sorted(set(sq.tolist())) == [2, 3] and len(d.nvec) == (12 + 8) // 2


def test_helmholtz_projection():
    rng = np.random.default_rng(5)
    nv = half_space_modes(1.0, 2.0)
    a = rng.normal(size=(len(nv), 6))
    p = helmholtz_solenoidal(nv, a)
    for part in (slice(0, 3), slice(3, 6)):
        assert np.max(np.abs(np.sum(nv * p[:, part], axis=1))) <= 1e-14
    assert np.max(np.abs(helmholtz_solenoidal(nv, p) - p)) <= 1e-15
    # the removed part is parallel to n: a - p = (n . a / |n|^2) n
    for part in (slice(0, 3), slice(3, 6)):
        r = a[:, part] - p[:, part]
        assert np.max(np.abs(np.cross(r, nv))) <= 1e-14


def test_ou_stationary_variance_and_correlation():
    """20,000 independent copies of one mode, 40 updates with f = e^-0.1:
    the variance stays sigma^2 and the lag-one correlation is f (5-sigma
    bands of the sample estimates)."""
    M, sigma = 20000, 0.7
    nv = np.tile(np.array([[1, 1, 0]], dtype=np.int32), (M, 1))
    rng = np.random.default_rng(11)
    d = OUDriving(nv, 2.0, 0.2, 1.0, rng.standard_normal((M, 6)), sigma=sigma)
    assert abs(d.f - math.exp(-0.1)) <= 1e-15
    prev, lag = None, []
    for _ in range(40):
        cur = d.theta.copy()
        if prev is not None:
            lag.append(np.mean(prev * cur) / sigma ** 2)
        prev = cur
        d.update(rng.standard_normal((M, 6)))
    x = d.theta.ravel()
    se_var = sigma ** 2 * math.sqrt(2.0 / x.size)
    assert abs(np.var(x) - sigma ** 2) <= 5 * se_var
    assert abs(np.mean(lag) - d.f) <= 5 * math.sqrt(1.0 / (x.size * len(lag)))
    assert d.n_updates == 40


def test_driving_rms_matches_the_field():
    """The mean of |a(x)|^2 over the unit box of the field the oracle
    evaluates from the amplitudes is sum_j |a_j|^2 / 2 (distinct half-space
    modes), the identity the turbulence driver scales its amplitude by."""
    nv = half_space_modes(1.0, 2.0)
    rng = np.random.default_rng(8)
    d = OUDriving(nv, 1.0, 0.1, 2.5, rng.standard_normal((len(nv), 6)))
    ah = d.ahat()
    o = oracle.Oracle((2, 2, 2), 1, syn.GAMMA)
    o.set_forcing(d.nvec, ah)
    M = 8  # exact for wave numbers up to 2 per axis
    g = np.arange(M) / M
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    a = o.forcing_accel(np.stack([X, Y, Z], -1).reshape(-1, 3))
    ms = np.mean(np.sum(a * a, axis=1))
    assert abs(ms - 0.5 * np.sum(ah ** 2)) <= 1e-12 * ms
    # and the field is divergence free: sum_j n_j . a_j = 0 per mode
    assert np.max(np.abs(np.sum(d.nvec * ah[:, :3], axis=1))) <= 1e-13
