"""Pins of the oracle's density PDF (Sect. 4.4): counts add up to the
number of samples; a uniform density falls in the bin of ln(rho0); a box
split into two uniform halves gives two bins of equal weight; samples
outside [lo, hi) land in the end entries."""
import math

import numpy as np

import oracle
import synthetic as syn

G = syn.GAMMA


def uniform(o, rho):
    w = np.zeros(o.state_shape)
    w[..., 0, 0] = rho
    w[..., 4, 0] = 1.0
    return w


def test_uniform_and_two_halves():
    n, k, sub, nb, lo, hi = (4, 4, 4), 2, 3, 40, -2.0, 2.0
    o = oracle.Oracle(n, k, G)
    M3 = (4 * sub) ** 3
    c = o.density_pdf(uniform(o, 1.7), sub, lo, hi, nb)
    j = int(math.floor((math.log(1.7) - lo) / (hi - lo) * nb))
    assert c.sum() == M3 and c[1 + j] == M3
    w = uniform(o, 0.5)
    w[:, :, 2:, 0, 0] = 3.0  # x index >= 2
    c = o.density_pdf(w, sub, lo, hi, nb)
    ja = int(math.floor((math.log(0.5) - lo) / (hi - lo) * nb))
    jb = int(math.floor((math.log(3.0) - lo) / (hi - lo) * nb))
    assert c[1 + ja] == M3 // 2 and c[1 + jb] == M3 // 2
    c = o.density_pdf(w, sub, -0.5, 0.5, nb)  # ln 0.5 below, ln 3 above
    assert c[0] == M3 // 2 and c[nb + 1] == M3 // 2 and c[1:nb + 1].sum() == 0


def test_counts_of_a_random_state_add_up():
    n, k, sub = (5, 5, 5), 3, 2
    o = oracle.Oracle(n, k, G)
    w = syn.random_state(n, o.N, G, seed=81, high=0.05)
    c = o.density_pdf(w, sub, -0.5, 0.5, 64)
    assert c.sum() == (5 * sub) ** 3
    r = o.sample_density(w, sub)
    assert c[1:65].sum() == np.count_nonzero((np.log(r) >= -0.5) & (np.log(r) < 0.5))


def test_non_positive_density_counts_below():
    """rho = 1 + a Pt1(x) with a sqrt(3) / 2 = 1.299 (sub = 2 puts the
    samples at x = +-1/2): half the samples have rho = -0.299, which has no
    logarithm and is counted in the low end entry, the other half
    rho = 2.299, counted in its own bin."""
    n, k, sub, nb, lo, hi = (3, 3, 3), 1, 2, 16, -1.0, 1.0
    o = oracle.Oracle(n, k, G)
    idx = {tuple(x): i for i, x in enumerate(oracle.mode_exponents(k))}
    w = uniform(o, 1.0)
    w[..., 4, 0] = 5.0
    w[..., 0, idx[(1, 0, 0)]] = 1.5
    M3 = (3 * sub) ** 3
    r = o.sample_density(w, sub)
    assert np.allclose(np.sort(np.unique(np.round(r, 12))), [1 - 0.75 * math.sqrt(3), 1 + 0.75 * math.sqrt(3)])
    c = o.density_pdf(w, sub, lo, hi, nb)
    j = int(math.floor((math.log(1 + 0.75 * math.sqrt(3)) - lo) / (hi - lo) * nb))
    assert c.sum() == M3 and c[0] == M3 // 2 and c[1 + j] == M3 // 2
