"""Pins of the optional limiter point set S u (volume Gauss points)
(Sect. 2.5 asks that the point set contain every point where fluxes are
evaluated): after limiting, density and pressure reach the floors at every
point of the union and the cell means are unchanged; a cell whose polynomial
dips below the floor only at interior Gauss points is left alone by the
S-only limiter and limited by the union."""
import numpy as np

import oracle
import synthetic as syn

G = syn.GAMMA


def points(k):
    Q, m = k + 1, oracle.gll_count(k)
    g, _ = oracle.gauss(Q)
    h, _ = oracle.gll(m)
    S = []
    for al in range(3):
        o = [a for a in range(3) if a != al]
        for r in h:
            for a in g:
                for b in g:
                    x = np.zeros(3)
                    x[al], x[o[0]], x[o[1]] = r, a, b
                    S.append(x)
    V = [np.array([a, b, c]) for c in g for b in g for a in g]
    return S, V


def prim_min(o, w, cell, pts):
    rmin = pmin = np.inf
    for x in pts:
        U = o.eval(w, cell, x)
        p = (G - 1) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0])
        rmin, pmin = min(rmin, U[0]), min(pmin, p)
    return rmin, pmin


def test_union_limiter_reaches_floors_and_keeps_means():
    n, k = (4, 4, 3), 2
    o = oracle.Oracle(n, k, G, limiter_points=oracle.LIMIT_S_VOLUME, eps_rho=1e-3, eps_p=1e-3)
    w = syn.random_state(n, oracle.nmodes(k), G, seed=31, high=0.25)
    st, wl, flags, nl = o.limit(w)
    assert st == 0 and nl > 0
    assert np.array_equal(wl[..., :, 0], w[..., :, 0])
    S, V = points(k)
    for cell in range(o.ncells):
        r, p = prim_min(o, wl, cell, S + V)
        assert r >= 1e-3 * (1 - 1e-12) and p >= 1e-3 * (1 - 1e-9), (cell, r, p)


def test_interior_dip_is_caught_only_by_the_union():
    """A degree-2 density rho = 1 - 0.3 (Pt1 Pt1 cross terms) + 0.26 (Pt2
    pure terms) is lowest at the interior Gauss points (+-s, +-s, +-s),
    s = sqrt(3/5), none of which lies in S. With the floor between its
    minimum over S and over the Gauss points, the S limiter leaves the cell
    unchanged and the union limits it (theta1 < 1) exactly to the floor."""
    k, n = 2, (1, 1, 1)
    S, V = points(k)
    probe = oracle.Oracle(n, k, G)
    idx = {tuple(x): i for i, x in enumerate(oracle.mode_exponents(k))}
    w = np.zeros(probe.state_shape)
    w[..., 0, 0] = 1.0
    w[..., 4, 0] = 50.0  # pressure far from its floor
    for m in ((1, 1, 0), (1, 0, 1), (0, 1, 1)):
        w[..., 0, idx[m]] = -0.3
    for m in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
        w[..., 0, idx[m]] = 0.26
    rS, _ = prim_min(probe, w, 0, S)
    rV, _ = prim_min(probe, w, 0, V)
    assert rV > 0.05 and rS - rV > 0.03
    eps = 0.5 * (rS + rV)
    oS = oracle.Oracle(n, k, G, eps_rho=eps, eps_p=1e-6)
    oU = oracle.Oracle(n, k, G, limiter_points=oracle.LIMIT_S_VOLUME, eps_rho=eps, eps_p=1e-6)
    stS, wS, fS, _ = oS.limit(w)
    stU, wU, fU, _ = oU.limit(w)
    assert stS == 0 and stU == 0
    assert fS[0] == 0 and np.array_equal(wS, w)
    assert fU[0] & 1
    assert abs(prim_min(oU, wU, 0, S + V)[0] - eps) <= 1e-12


def test_face_minimum_gives_the_same_limit_for_both_sets():
    """A linear density rho = 1 + a Pt1(x) takes its minimum at x = -1, a
    GLL end point in S; the interior Gauss points lie above it. With the
    floor above that minimum, theta1 over S and over the union coincide and
    both limiters return the same state bit for bit (pressure stays far from
    its floor at rest)."""
    k, n = 2, (2, 1, 1)
    probe = oracle.Oracle(n, k, G)
    idx = {tuple(x): i for i, x in enumerate(oracle.mode_exponents(k))}
    w = np.zeros(probe.state_shape)
    w[..., 0, 0] = 1.0
    w[..., 4, 0] = 50.0
    w[..., 0, idx[(1, 0, 0)]] = 0.5  # minimum 1 - 0.5 sqrt(3) = 0.134 at x = -1
    S, V = points(k)
    rS, _ = prim_min(probe, w, 0, S)
    rV, _ = prim_min(probe, w, 0, V)
    assert abs(rS - (1 - 0.5 * np.sqrt(3))) <= 1e-14 and rV > rS + 0.05
    eps = 0.2
    oS = oracle.Oracle(n, k, G, eps_rho=eps, eps_p=1e-6)
    oU = oracle.Oracle(n, k, G, limiter_points=oracle.LIMIT_S_VOLUME, eps_rho=eps, eps_p=1e-6)
    stS, wS, fS, _ = oS.limit(w)
    stU, wU, fU, _ = oU.limit(w)
    assert stS == 0 and stU == 0
    assert np.all(fS & 1) and np.array_equal(fS, fU) and np.array_equal(wS, wU)
    assert abs(prim_min(oS, wS, 0, S + V)[0] - eps) <= 1e-12
