"""Pins of the oracle's exact Riemann solver (the exact flux option of
Sect. 2.3, after Eq. dg:eqn:surface_int) against what the Euler equations
fix independently of the solver's construction: the integral conservation
law over the self-similar solution, the Rankine-Hugoniot and Riemann-invariant
relations across its waves, symmetry and Galilean invariance, the supersonic
and contact special cases, and second-order agreement with HLLC for weak
jumps."""
import math

import numpy as np
import pytest

import oracle

G = 1.4


def prim_to_cons(W, vt=(0.0, 0.0), d=0, gamma=G):
    rho, u, p = W
    v = [0.0, 0.0, 0.0]
    v[d] = u
    others = [a for a in range(3) if a != d]
    v[others[0]], v[others[1]] = vt
    E = p / (gamma - 1.0) + 0.5 * rho * sum(x * x for x in v)
    return np.array([rho, rho * v[0], rho * v[1], rho * v[2], E])


def flux1d(W, gamma=G):
    rho, u, p = W
    E = p / (gamma - 1.0) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, (E + p) * u])


def cons1d(W, gamma=G):
    rho, u, p = W
    return np.array([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


CASES = [  # (WL, WR): shock tube, two rarefactions, two shocks, strong shock, mixed, near vacuum
    ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),
    ((1.0, -1.8, 0.5), (1.0, 2.1, 0.4)),
    ((6.0, 19.6, 460.0), (6.0, -6.2, 46.0)),
    ((1.0, 0.0, 800.0), (1.0, 0.0, 0.02)),
    ((0.5, 0.3, 2.0), (1.5, -0.7, 0.3)),
    ((1.0, -3.5, 0.5), (0.8, 3.6, 0.45)),
    ((1.0, -3.7, 0.4), (1.0, 3.7, 0.4)),  # two rarefactions just short of a vacuum
]


@pytest.mark.parametrize("WL,WR", CASES)
def test_integral_conservation_of_sampled_solution(WL, WR):
    """For the Riemann problem at t = 1, int_{-M}^{M} U(x) dx equals
    M (U_L + U_R) + F(U_L) - F(U_R) for M beyond the fastest wave: the
    sampled solution carries the right mass, momentum and energy (wrong star
    densities, wave speeds or fan profiles all break it)."""
    WL, WR = np.array(WL), np.array(WR)
    cmax = max(abs(WL[1]) + math.sqrt(G * WL[2] / WL[0]), abs(WR[1]) + math.sqrt(G * WR[2] / WR[0]))
    st, ps, us = oracle.exact_star(G, WL, WR)
    assert st in (0, 1)
    M = 3.0 * (cmax + abs(us) + 1.0)
    n = 200000
    xs = -M + (np.arange(n) + 0.5) * (2 * M / n)
    tot, umax = np.zeros(3), np.zeros(3)
    for x in xs:
        s2, W = oracle.exact_sample(G, WL, WR, x)
        if W[0] > 0:
            U = cons1d(W)
            tot += U
            umax = np.maximum(umax, np.abs(U))
    tot *= 2 * M / n
    expect = M * (cons1d(WL) + cons1d(WR)) + flux1d(WL) - flux1d(WR)
    # midpoint rule over a few jumps: error ~ (2M/n) x jump, far below the
    # 1e-3 relative effect of a 1% error in a star state
    assert np.all(np.abs(tot - expect) <= 5e-5 * M * umax), (tot, expect)


def sample(WL, WR, s):
    st, W = oracle.exact_sample(G, WL, WR, s)
    assert st >= 0
    return W


@pytest.mark.parametrize("WL,WR", CASES[:5])
def test_wave_relations(WL, WR):
    """Star-region states satisfy the Rankine-Hugoniot conditions across a
    shock (speed from the mass jump) and the isentrope and Riemann invariant
    across a rarefaction, on each side."""
    st, ps, us = oracle.exact_star(G, WL, WR)
    assert st == 0
    for side, Wk in ((0, np.array(WL)), (1, np.array(WR))):
        eps = 1e-9 * (1 + abs(us))
        Ws = sample(WL, WR, us - eps if side == 0 else us + eps)
        assert abs(Ws[2] - ps) <= 1e-12 * ps and abs(Ws[1] - us) <= 1e-12 * (1 + abs(us))
        ck = math.sqrt(G * Wk[2] / Wk[0])
        cs = math.sqrt(G * Ws[2] / Ws[0])
        if ps > Wk[2]:
            Us, Uk = cons1d(Ws), cons1d(Wk)
            S = (Us[1] - Uk[1]) / (Us[0] - Uk[0])
            jump_f = flux1d(Ws) - flux1d(Wk)
            assert np.allclose(jump_f, S * (Us - Uk), rtol=1e-11, atol=1e-11 * np.abs(flux1d(Wk)).max())
        else:
            sgn = 1.0 if side == 0 else -1.0
            # isentrope p / rho^gamma and Riemann invariant u +- 2c/(gamma-1)
            assert abs(Ws[2] / Ws[0] ** G - Wk[2] / Wk[0] ** G) <= 1e-12 * Wk[2] / Wk[0] ** G
            assert abs((Ws[1] + sgn * 2 * cs / (G - 1)) - (Wk[1] + sgn * 2 * ck / (G - 1))) <= 1e-11 * (1 + ck)


def test_fan_is_self_similar_and_continuous():
    """Inside a rarefaction fan, u - c = x/t (left fan) and the state joins
    the outer and star states continuously at the fan edges."""
    WL, WR = np.array([1.0, -1.0, 1.0]), np.array([1.0, 1.0, 1.0])
    st, ps, us = oracle.exact_star(G, WL, WR)
    assert st == 0 and ps < 1.0 and abs(us) < 1e-14
    cL = math.sqrt(G)
    head, tail = WL[1] - cL, us - cL * (ps / WL[2]) ** ((G - 1) / (2 * G))
    for s in np.linspace(head + 1e-6, tail - 1e-6, 7):
        W = sample(WL, WR, s)
        assert abs(W[1] - math.sqrt(G * W[2] / W[0]) - s) < 1e-12
    for edge in (head, tail):
        a, b = sample(WL, WR, edge - 1e-10), sample(WL, WR, edge + 1e-10)
        assert np.allclose(a, b, rtol=1e-8)


def test_symmetric_collision_two_shock_closed_form():
    """u_L = -u_R = U, equal rho and p: u* = 0 and (p* - p)^2 A = U^2 (p* + B)
    with A = 2/((gamma+1) rho), B = (gamma-1)/(gamma+1) p (two equal shocks)."""
    rho, p, U = 1.3, 0.7, 2.0
    st, ps, us = oracle.exact_star(G, [rho, U, p], [rho, -U, p])
    A, B = 2 / ((G + 1) * rho), (G - 1) / (G + 1) * p
    x = (U * U + math.sqrt(U ** 4 + 4 * A * U * U * (p + B))) / (2 * A)
    assert st == 0 and abs(us) <= 1e-14 and abs(ps - (p + x)) <= 1e-13 * ps


def test_two_rarefaction_closed_form():
    """When both waves are rarefactions the Riemann invariants give p* in
    closed form: p* = ((cL + cR - (gamma-1)/2 (uR - uL)) / (cL pL^-z + cR pR^-z))^(1/z),
    z = (gamma-1)/(2 gamma)."""
    WL, WR = [1.0, -0.5, 1.0], [0.6, 0.8, 0.7]
    cL, cR = math.sqrt(G * 1.0 / 1.0), math.sqrt(G * 0.7 / 0.6)
    z = (G - 1) / (2 * G)
    p = ((cL + cR - 0.5 * (G - 1) * (0.8 + 0.5)) / (cL / 1.0 ** z + cR / 0.7 ** z)) ** (1 / z)
    st, ps, us = oracle.exact_star(G, WL, WR)
    assert st == 0 and ps < 0.7 and abs(ps - p) <= 1e-13 * p


def test_galilean_invariance_and_mirror_symmetry():
    WL, WR = np.array([1.0, 0.2, 1.0]), np.array([0.3, -0.4, 0.2])
    st, ps, us = oracle.exact_star(G, WL, WR)
    V = 0.77
    st2, ps2, us2 = oracle.exact_star(G, WL + [0, V, 0], WR + [0, V, 0])
    assert abs(ps2 - ps) <= 1e-13 * ps and abs(us2 - (us + V)) <= 1e-13
    for s in (-1.5, -0.3, 0.0, 0.4, 1.2):
        a, b = sample(WL, WR, s), sample(WL + [0, V, 0], WR + [0, V, 0], s + V)
        assert np.allclose(a + [0, V, 0], b, rtol=1e-12, atol=1e-12)
    # mirror x -> -x: swap the sides and negate the velocities
    st3, ps3, us3 = oracle.exact_star(G, WR * [1, -1, 1], WL * [1, -1, 1])
    assert abs(ps3 - ps) <= 1e-13 * ps and abs(us3 + us) <= 1e-13
    for s in (-1.0, -0.2, 0.3):
        a, b = sample(WL, WR, s), sample(WR * [1, -1, 1], WL * [1, -1, 1], -s)
        assert np.allclose(a * [1, -1, 1], b, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_flux_special_cases(d):
    """Consistency F(U, U) = F(U); a contact (equal u and p) gives the
    upwind physical flux with the upwind tangential velocity; supersonic
    flow gives the upwind flux; the flux is rotation-consistent."""
    rng = np.random.default_rng(5 + d)
    for _ in range(5):
        W = np.array([rng.uniform(0.5, 2), rng.uniform(-0.5, 0.5), rng.uniform(0.5, 2)])
        U = prim_to_cons(W, vt=rng.uniform(-1, 1, 2), d=d)
        assert np.allclose(oracle.exact_flux(d, G, U, U), oracle.euler_flux(d, G, U), rtol=1e-13, atol=1e-13)
        # contact: same u (> 0) and p, other density and tangential velocity
        UL = prim_to_cons([1.0, 0.3, 1.0], vt=(0.5, -0.2), d=d)
        UR = prim_to_cons([0.4, 0.3, 1.0], vt=(-0.9, 0.1), d=d)
        assert np.allclose(oracle.exact_flux(d, G, UL, UR), oracle.euler_flux(d, G, UL), rtol=1e-13, atol=1e-14)
        UL = prim_to_cons([1.0, -0.3, 1.0], vt=(0.5, -0.2), d=d)
        UR = prim_to_cons([0.4, -0.3, 1.0], vt=(-0.9, 0.1), d=d)
        assert np.allclose(oracle.exact_flux(d, G, UL, UR), oracle.euler_flux(d, G, UR), rtol=1e-13, atol=1e-14)
        # supersonic to the right and to the left
        UL = prim_to_cons([1.0, 3.0, 1.0], vt=(0.1, 0.2), d=d)
        UR = prim_to_cons([0.5, 2.5, 0.8], vt=(0.3, 0.0), d=d)
        assert np.allclose(oracle.exact_flux(d, G, UL, UR), oracle.euler_flux(d, G, UL), rtol=1e-13)
        UL = prim_to_cons([1.0, -3.0, 1.0], vt=(0.1, 0.2), d=d)
        UR = prim_to_cons([0.5, -2.9, 0.8], vt=(0.3, 0.0), d=d)
        assert np.allclose(oracle.exact_flux(d, G, UL, UR), oracle.euler_flux(d, G, UR), rtol=1e-13)
    # rotation: direction d with permuted components equals direction 0
    WL, WR = [1.0, 0.4, 1.2], [0.7, -0.6, 0.5]
    F0 = oracle.exact_flux(0, G, prim_to_cons(WL, (0.2, -0.1), 0), prim_to_cons(WR, (0.3, 0.4), 0))
    Fd = oracle.exact_flux(d, G, prim_to_cons(WL, (0.2, -0.1), d), prim_to_cons(WR, (0.3, 0.4), d))
    others = [a for a in range(3) if a != d]
    assert np.allclose([Fd[0], Fd[1 + d], Fd[1 + others[0]], Fd[1 + others[1]], Fd[4]], F0, rtol=1e-13)


def test_weak_jumps_agree_with_hllc_to_second_order():
    """Both Riemann fluxes reduce to the same linearised flux for weak jumps:
    their difference shrinks like the square of the jump."""
    U0 = prim_to_cons([1.0, 0.2, 1.0], vt=(0.1, -0.3))
    dU = np.array([0.3, -0.2, 0.1, 0.25, 0.4])
    diffs = []
    for h in (1e-1, 5e-2, 2.5e-2):
        UL, UR = U0 - h * dU, U0 + h * dU
        diffs.append(np.abs(oracle.exact_flux(0, G, UL, UR) - oracle.hllc(0, G, UL, UR)).max())
    r = np.log2(np.array(diffs[:-1]) / np.array(diffs[1:]))
    assert np.all(r > 1.7), (diffs, r)


def test_vacuum_generation():
    """Strong expansion (2(cL + cR)/(gamma-1) <= uR - uL) opens a vacuum:
    status 1, zero density between the rarefaction tails, zero flux through a
    face at the centre of a symmetric expansion."""
    WL, WR = [1.0, -10.0, 1.0], [1.0, 10.0, 1.0]
    st, ps, us = oracle.exact_star(G, WL, WR)
    assert st == 1 and ps == 0.0
    st, W = oracle.exact_sample(G, WL, WR, 0.0)
    assert st == 1 and W[0] == 0.0 and W[2] == 0.0
    F = oracle.exact_flux(0, G, prim_to_cons(WL), prim_to_cons(WR))
    assert np.abs(F).max() == 0.0


def test_rhs_with_exact_flux_free_stream_and_conservation():
    """With the exact flux, R vanishes on a uniform state and the totals
    sum_K |K| w_i0 are conserved over steps of a random smooth state."""
    import synthetic as syn
    n, k = (4, 3, 5), 2
    o = oracle.Oracle(n, k, syn.GAMMA, flux=oracle.FLUX_EXACT)
    w = np.zeros(o.state_shape)
    w[..., :, 0] = prim_to_cons([1.2, 0.3, 0.9], vt=(-0.2, 0.1), gamma=syn.GAMMA)
    R = o.rhs(w)
    assert np.abs(R).max() <= 1e-13 * np.abs(w).max() * max(n)
    w = syn.random_state(n, o.N, syn.GAMMA, seed=77, high=0.01)
    t0 = o.totals(w)
    for _ in range(5):
        st, w = o.step(w, 0.2 * o.cfl_dt(w, 0.3)[1])
        assert st == 0
    assert np.allclose(o.totals(w), t0, rtol=1e-14, atol=1e-14)
