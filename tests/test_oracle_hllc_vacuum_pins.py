"""Pins of the oracle's HLLC flux at vacuum-level pressures (Sect. 2.3 asks
for a positivity-preserving flux; at the positivity floor a face pressure
can round to <= 0): the sound speed of such a state is 0, the limit
p -> 0+, so the flux is finite and continuous as p passes through zero; a
receding pair with both sound speeds 0 has no wave structure and gets the
flux of a vacuum interface, (0, p_L e_d, 0)."""
import numpy as np

import oracle
import synthetic as syn

G = syn.GAMMA


def cons(rho, v, p):
    return np.array([rho, rho * v[0], rho * v[1], rho * v[2], p / (G - 1) + 0.5 * rho * np.dot(v, v)])


def test_continuous_through_zero_pressure():
    for d in range(3):
        vL, vR = np.zeros(3), np.zeros(3)
        vL[d], vR[d] = -0.3, 0.2
        vL[(d + 1) % 3] = 0.1
        UR = cons(0.9, vR, 0.5)
        F = [oracle.hllc(d, G, cons(1.0, vL, p), UR) for p in (-1e-14, 0.0, 1e-14)]
        assert all(np.all(np.isfinite(f)) for f in F)
        # |F(p) - F(0)| ~ rho u c with c ~ sqrt(p): small at p ~ 1e-14
        assert np.max(np.abs(F[0] - F[1])) <= 1e-6 and np.max(np.abs(F[2] - F[1])) <= 1e-6


def test_receding_vacuum_interface():
    for d in range(3):
        vL, vR = np.zeros(3), np.zeros(3)
        vL[d], vR[d] = -0.24, 0.12
        vL[(d + 1) % 3] = 0.07
        for pL, pR in ((-1e-4, -3e-4), (0.0, 0.0), (-1e-12, 0.0)):
            F = oracle.hllc(d, G, cons(0.9989, vL, pL), cons(0.9451, vR, pR))
            expect = np.zeros(5)
            expect[1 + d] = pL
            assert np.max(np.abs(F - expect)) <= 1e-15, (d, pL, pR, F)


def test_unchanged_for_positive_pressures():
    """Away from zero pressure the flux is Toro's HLLC: consistency
    F(U, U) = F(U), and the upwind flux when both states are supersonic in
    the same direction."""
    rng = np.random.default_rng(5)
    for _ in range(10):
        d = int(rng.integers(3))
        U = cons(rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.2, 2))
        assert np.max(np.abs(oracle.hllc(d, G, U, U) - oracle.euler_flux(d, G, U))) <= 1e-14 * np.max(np.abs(U))
        # both states supersonic to +e_d (S_L = min(u_L - c_L, u~ - c~) > 0):
        # the upwind flux F(U_L)
        vl, vr = rng.uniform(-0.5, 0.5, 3), rng.uniform(-0.5, 0.5, 3)
        vl[d], vr[d] = 5.0, 4.5
        UL, UR = cons(1.0, vl, 0.5), cons(0.8, vr, 0.4)
        assert np.max(np.abs(oracle.hllc(d, G, UL, UR) - oracle.euler_flux(d, G, UL))) <= 1e-13
