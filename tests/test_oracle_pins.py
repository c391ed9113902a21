"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's formulas: each check goes through an
independent route (numpy's Legendre module and Gauss rule, closed forms of
the 1D upwind DG operator, exactness theorems, invariants, brute force in
physical coordinates, numpy's FFT), chosen so that a dropped term, a wrong
sign or index, or a transposed operand fails at least one of them.
"""
import json
import math
import os

import numpy as np
import numpy.polynomial.legendre as npl
import pytest

import synthetic as syn

HERE = os.path.dirname(os.path.abspath(__file__))


def ptilde(u, x):
    """Orthonormal-scaled Legendre polynomial sqrt(2u+1) P_u via numpy."""
    c = np.zeros(u + 1)
    c[u] = 1.0
    return math.sqrt(2 * u + 1) * npl.legval(x, c)


def dptilde(u, x):
    c = np.zeros(u + 1)
    c[u] = 1.0
    return math.sqrt(2 * u + 1) * npl.legval(x, npl.legder(c))


GLL = {2: (np.array([-1.0, 1.0]), np.array([1.0, 1.0])),
       3: (np.array([-1.0, 0.0, 1.0]), np.array([1 / 3, 4 / 3, 1 / 3]))}


# --------------------------------------------------------------- tables

def test_paper_constants(orc):
    gold = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))
    for k, n in gold["modes_per_cell"]["by_degree"].items():
        assert orc.nmodes(int(k)) == n
    for k, w1 in gold["first_gll_weight"]["by_degree"].items():
        x, w = orc.gll(orc.gll_count(int(k)))
        assert abs(w[0] - w1) < 1e-15


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_gauss_matches_numpy(orc, q):
    x, w = orc.gauss(q)
    xr, wr = npl.leggauss(q)
    assert np.max(np.abs(x - xr)) < 1e-15
    assert np.max(np.abs(w - wr)) < 1e-15


@pytest.mark.parametrize("m", [2, 3])
def test_gll_closed_form_and_exactness(orc, m):
    x, w = orc.gll(m)
    assert np.allclose(x, GLL[m][0], atol=1e-15, rtol=0)
    assert np.allclose(w, GLL[m][1], atol=1e-15, rtol=0)
    for d in range(2 * m - 2):  # exact for degree <= 2m - 3
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-15


def test_mode_order(orc):
    e = orc.mode_exponents(2)
    assert [tuple(r) for r in e] == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0),
                                     (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    for k in range(4):
        e = orc.mode_exponents(k)
        assert len(e) == (k + 1) * (k + 2) * (k + 3) // 6
        assert len({tuple(r) for r in e}) == len(e)
        assert np.all(e.sum(1) <= k)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_basis_vs_numpy_legendre(orc, k):
    rng = np.random.default_rng(k)
    e = orc.mode_exponents(k)
    for _ in range(5):
        xi = rng.uniform(-1, 1, 3)
        phi, dphi = orc.basis(k, xi)
        for l, (u, v, w) in enumerate(e):
            pu, pv, pw = ptilde(u, xi[0]), ptilde(v, xi[1]), ptilde(w, xi[2])
            assert abs(phi[l] - pu * pv * pw) < 1e-13
            assert abs(dphi[l, 0] - dptilde(u, xi[0]) * pv * pw) < 1e-12
            assert abs(dphi[l, 1] - pu * dptilde(v, xi[1]) * pw) < 1e-12
            assert abs(dphi[l, 2] - pu * pv * dptilde(w, xi[2])) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3])
def test_basis_orthonormal(orc, k):
    xg, wg = npl.leggauss(k + 2)
    N = orc.nmodes(k)
    G = np.zeros((N, N))
    for a in range(len(xg)):
        for b in range(len(xg)):
            for c in range(len(xg)):
                phi, _ = orc.basis(k, [xg[a], xg[b], xg[c]])
                G += np.outer(phi, phi) * wg[a] * wg[b] * wg[c] / 8.0
    assert np.max(np.abs(G - np.eye(N))) < 1e-14


# ----------------------------------------------------------- projection

@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_projection_exact_for_degree_k(orc, k):
    """Sect. 2.3: with k+1 Gauss points the projection is exact for degree
    <= k polynomials; degree k+1 Legendre terms are orthogonal and must
    vanish exactly as well."""
    rng = np.random.default_rng(10 + k)
    o = orc.Oracle((1, 1, 1), k, syn.GAMMA, L=(2.0, 2.0, 2.0))  # xi = x - 1
    e = orc.mode_exponents(k)
    coef = rng.normal(size=(5, len(e)))
    extra = rng.normal(size=5)

    def fn(x, y, z):
        xi = (x - 1.0, y - 1.0, z - 1.0)
        out = np.zeros((5,) + np.shape(x))
        for i in range(5):
            for l, (u, v, w) in enumerate(e):
                cu = np.zeros(u + 1); cu[u] = 1
                cv = np.zeros(v + 1); cv[v] = 1
                cw = np.zeros(w + 1); cw[w] = 1
                out[i] += coef[i, l] * npl.legval(xi[0], cu) * npl.legval(xi[1], cv) * \
                    npl.legval(xi[2], cw)
            ck = np.zeros(k + 2); ck[k + 1] = 1
            out[i] += extra[i] * npl.legval(xi[1], ck)
        return out

    w = o.project_fn(fn)[0, 0, 0]
    norm = np.array([math.sqrt((2 * u + 1) * (2 * v + 1) * (2 * ww + 1)) for u, v, ww in e])
    assert np.max(np.abs(w - coef / norm)) < 1e-14


# ---------------------------------------------------------------- fluxes

def test_euler_flux_closed_form(orc):
    g = 1.4
    rho, v, p = 1.3, np.array([0.4, -0.7, 0.25]), 2.1
    U = syn.conserved(rho, v[0], v[1], v[2], p, g)
    E = U[4]
    for d in range(3):
        F = orc.euler_flux(d, g, U)
        ref = np.array([rho * v[d], rho * v[d] * v[0], rho * v[d] * v[1], rho * v[d] * v[2],
                        (E + p) * v[d]])
        ref[1 + d] += p
        assert np.max(np.abs(F - ref)) < 1e-14


def _rand_prim(rng, g, vmax=1.0):
    rho = rng.uniform(0.2, 2.0)
    v = rng.uniform(-vmax, vmax, 3)
    p = rng.uniform(0.1, 3.0)
    return syn.conserved(rho, v[0], v[1], v[2], p, g)


def test_hllc_consistency_and_supersonic(orc):
    rng = np.random.default_rng(3)
    g = syn.GAMMA
    for _ in range(50):
        U = _rand_prim(rng, g)
        for d in range(3):
            assert np.allclose(orc.hllc(d, g, U, U), orc.euler_flux(d, g, U), rtol=1e-13, atol=1e-13)
    # supersonic to the right: the flux is the left state's
    UL = syn.conserved(1.0, 5.0, 0.1, 0.0, 0.5, g)
    UR = syn.conserved(0.5, 4.5, -0.2, 0.3, 0.4, g)
    assert np.allclose(orc.hllc(0, g, UL, UR), orc.euler_flux(0, g, UL), rtol=1e-14, atol=0)
    # supersonic to the left: the right state's
    UL = syn.conserved(1.0, -5.0, 0.1, 0.0, 0.5, g)
    UR = syn.conserved(0.5, -4.5, -0.2, 0.3, 0.4, g)
    assert np.allclose(orc.hllc(0, g, UL, UR), orc.euler_flux(0, g, UR), rtol=1e-14, atol=0)


def test_hllc_contact_is_upwind(orc):
    """A contact (equal normal velocity and pressure) is resolved exactly:
    the flux is the upwind state's physical flux."""
    g = syn.GAMMA
    for u in (0.7, -0.4):
        UL = syn.conserved(1.0, u, 0.3, -0.2, 1.0, g)
        UR = syn.conserved(0.3, u, -0.5, 0.1, 1.0, g)
        up = UL if u > 0 else UR
        assert np.allclose(orc.hllc(0, g, UL, UR), orc.euler_flux(0, g, up), rtol=1e-13, atol=1e-14)
    # stationary contact: only the pressure crosses the face
    UL = syn.conserved(1.0, 0.0, 0.0, 0.0, 0.8, g)
    UR = syn.conserved(0.2, 0.0, 0.0, 0.0, 0.8, g)
    assert np.allclose(orc.hllc(2, g, UL, UR), [0, 0, 0, 0.8, 0], atol=1e-14, rtol=0)


def test_hllc_mirror_and_rotation(orc):
    rng = np.random.default_rng(4)
    g = 1.4
    for _ in range(30):
        UL, UR = _rand_prim(rng, g), _rand_prim(rng, g)
        F = orc.hllc(0, g, UL, UR)
        # mirror x -> -x swaps the states and flips normal momentum
        M = np.diag([1.0, -1.0, 1.0, 1.0, 1.0])
        Fm = orc.hllc(0, g, M @ UR, M @ UL)
        assert np.allclose(Fm, -(M @ F), rtol=1e-12, atol=1e-13)
        # rotation: direction 1 (y) with cyclically permuted momenta
        P = np.zeros((5, 5))
        P[0, 0] = P[4, 4] = 1
        P[2, 1] = P[3, 2] = P[1, 3] = 1  # (mx,my,mz) -> (mz,mx,my)
        Fy = orc.hllc(1, g, P @ UL, P @ UR)
        assert np.allclose(Fy, P @ F, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------------ R(w)

def test_free_stream_preservation(orc):
    for k in (1, 2, 3):
        o = orc.Oracle((3, 2, 4), k, 1.4, L=(1.0, 0.7, 1.3))
        w = np.zeros(o.state_shape)
        w[..., 0] = syn.conserved(1.2, 0.3, -0.6, 0.2, 0.9, 1.4)
        R = o.rhs(w)
        assert np.max(np.abs(R)) < 1e-12, k


def _mode_index(orc, k, uvw):
    e = [tuple(r) for r in orc.mode_exponents(k)]
    return e.index(tuple(uvw))


def upwind_dg_1d_operator(nx, k, u, dx):
    """Closed-form 1D upwind DG operator for rho_t + u rho_x = 0 (u > 0) in
    the orthonormal Legendre basis: dx dw_i/dt = u sum_m S_im w_m
    - u rho_j(+1) Pt_i(+1) + u rho_{j-1}(+1) Pt_i(-1), with
    Pt_i(+-1) = (+-1)^i sqrt(2i+1) and S_im = int Pt_m Pt_i' =
    2 sqrt((2i+1)(2m+1)) for m < i, i+m odd."""
    n = k + 1
    S = np.zeros((n, n))
    for i in range(n):
        for m in range(i):
            if (i + m) % 2:
                S[i, m] = 2 * math.sqrt((2 * i + 1) * (2 * m + 1))
    pr = np.array([math.sqrt(2 * i + 1) for i in range(n)])
    pl = np.array([(-1) ** i * math.sqrt(2 * i + 1) for i in range(n)])
    A = np.zeros((nx * n, nx * n))
    for j in range(nx):
        jl = (j - 1) % nx
        A[j * n:(j + 1) * n, j * n:(j + 1) * n] += u * S - u * np.outer(pr, pr)
        A[j * n:(j + 1) * n, jl * n:(jl + 1) * n] += u * np.outer(pl, pr)
    return A / dx


def _wave_state_1d(orc, o, a1d, u, p, g, ny, nz):
    k = o.k
    w = np.zeros(o.state_shape)
    for i in range(k + 1):
        l = _mode_index(orc, k, (i, 0, 0))
        w[:, :, :, 0, l] = a1d[:, i][None, None, :]
        w[:, :, :, 1, l] = u * a1d[:, i][None, None, :]
        w[:, :, :, 4, l] = 0.5 * u * u * a1d[:, i][None, None, :]
    w[..., 4, 0] += p / (g - 1.0)
    return w


@pytest.mark.parametrize("k", [1, 2, 3])
def test_contact_wave_equals_1d_upwind_dg(orc, k):
    """Uniform v = (u,0,0) and p: the density modes follow the 1D upwind DG
    scheme exactly, momentum is u times density, energy 1/2 u^2 times
    density; every mode varying in y or z stays zero."""
    nx, u, p, g = 6, 0.8, 1.0, syn.GAMMA
    rng = np.random.default_rng(20 + k)
    a1d = np.zeros((nx, k + 1))
    a1d[:, 0] = 1.0 + 0.1 * rng.uniform(-1, 1, nx)
    a1d[:, 1:] = 0.05 * rng.normal(size=(nx, k))
    o = orc.Oracle((nx, 2, 3), k, g, L=(1.0, 0.5, 2.0))
    w = _wave_state_1d(orc, o, a1d, u, p, g, 2, 3)
    dw = -o.rhs(w)
    A = upwind_dg_1d_operator(nx, k, u, 1.0 / nx)
    drho = (A @ a1d.reshape(-1)).reshape(nx, k + 1)
    exp = np.zeros_like(dw)
    for i in range(k + 1):
        l = _mode_index(orc, k, (i, 0, 0))
        exp[:, :, :, 0, l] = drho[:, i]
        exp[:, :, :, 1, l] = u * drho[:, i]
        exp[:, :, :, 4, l] = 0.5 * u * u * drho[:, i]
    scale = np.max(np.abs(exp))
    assert np.max(np.abs(dw - exp)) < 1e-12 * scale


def test_rk3_amplification_polynomial(orc):
    """SSP-RK3 on the linear contact-wave operator equals
    I + dt A + dt^2 A^2/2 + dt^3 A^3/6 (Sect. 2.4)."""
    k, nx, u, p, g = 2, 5, 1.0, 1.0, syn.GAMMA
    rng = np.random.default_rng(30)
    a1d = np.zeros((nx, k + 1))
    a1d[:, 0] = 1.0 + 0.1 * rng.uniform(-1, 1, nx)
    a1d[:, 1:] = 0.02 * rng.normal(size=(nx, k))
    o = orc.Oracle((nx, 1, 1), k, g)
    w = _wave_state_1d(orc, o, a1d, u, p, g, 1, 1)
    dt = 0.01
    st, w1 = o.step(w, dt)
    assert st == 0
    A = upwind_dg_1d_operator(nx, k, u, 1.0 / nx) * dt
    M = np.eye(len(A)) + A + A @ A / 2 + A @ A @ A / 6
    exp = (M @ a1d.reshape(-1)).reshape(nx, k + 1)
    got = np.stack([w1[0, 0, :, 0, _mode_index(orc, k, (i, 0, 0))] for i in range(k + 1)], 1)
    assert np.max(np.abs(got - exp)) < 1e-13


def _brute_force_dwdt(orc, n, L, k, g, w):
    """Naive transcription in physical coordinates:
    |K| dw/dt = int_K F . grad(phi) dV - oint_dK (Fhat . n) phi dA, with the
    method's Gauss rules, numpy's Legendre basis, and the outward normal of
    each face handled explicitly (left state = lower cell)."""
    nx, ny, nz = n
    dx = np.array(L) / np.array(n)
    vol = dx.prod()
    e = orc.mode_exponents(k)
    Q = k + 1
    xg, wg = npl.leggauss(Q)

    def phi_at(xi):
        return np.array([ptilde(u, xi[0]) * ptilde(v, xi[1]) * ptilde(ww, xi[2]) for u, v, ww in e])

    def grad_at(xi):  # physical gradient
        return np.array([[dptilde(u, xi[0]) * ptilde(v, xi[1]) * ptilde(ww, xi[2]) * 2 / dx[0],
                          ptilde(u, xi[0]) * dptilde(v, xi[1]) * ptilde(ww, xi[2]) * 2 / dx[1],
                          ptilde(u, xi[0]) * ptilde(v, xi[1]) * dptilde(ww, xi[2]) * 2 / dx[2]]
                         for u, v, ww in e])

    def state(cell, xi):
        ix, iy, iz = cell
        return w[iz % nz, iy % ny, ix % nx] @ phi_at(xi)

    out = np.zeros_like(w)
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                acc = np.zeros((5, len(e)))
                for a in range(Q):
                    for b in range(Q):
                        for c in range(Q):
                            xi = np.array([xg[a], xg[b], xg[c]])
                            dV = wg[a] * wg[b] * wg[c] * vol / 8
                            U = state((ix, iy, iz), xi)
                            G = grad_at(xi)
                            for d in range(3):
                                acc += np.outer(orc.euler_flux(d, g, U), G[:, d]) * dV
                for d in range(3):
                    area = vol / dx[d]
                    others = [o for o in range(3) if o != d]
                    for side in (-1, 1):
                        nb = [ix, iy, iz]
                        nb[d] += side
                        for s in range(Q):
                            for t in range(Q):
                                xi_in = np.zeros(3)
                                xi_in[d] = side
                                xi_in[others[0]] = xg[s]
                                xi_in[others[1]] = xg[t]
                                xi_out = xi_in.copy()
                                xi_out[d] = -side
                                Uin = state((ix, iy, iz), xi_in)
                                Uout = state(tuple(nb), xi_out)
                                if side > 0:
                                    Fh = orc.hllc(d, g, Uin, Uout)
                                else:
                                    Fh = orc.hllc(d, g, Uout, Uin)
                                dA = wg[s] * wg[t] * area / 4
                                acc -= np.outer(Fh * side, phi_at(xi_in)) * dA
                out[iz, iy, ix] = acc / vol
    return out


@pytest.mark.parametrize("k,n,L", [(1, (2, 2, 2), (1.0, 1.0, 1.0)),
                                   (2, (2, 2, 2), (1.0, 1.0, 1.0)),
                                   (2, (3, 2, 2), (1.0, 0.7, 1.3))])
def test_rhs_brute_force_small_mesh(orc, k, n, L):
    g = syn.GAMMA
    o = orc.Oracle(n, k, g, L=L)
    w = syn.random_state(n, o.N, g, seed=40 + k, high=0.02)
    ref = _brute_force_dwdt(orc, n, L, k, g, w)
    got = -o.rhs(w)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_rhs_cells_matches_full(orc):
    o = orc.Oracle((4, 3, 2), 2, syn.GAMMA)
    w = syn.random_state(o.n, o.N, seed=3, high=0.02)
    cells = np.array([0, 5, 23])
    R = o.rhs(w).reshape(o.ncells, 5, o.N)
    assert np.all(np.isfinite(R))
    assert np.array_equal(o.rhs_cells(w, cells), R[cells])


def test_conservation(orc):
    """Face fluxes enter the two cells with opposite signs: the totals
    sum_K |K| w_{i,0} are constant (no forcing, no reset)."""
    o = orc.Oracle((3, 4, 2), 2, syn.GAMMA, L=(1.0, 1.2, 0.8))
    w = syn.random_state(o.n, o.N, seed=8, high=0.02)
    t0 = o.totals(w)
    R = o.rhs(w)
    assert np.max(np.abs(R[..., 0].sum(axis=(0, 1, 2)))) < 1e-12
    for _ in range(3):
        st, w = o.step(w, 2e-3)
        assert st == 0
    assert np.max(np.abs(o.totals(w) - t0) / np.abs(t0).clip(1e-3)) < 1e-13


# --------------------------------------------------------------- limiter

def _limiter_points(k, Q):
    m = 2 if k <= 1 else 3
    h = GLL[m][0]
    xg, _ = npl.leggauss(Q)
    pts = []
    for al in range(3):
        others = [o for o in range(3) if o != al]
        for r in h:
            for s in xg:
                for t in xg:
                    p = np.zeros(3)
                    p[al] = r
                    p[others[0]] = s
                    p[others[1]] = t
                    pts.append(p)
    return np.array(pts)


def _press(U, g):
    return (g - 1) * (U[..., 4] - 0.5 * (U[..., 1] ** 2 + U[..., 2] ** 2 + U[..., 3] ** 2) / U[..., 0])


@pytest.mark.parametrize("k", [1, 2, 3])
def test_limiter_noop_on_smooth(orc, k):
    o = orc.Oracle((3, 3, 3), k, syn.GAMMA)
    w = syn.random_state(o.n, o.N, seed=50 + k, high=0.005)
    st, wl, flags, nl = o.limit(w)
    assert st == 0 and nl == 0
    assert np.array_equal(w, wl)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_limiter_invariants(orc, k):
    """Means unchanged, min over S of density and pressure >= eps after
    limiting, tight where theta1 < 1."""
    g, eps = syn.GAMMA, 1e-2
    o = orc.Oracle((4, 4, 4), k, g, eps_rho=eps, eps_p=eps)
    w = syn.random_state(o.n, o.N, g, seed=60 + k, high=0.6)
    st, wl, flags, nl = o.limit(w)
    assert st == 0
    assert nl > 5
    assert np.array_equal(w[..., 0], wl[..., 0])
    pts = _limiter_points(k, k + 1)
    e = orc.mode_exponents(k)
    phis = np.array([[ptilde(u, p[0]) * ptilde(v, p[1]) * ptilde(ww, p[2]) for u, v, ww in e]
                     for p in pts])
    Ub = np.einsum("zyxil,sl->zyxsi", w, phis)
    Ua = np.einsum("zyxil,sl->zyxsi", wl, phis)
    assert Ua[..., 0].min() >= eps - 1e-12
    assert _press(Ua, g).min() >= eps - 1e-11
    fl = flags.reshape(o.n[2], o.n[1], o.n[0])
    dens_lim = (fl & 1) != 0
    assert np.all(Ub[..., 0].min(-1)[dens_lim] < eps)
    # theta1 is the largest scaling that keeps rho >= eps: the minimum is tight
    # unless the pressure stage scaled the polynomial down further
    only_rho = dens_lim & ((fl & 2) == 0)
    if only_rho.any():
        assert np.max(np.abs(Ua[..., 0].min(-1)[only_rho] - eps)) < 1e-12
    untouched = fl == 0
    assert np.array_equal(w[untouched], wl[untouched])


def test_zhang_shu_mean_identity(orc):
    """The cell mean equals the GLL x Gauss^2 quadrature over each S_alpha
    (exact for degree <= 2m-3), the identity the limiter relies on."""
    for k in (1, 2, 3):
        o = orc.Oracle((2, 2, 2), k, syn.GAMMA)
        w = syn.random_state(o.n, o.N, seed=70 + k, high=0.3)
        m = 2 if k <= 1 else 3
        h, hw = GLL[m]
        xg, wg = npl.leggauss(k + 1)
        for cell in range(8):
            wc = w.reshape(8, 5, o.N)[cell]
            for al in range(3):
                others = [o_ for o_ in range(3) if o_ != al]
                s = np.zeros(5)
                for r, hr in zip(h, hw):
                    for a, wa in zip(xg, wg):
                        for b, wb in zip(xg, wg):
                            xi = np.zeros(3)
                            xi[al] = r
                            xi[others[0]] = a
                            xi[others[1]] = b
                            s += o.eval(w, cell, xi) * hr * wa * wb / 8
                assert np.max(np.abs(s - wc[:, 0])) < 1e-14


def test_newton_tau_vs_quadratic_root(orc):
    """rho(tau) P(tau)/(gamma-1) - rho(tau) eps/(gamma-1) is a quadratic in
    tau along the segment; Newton's root must equal its root in (0,1)."""
    rng = np.random.default_rng(80)
    g, eps = 1.4, 1e-3
    n_checked = 0
    for _ in range(200):
        qbar = syn.conserved(rng.uniform(0.5, 2), *rng.uniform(-1, 1, 3), rng.uniform(0.2, 2), g)
        q = qbar + rng.normal(size=5) * np.array([0.2, 1, 1, 1, 2])
        if q[0] <= 0 or _press(q, g) >= eps:
            continue
        tau, it = orc.pressure_tau(g, qbar, q, eps)
        d = q - qbar
        ep = eps / (g - 1)
        a = d[0] * d[4] - 0.5 * d[1:4] @ d[1:4]
        b = qbar[0] * d[4] + d[0] * qbar[4] - qbar[1:4] @ d[1:4] - ep * d[0]
        c = qbar[0] * qbar[4] - 0.5 * qbar[1:4] @ qbar[1:4] - ep * qbar[0]
        roots = np.roots([a, b, c])
        roots = roots[np.isreal(roots)].real
        roots = roots[(roots > 0) & (roots <= 1)]
        assert len(roots) >= 1
        assert abs(tau - roots.min()) < 1e-13
        assert it < 50
        n_checked += 1
    assert n_checked > 50


# ------------------------------------------------------------- time step

def test_cfl_closed_form(orc):
    g = 1.4
    rho, v, p = 1.1, np.array([0.3, -0.2, 0.1]), 0.9
    c = math.sqrt(g * p / rho)
    n, L = (4, 3, 2), (1.0, 0.9, 0.5)
    dx = np.array(L) / np.array(n)
    # C min(1/(2k+1), w1/2) with w1 = 1 (k=1), 1/3 (k=2,3)
    fac = {1: 1 / 3, 2: 1 / 6, 3: 1 / 7}
    for k in (1, 2, 3):
        o = orc.Oracle(n, k, g, L=L)
        w = np.zeros(o.state_shape)
        w[..., 0] = syn.conserved(rho, v[0], v[1], v[2], p, g)
        w[1, 2, 3, :, 0] = syn.conserved(rho, 2.0, 0.0, 0.0, p, g)  # the fastest cell
        st, dt = o.cfl_dt(w, 0.3)
        vf = np.array([2.0, 0.0, 0.0])
        ref = 0.3 * fac[k] / np.sum((np.abs(vf) + c) / dx)
        assert st == 0 and abs(dt - ref) < 1e-15 * ref


# ------------------------------------------------------------ accuracy

def _l2_error_1d(orc, k, w, nx, exact):
    e = orc.mode_exponents(k)
    xg, wg = npl.leggauss(6)
    err = 0.0
    dx = 1.0 / nx
    for j in range(nx):
        x = (j + 0.5) * dx + 0.5 * dx * xg
        val = np.zeros_like(x)
        for i in range(k + 1):
            l = e.tolist().index([i, 0, 0])
            val += w[0, 0, j, 0, l] * ptilde(i, xg)
        err += np.sum((val - exact(x)) ** 2 * wg) * dx / 2
    return math.sqrt(err)


@pytest.mark.parametrize("k", [1, 2])
def test_convergence_rate_1d_wave(orc, k):
    """Smooth advected density wave: L2 error falls at order k+1 (Sect. 2.1)."""
    g, t_end = syn.GAMMA, 0.2
    fn = syn.smooth_wave_1d(g, amp=0.1, v=(1.0, 0.0, 0.0), p=1.0)
    errs = []
    for nx in (8, 16, 32):
        o = orc.Oracle((nx, 1, 1), k, g)
        w = o.project_fn(fn)
        t = 0.0
        while t < t_end - 1e-14:
            st, dt = o.cfl_dt(w, 0.3)
            dt = min(dt, t_end - t)
            st, w = o.step(w, dt)
            assert st == 0
            t += dt
        errs.append(_l2_error_1d(orc, k, w, nx, lambda x: 1 + 0.1 * np.sin(2 * np.pi * (x - t_end))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > k + 1 - 0.3), (errs, rates)


# ------------------------------------------------------- forcing, reset

def test_forcing_field_vs_fft(orc):
    rng = np.random.default_rng(90)
    nv = syn.driving_modes(1.0, 2.0)
    ah = rng.normal(size=(len(nv), 6))
    o = orc.Oracle((2, 2, 2), 1, syn.GAMMA)
    o.set_forcing(nv, ah)
    M = 8
    grid = np.arange(M) / M
    X, Y, Z = np.meshgrid(grid, grid, grid, indexing="ij")
    xyz = np.stack([X, Y, Z], -1).reshape(-1, 3)
    a = o.forcing_accel(xyz).reshape(M, M, M, 3)
    for d in range(3):
        spec = np.zeros((M, M, M), dtype=complex)
        for j, n in enumerate(nv):
            c = ah[j, d] + 1j * ah[j, 3 + d]
            spec[n[0] % M, n[1] % M, n[2] % M] += c / 2
            spec[-n[0] % M, -n[1] % M, -n[2] % M] += np.conj(c) / 2
        ref = np.real(np.fft.ifftn(spec)) * M ** 3
        assert np.max(np.abs(a[..., d] - ref)) < 1e-12


def test_constant_forcing_source(orc):
    """A spatially constant acceleration (wave vector 0) adds rho a to the
    momentum and m.a to the energy rate of every cell, nothing to higher
    modes of a uniform state."""
    g = syn.GAMMA
    o = orc.Oracle((2, 3, 2), 2, g)
    acc = np.array([0.3, -0.1, 0.2])
    o.set_forcing(np.zeros((1, 3), dtype=np.int32), np.concatenate([acc, [5.0, 5.0, 5.0]]))
    U = syn.conserved(1.3, 0.2, 0.4, -0.3, 0.8, g)
    w = np.zeros(o.state_shape)
    w[..., 0] = U
    dw = -o.rhs(w)
    exp = np.zeros(5)
    exp[1:4] = U[0] * acc
    exp[4] = U[1:4] @ acc
    assert np.max(np.abs(dw[..., 0] - exp)) < 1e-13
    assert np.max(np.abs(dw[..., 1:])) < 1e-13


def test_energy_reset_pins(orc):
    g = syn.GAMMA
    o = orc.Oracle((3, 3, 3), 2, g)
    # driven-turbulence initial state rho = 1, v = 0, p = 1/gamma, c^2 = p/rho:
    # the reset leaves it unchanged
    w = np.zeros(o.state_shape)
    w[..., 0] = syn.conserved(1.0, 0, 0, 0, 1 / g, g)
    st, w2, d = o.energy_reset(w, math.sqrt(1 / g), 1.0)
    assert st == 0 and np.max(np.abs(w2 - w)) < 1e-15 and abs(d) < 1e-15
    # uniform rho != rho0: E = 1/2 m^2/rho + c^2/(gamma-1) rho (rho/rho0)^(gamma-1)
    w[..., 0] = syn.conserved(1.7, 0.3, 0.1, -0.2, 2.0, g)
    st, w2, d = o.energy_reset(w, 0.6, 1.0)
    m2 = (1.7 * 0.3) ** 2 + (1.7 * 0.1) ** 2 + (1.7 * 0.2) ** 2
    E = 0.5 * m2 / 1.7 + 0.36 / (g - 1) * 1.7 * 1.7 ** (g - 1)
    assert abs(w2[0, 0, 0, 4, 0] - E) < 1e-13
    # smooth random state: rho, m untouched; idempotent; dissipation from means
    w = syn.random_state(o.n, o.N, g, seed=95, high=0.01, v_mean=(-0.2, 0.2))
    st, w2, d = o.energy_reset(w, 0.7, 1.0)
    assert o.limit(w2)[3] == 0
    assert np.array_equal(w2[..., :4, :], w[..., :4, :])
    st, w3, d2 = o.energy_reset(w2, 0.7, 1.0)
    assert np.max(np.abs(w3 - w2)) < 1e-14 and abs(d2) < 1e-13

    def e_int(v):
        return v[..., 4, 0] - 0.5 * (v[..., 1, 0] ** 2 + v[..., 2, 0] ** 2 + v[..., 3, 0] ** 2) / v[..., 0, 0]
    ref = np.sum(e_int(w) - e_int(w2)) / o.ncells
    assert abs(d - ref) < 1e-13
