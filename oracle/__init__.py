"""FP64 CPU oracle of the TENET modal DG method (arXiv:1602.09079, Sect. 2-3).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow reference that the
CUDA library is checked against. Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference arm may import it; the product
package never does, and it imports nothing from the product package.

The arithmetic lives in ``dg_oracle.c`` (plain C, FP64, OpenMP over cells);
this module compiles it with gcc and marshals numpy arrays through ctypes.
State layout is the canonical exchange layout ``[nz][ny][nx][5][N]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NONFINITE, ERR_POSITIVITY, ERR_NEWTON = 0, -1, -4, -5, -6


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (portable C, no
    machine-specific flags; FMA contraction off so x86 and Arm agree)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    hdr = os.path.join(_HERE, "dg_oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("k", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3),
                ("gamma", C.c_double), ("eps_rho", C.c_double), ("eps_p", C.c_double),
                ("n_force", C.c_int), ("force_n", C.POINTER(C.c_int32)),
                ("force_a", C.POINTER(C.c_double)), ("flux", C.c_int), ("limiter_points", C.c_int)]

FLUX_HLLC, FLUX_EXACT = 0, 1
LIMIT_S, LIMIT_S_VOLUME = 0, 1


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(Params)
            dp = C.POINTER(C.c_double)
            i64p = C.POINTER(C.c_int64)
            i8p = C.POINTER(C.c_int8)
            i32p = C.POINTER(C.c_int32)
            sig = {
                "orc_nmodes": (C.c_int, [C.c_int]),
                "orc_mode_exponents": (None, [C.c_int, i32p]),
                "orc_gauss": (None, [C.c_int, dp, dp]),
                "orc_gll": (None, [C.c_int, dp, dp]),
                "orc_gll_count": (C.c_int, [C.c_int]),
                "orc_basis": (None, [C.c_int, dp, dp, dp]),
                "orc_volume_points": (C.c_int, [P, dp]),
                "orc_project": (C.c_int, [P, dp, dp]),
                "orc_eval": (None, [P, dp, C.c_long, dp, dp]),
                "orc_euler_flux": (None, [C.c_int, C.c_double, dp, dp]),
                "orc_hllc": (None, [C.c_int, C.c_double, dp, dp, dp]),
                "orc_exact_star": (C.c_int, [C.c_double, dp, dp, dp, dp]),
                "orc_exact_sample": (C.c_int, [C.c_double, dp, dp, C.c_double, dp]),
                "orc_exact_flux": (C.c_int, [C.c_int, C.c_double, dp, dp, dp]),
                "orc_rhs": (C.c_int, [P, dp, dp]),
                "orc_rhs_cells": (C.c_int, [P, dp, C.c_long, i64p, dp]),
                "orc_forcing_accel": (None, [P, C.c_long, dp, dp]),
                "orc_limit": (C.c_int, [P, dp, i8p, i64p]),
                "orc_limit_cells": (C.c_int, [P, dp, C.c_long, i64p, i8p]),
                "orc_pressure_tau": (C.c_double, [C.c_double, dp, dp, C.c_double,
                                                  C.POINTER(C.c_int)]),
                "orc_cfl_dt": (C.c_int, [P, dp, C.c_double, dp]),
                "orc_step": (C.c_int, [P, dp, C.c_double]),
                "orc_energy_reset": (C.c_int, [P, dp, C.c_double, C.c_double, dp]),
                "orc_energy_reset_cells": (C.c_int, [P, dp, C.c_long, i64p, C.c_double,
                                                     C.c_double]),
                "orc_totals": (None, [P, dp, dp]),
                "orc_diagnostics": (None, [P, dp, dp]),
                "orc_sample_velocity": (C.c_int, [P, dp, C.c_int, C.c_int, dp]),
                "orc_sample_density": (C.c_int, [P, dp, C.c_int, dp]),
                "orc_num_threads": (C.c_int, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def nmodes(k: int) -> int:
    return _load().orc_nmodes(k)


def mode_exponents(k: int) -> np.ndarray:
    out = np.zeros((nmodes(k), 3), dtype=np.int32)
    _load().orc_mode_exponents(k, out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out


def gauss(q: int):
    x = np.zeros(q)
    w = np.zeros(q)
    _load().orc_gauss(q, _dp(x), _dp(w))
    return x, w


def gll(m: int):
    x = np.zeros(m)
    w = np.zeros(m)
    _load().orc_gll(m, _dp(x), _dp(w))
    return x, w


def gll_count(k: int) -> int:
    return _load().orc_gll_count(k)


def basis(k: int, xi):
    N = nmodes(k)
    phi = np.zeros(N)
    dphi = np.zeros((N, 3))
    _load().orc_basis(k, _dp(_f64(xi)), _dp(phi), _dp(dphi))
    return phi, dphi


def euler_flux(direction: int, gamma: float, U):
    F = np.zeros(5)
    _load().orc_euler_flux(direction, gamma, _dp(_f64(U)), _dp(F))
    return F


def hllc(direction: int, gamma: float, UL, UR):
    F = np.zeros(5)
    _load().orc_hllc(direction, gamma, _dp(_f64(UL)), _dp(_f64(UR)), _dp(F))
    return F


def exact_star(gamma: float, WL, WR):
    """(status, p*, u*) of the exact Riemann solution for primitive states
    W = (rho, u, p); status 1 = vacuum between two rarefactions."""
    ps, us = np.zeros(1), np.zeros(1)
    st = _load().orc_exact_star(gamma, _dp(_f64(WL)), _dp(_f64(WR)), _dp(ps), _dp(us))
    return st, float(ps[0]), float(us[0])


def exact_sample(gamma: float, WL, WR, s: float):
    W = np.zeros(3)
    st = _load().orc_exact_sample(gamma, _dp(_f64(WL)), _dp(_f64(WR)), float(s), _dp(W))
    return st, W


def exact_flux(direction: int, gamma: float, UL, UR):
    F = np.zeros(5)
    st = _load().orc_exact_flux(direction, gamma, _dp(_f64(UL)), _dp(_f64(UR)), _dp(F))
    assert st >= 0, st
    return F


def pressure_tau(gamma: float, qbar, q, eps: float):
    it = C.c_int(0)
    tau = _load().orc_pressure_tau(gamma, _dp(_f64(qbar)), _dp(_f64(q)), eps, C.byref(it))
    return tau, it.value


def num_threads() -> int:
    return _load().orc_num_threads()


class Oracle:
    """One periodic Cartesian mesh, degree k, ideal gas gamma, optional
    forcing modes; every method takes and returns canonical-layout arrays."""

    def __init__(self, n, k, gamma, L=(1.0, 1.0, 1.0), eps_rho=1e-12, eps_p=1e-12, flux=FLUX_HLLC,
                 limiter_points=LIMIT_S):
        self.n = tuple(int(v) for v in n)
        self.k = int(k)
        self.N = nmodes(self.k)
        self.Q = self.k + 1
        self.gamma = float(gamma)
        self.L = tuple(float(v) for v in L)
        self.ncells = self.n[0] * self.n[1] * self.n[2]
        self._force_n = np.zeros(3, dtype=np.int32)
        self._force_a = np.zeros(6)
        self._p = Params()
        self._p.k = self.k
        for a in range(3):
            self._p.n[a] = self.n[a]
            self._p.L[a] = self.L[a]
        self._p.gamma = self.gamma
        self._p.eps_rho = eps_rho
        self._p.eps_p = eps_p
        self._p.n_force = 0
        self._p.flux = int(flux)
        self._p.limiter_points = int(limiter_points)
        self._p.force_n = self._force_n.ctypes.data_as(C.POINTER(C.c_int32))
        self._p.force_a = _dp(self._force_a)

    @property
    def state_shape(self):
        return (self.n[2], self.n[1], self.n[0], 5, self.N)

    def set_forcing(self, nvec, ahat):
        nvec = np.ascontiguousarray(nvec, dtype=np.int32).reshape(-1, 3)
        ahat = _f64(ahat).reshape(-1, 6)
        assert len(nvec) == len(ahat)
        self._force_n = nvec.copy()
        self._force_a = ahat.copy()
        self._p.n_force = len(nvec)
        self._p.force_n = self._force_n.ctypes.data_as(C.POINTER(C.c_int32))
        self._p.force_a = _dp(self._force_a)

    def _call(self, name, *args):
        st = getattr(_load(), name)(C.byref(self._p), *args)
        return st

    def volume_points(self):
        xyz = np.zeros((self.ncells, self.Q ** 3, 3))
        assert self._call("orc_volume_points", _dp(xyz)) == OK
        return xyz

    def project(self, f):
        f = _f64(f).reshape(self.ncells, 5, self.Q ** 3)
        w = np.zeros(self.state_shape)
        assert self._call("orc_project", _dp(f), _dp(w)) == OK
        return w

    def project_fn(self, fn):
        """Project a callable fn(x, y, z) -> (5, ...) of conserved variables."""
        xyz = self.volume_points()
        vals = np.asarray(fn(xyz[..., 0], xyz[..., 1], xyz[..., 2]), dtype=np.float64)
        return self.project(np.moveaxis(vals, 0, 1))

    def eval(self, w, cell, xi):
        U = np.zeros(5)
        _load().orc_eval(C.byref(self._p), _dp(_f64(w)), int(cell), _dp(_f64(xi)), _dp(U))
        return U

    def rhs(self, w):
        w = _f64(w)
        R = np.zeros_like(w)
        assert self._call("orc_rhs", _dp(w), _dp(R)) == OK
        return R

    def rhs_cells(self, w, cells):
        w = _f64(w)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        R = np.zeros((len(cells), 5, self.N))
        assert self._call("orc_rhs_cells", _dp(w), len(cells),
                          cells.ctypes.data_as(C.POINTER(C.c_int64)), _dp(R)) == OK
        return R

    def forcing_accel(self, xyz):
        xyz = _f64(xyz).reshape(-1, 3)
        a = np.zeros_like(xyz)
        _load().orc_forcing_accel(C.byref(self._p), len(xyz), _dp(xyz), _dp(a))
        return a

    def limit(self, w):
        """Returns (status, limited copy, flags, n_limited)."""
        w = _f64(w).copy()
        flags = np.zeros(self.ncells, dtype=np.int8)
        n = C.c_int64(0)
        st = self._call("orc_limit", _dp(w), flags.ctypes.data_as(C.POINTER(C.c_int8)),
                        C.byref(n))
        return st, w, flags, n.value

    def limit_cells(self, w, cells):
        """Limits the listed cells of a copy; returns (status, copy, flags)."""
        w = _f64(w).copy()
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        flags = np.zeros(len(cells), dtype=np.int8)
        st = self._call("orc_limit_cells", _dp(w), len(cells),
                        cells.ctypes.data_as(C.POINTER(C.c_int64)),
                        flags.ctypes.data_as(C.POINTER(C.c_int8)))
        return st, w, flags

    def cfl_dt(self, w, courant):
        dt = C.c_double(0.0)
        st = self._call("orc_cfl_dt", _dp(_f64(w)), courant, C.byref(dt))
        return st, dt.value

    def step(self, w, dt):
        """One SSP-RK3 step on a copy; returns (status, new state)."""
        w = _f64(w).copy()
        st = self._call("orc_step", _dp(w), float(dt))
        return st, w

    def energy_reset(self, w, c_iso, rho0=1.0):
        w = _f64(w).copy()
        d = C.c_double(0.0)
        st = self._call("orc_energy_reset", _dp(w), float(c_iso), float(rho0), C.byref(d))
        return st, w, d.value

    def energy_reset_cells(self, w, cells, c_iso, rho0=1.0):
        w = _f64(w).copy()
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        st = self._call("orc_energy_reset_cells", _dp(w), len(cells),
                        cells.ctypes.data_as(C.POINTER(C.c_int64)), float(c_iso), float(rho0))
        return st, w

    def totals(self, w):
        out = np.zeros(5)
        _load().orc_totals(C.byref(self._p), _dp(_f64(w)), _dp(out))
        return out

    def sample_velocity(self, w, sub, comp):
        """Velocity component on the (n sub)^3 sub-cell-centre grid,
        array [Z][Y][X]."""
        M = self.n[0] * sub
        out = np.zeros((M, M, M))
        assert self._call("orc_sample_velocity", _dp(_f64(w)), int(sub), int(comp), _dp(out)) == OK
        return out

    def sample_density(self, w, sub):
        M = self.n[0] * sub
        out = np.zeros((M, M, M))
        assert self._call("orc_sample_density", _dp(_f64(w)), int(sub), _dp(out)) == OK
        return out

    def density_pdf(self, w, sub, lo, hi, nb):
        """Sect. 4.4: counts of ln(rho) at the sub-cell centres in nb equal
        bins of [lo, hi), plus the counts below lo (or rho not positive) and
        at or above hi: array of nb + 2."""
        r = self.sample_density(w, sub).ravel()
        out = np.zeros(nb + 2, dtype=np.int64)
        good = r > 0
        out[0] += int(np.count_nonzero(~good))
        sv = np.log(r[good])
        out[0] += int(np.count_nonzero(sv < lo))
        out[nb + 1] = int(np.count_nonzero(sv >= hi))
        mid = sv[(sv >= lo) & (sv < hi)]
        j = np.minimum(np.floor((mid - lo) / (hi - lo) * nb).astype(np.int64), nb - 1)
        out[1:nb + 1] = np.bincount(j, minlength=nb)
        return out

    def velocity_spectrum(self, w, sub):
        """Sect. 3.3: E[b] = sum over integer wave vectors with round(|n|) = b
        of |v_hat(n)|^2 / M^6, summed over the three velocity components (the
        unnormalised DFT of the sampled field by numpy; sum_b E[b] is the
        mean square of the samples by Parseval)."""
        M = self.n[0] * sub
        nb = int(np.floor(np.sqrt(3.0) * M / 2.0)) + 2
        f = np.fft.fftfreq(M, 1.0 / M)
        kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
        b = np.floor(np.sqrt(kx ** 2 + ky ** 2 + kz ** 2) + 0.5).astype(np.int64)
        E = np.zeros(nb)
        for comp in range(3):
            vh = np.fft.fftn(self.sample_velocity(w, sub, comp))
            E += np.bincount(b.ravel(), weights=(np.abs(vh) ** 2).ravel(), minlength=nb)[:nb] / float(M) ** 6
        return E

    def diagnostics(self, w):
        """(rms Mach of the cell means, kinetic energy of the means,
        injected power of the driving force)."""
        out = np.zeros(3)
        _load().orc_diagnostics(C.byref(self._p), _dp(_f64(w)), _dp(out))
        return out
