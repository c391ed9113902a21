"""Host side of the turbulence driving (arXiv:1602.09079, Sect. 3.1).

The acceleration field lives on a few Fourier modes n (k = 2 pi n / L) with
1 <= |n| <= 2 (k_min = 6.27, k_max = 12.57 for L = 1). Each mode carries a
complex 3-vector driven by an Ornstein-Uhlenbeck process
    theta_t = f theta_{t - dt} + sigma sqrt(1 - f^2) z_n,  f = exp(-dt / t_s),
shaped by a paraboloid in |n| centred between the end points, and made
solenoidal by the Helmholtz projection (delta_ij - n_i n_j / |n|^2). The
Gaussian draws z_n are inputs (the caller supplies them, seeded), so the
sequence is reproducible. Only the resulting amplitudes cross into the CUDA
library (dg_set_forcing); the field is evaluated on the device.
"""
from __future__ import annotations

import math

import numpy as np


def half_space_modes(nmin=1.0, nmax=2.0):
    """Integer wave vectors n with nmin <= |n| <= nmax, one of each +-n pair
    (first nonzero component positive), in lexicographic order."""
    r = int(math.floor(nmax))
    out = []
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            for c in range(-r, r + 1):
                m = math.sqrt(a * a + b * b + c * c)
                first = a if a != 0 else (b if b != 0 else c)
                if first > 0 and nmin - 1e-12 <= m <= nmax + 1e-12:
                    out.append((a, b, c))
    return np.array(out, dtype=np.int32)


def paraboloid(nmag, nmin=1.0, nmax=2.0):
    """Mode amplitude: 1 at the centre (nmin+nmax)/2, 0 at both ends."""
    c = 0.5 * (nmin + nmax)
    h = 0.5 * (nmax - nmin)
    return np.maximum(0.0, 1.0 - ((np.asarray(nmag, dtype=np.float64) - c) / h) ** 2)


def helmholtz_solenoidal(nvec, a):
    """Remove the component of each complex amplitude along its wave vector.
    a: (M, 6) as (Re x, y, z, Im x, y, z)."""
    n = np.asarray(nvec, dtype=np.float64)
    n2 = np.sum(n * n, axis=1, keepdims=True)
    out = np.array(a, dtype=np.float64, copy=True)
    for part in (slice(0, 3), slice(3, 6)):
        v = out[:, part]
        out[:, part] = v - n * np.sum(n * v, axis=1, keepdims=True) / n2
    return out


class OUDriving:
    """OU-driven solenoidal acceleration amplitudes.

    nvec: (M, 3) integer wave vectors (one of each +-n pair); t_s: correlation
    time; dt_update: interval between updates (the paper uses 0.1 t_s);
    amplitude: overall scale (the paper rescales it to reach a target Mach
    number); sigma: OU standard deviation. Modes whose paraboloid weight is
    zero are dropped."""

    def __init__(self, nvec, t_s, dt_update, amplitude, z0, sigma=1.0, nmin=1.0, nmax=2.0):
        nvec = np.asarray(nvec, dtype=np.int32).reshape(-1, 3)
        w = paraboloid(np.linalg.norm(nvec, axis=1), nmin, nmax)
        keep = w > 0
        self.keep = keep
        self.nvec = nvec[keep]
        self.weight = w[keep]
        self.t_s = float(t_s)
        self.dt_update = float(dt_update)
        self.amplitude = float(amplitude)
        self.sigma = float(sigma)
        self.f = math.exp(-self.dt_update / self.t_s)
        z0 = np.asarray(z0, dtype=np.float64).reshape(len(nvec), 6)[keep]
        self.theta = self.sigma * z0  # stationary start
        self.n_updates = 0

    def update(self, z):
        """One OU update with Gaussian draws z of shape (M_all, 6) (the rows
        of dropped modes are ignored)."""
        z = np.asarray(z, dtype=np.float64).reshape(-1, 6)
        if z.shape[0] == len(self.keep):
            z = z[self.keep]
        self.theta = self.f * self.theta + self.sigma * math.sqrt(1.0 - self.f * self.f) * z
        self.n_updates += 1

    def ahat(self):
        """(M, 6) amplitudes for dg_set_forcing."""
        a0 = self.weight[:, None] * self.theta
        return self.amplitude * helmholtz_solenoidal(self.nvec, a0)
