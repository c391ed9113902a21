"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests
and the benchmark.

This module holds no arithmetic of the DG method: it produces random arrays
and closed-form initial-condition callables ``fn(x, y, z) -> (5, ...)`` of
conserved variables (rho, rho vx, rho vy, rho vz, E) in physical
coordinates. Each side (oracle or CUDA library) evaluates a callable at its
own quadrature points and projects it with its own code.

Workload shapes follow arXiv:1602.09079: periodic unit box (Sect. 3),
smooth advected waves for the accuracy checks, and subsonic driven
turbulence whose driving lives on Fourier modes 1 <= |n| <= 2 (Sect. 3.1).
"""
from __future__ import annotations

import numpy as np

GAMMA = 5.0 / 3.0


def conserved(rho, vx, vy, vz, p, gamma):
    """Primitive -> conserved for an ideal gas."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = np.broadcast(rho, vx, vy, vz, p).shape
    out = np.empty((5,) + shape)
    out[0] = rho
    out[1] = rho * vx
    out[2] = rho * vy
    out[3] = rho * vz
    out[4] = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return out


def random_state(n, N, gamma=GAMMA, seed=0, high=0.02, rho_mean=(0.8, 1.2),
                 v_mean=(-0.5, 0.5), p_mean=(0.6, 1.0)):
    """Random modal state in the canonical layout [nz][ny][nx][5][N].

    Cell means come from primitive means drawn uniformly in the given
    ranges; the higher modes are Gaussian with standard deviation
    ``high`` times the scale of each variable. Small ``high`` gives a smooth
    positive state on which the positivity limiter is inactive; large
    ``high`` gives cells whose polynomial goes negative somewhere."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    shp = (nz, ny, nx)
    rho = rng.uniform(*rho_mean, size=shp)
    v = rng.uniform(*v_mean, size=(3,) + shp)
    p = rng.uniform(*p_mean, size=shp)
    means = conserved(rho, v[0], v[1], v[2], p, gamma)  # (5, nz, ny, nx)
    w = np.zeros(shp + (5, N))
    w[..., 0] = np.moveaxis(means, 0, -1)
    if N > 1:
        scale = np.abs(np.moveaxis(means, 0, -1)) + 0.3
        w[..., 1:] = rng.normal(0.0, 1.0, size=shp + (5, N - 1)) * high * scale[..., None]
    return w


def smooth_wave_1d(gamma=GAMMA, amp=0.1, v=(1.0, 0.0, 0.0), p=1.0):
    """rho = 1 + amp sin(2 pi x), uniform v and p: the advected density
    wave of the 8^3, degree-1 accuracy case."""
    def fn(x, y, z):
        rho = 1.0 + amp * np.sin(2 * np.pi * x)
        one = np.ones_like(rho)
        return conserved(rho, v[0] * one, v[1] * one, v[2] * one, p * one, gamma)
    return fn


def smooth_wave_diag(gamma=GAMMA, amp=0.2, v=(1.0, 1.0, 1.0), p=1.0):
    """rho = 1 + amp sin(2 pi (x+y+z)), uniform v and p: the convergence
    sweep's smooth density wave."""
    def fn(x, y, z):
        rho = 1.0 + amp * np.sin(2 * np.pi * (x + y + z))
        one = np.ones_like(rho)
        return conserved(rho, v[0] * one, v[1] * one, v[2] * one, p * one, gamma)
    return fn


def exact_advected_density(fn_rho, v, t):
    """rho(x, t) = rho0(x - v t) for uniform v and p (entropy wave)."""
    def g(x, y, z):
        return fn_rho(x - v[0] * t, y - v[1] * t, z - v[2] * t)
    return g


def driving_modes(nmin=1.0, nmax=2.0):
    """Integer wave vectors n (k = 2 pi n / L) with nmin <= |n| <= nmax, one
    of each +-n pair (first nonzero component positive)."""
    out = []
    r = int(np.ceil(nmax))
    for a in range(-r, r + 1):
        for b in range(-r, r + 1):
            for c in range(-r, r + 1):
                m = np.sqrt(a * a + b * b + c * c)
                if m < nmin - 1e-12 or m > nmax + 1e-12:
                    continue
                first = next(v for v in (a, b, c) if v != 0)
                if first > 0:
                    out.append((a, b, c))
    return np.array(out, dtype=np.int32)


def ou_noise(seed, n_updates, n_modes):
    """Gaussian draws z_n of the Ornstein-Uhlenbeck driving process
    (Sect. 3.1): shape (n_updates, n_modes, 6), one complex 3-vector per
    mode and update."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_updates, n_modes, 6))


def solenoidal_velocity(seed=1234, mach=0.3, gamma=GAMMA, rho=1.0, p=None, nmin=1.0, nmax=2.0):
    """Warm-start subsonic turbulence: rho = 1, p = 1/gamma, and a
    divergence-free velocity field on the driving modes with random complex
    amplitudes, scaled so its rms over the box equals mach * c, with
    c = sqrt(gamma p / rho). Returns the conserved-variable callable."""
    if p is None:
        p = 1.0 / gamma
    rng = np.random.default_rng(seed)
    nv = driving_modes(nmin, nmax).astype(np.float64)
    amp = rng.standard_normal((len(nv), 2, 3))
    for j, n in enumerate(nv):
        nn = n / np.linalg.norm(n)
        for part in range(2):  # remove the component along n: div v = 0
            amp[j, part] -= nn * (nn @ amp[j, part])
    # mean of |v|^2 over the box for sum_j Re(a_j e^{i k.x}) = 1/2 sum |a_j|^2
    ms = 0.5 * np.sum(amp ** 2)
    cs = np.sqrt(gamma * p / rho)
    scale = mach * cs / np.sqrt(ms)
    amp *= scale

    def fn(x, y, z):
        v = np.zeros((3,) + np.shape(x))
        for j, n in enumerate(nv):
            ph = 2 * np.pi * (n[0] * x + n[1] * y + n[2] * z)
            c, s = np.cos(ph), np.sin(ph)
            for d in range(3):
                v[d] += amp[j, 0, d] * c - amp[j, 1, d] * s
        return conserved(rho * np.ones_like(x), v[0], v[1], v[2], p * np.ones_like(x), gamma)
    return fn


def supersonic_velocity(seed, mach, gamma=GAMMA, compressive=0.5):
    """Supersonic turbulence-like field (rms Mach 2-4): velocity on the
    modes 1 <= |n| <= 3 with a mix of solenoidal and compressive parts, and
    a log-normal density perturbation; used for troubled-cell labels."""
    rng = np.random.default_rng(seed)
    nv = driving_modes(1.0, 3.0).astype(np.float64)
    amp = rng.standard_normal((len(nv), 2, 3))
    for j, n in enumerate(nv):
        nn = n / np.linalg.norm(n)
        for part in range(2):
            lon = nn * (nn @ amp[j, part])
            amp[j, part] = (amp[j, part] - lon) + compressive * lon
    ms = 0.5 * np.sum(amp ** 2)
    p0 = 1.0 / gamma
    scale = mach * np.sqrt(gamma * p0) / np.sqrt(ms)
    amp *= scale
    damp = rng.standard_normal((len(nv), 2)) * 0.3

    def fn(x, y, z):
        v = np.zeros((3,) + np.shape(x))
        lr = np.zeros(np.shape(x))
        for j, n in enumerate(nv):
            ph = 2 * np.pi * (n[0] * x + n[1] * y + n[2] * z)
            c, s = np.cos(ph), np.sin(ph)
            for d in range(3):
                v[d] += amp[j, 0, d] * c - amp[j, 1, d] * s
            lr += damp[j, 0] * c - damp[j, 1] * s
        rho = np.exp(lr)
        return conserved(rho, v[0], v[1], v[2], p0 * rho, gamma)
    return fn


def sod_tube(seed, gamma=GAMMA):
    """3D Sod-type shock tube: rho 1 / 0.125, p 1 / 0.1, v = 0, separated by
    two planes (periodic box) with a random unit normal."""
    rng = np.random.default_rng(seed)
    nrm = rng.standard_normal(3)
    nrm /= np.linalg.norm(nrm)
    off = rng.uniform(0, 1)

    def fn(x, y, z):
        s = (nrm[0] * (x - 0.5) + nrm[1] * (y - 0.5) + nrm[2] * (z - 0.5) + off) % 1.0
        left = s < 0.5
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        zero = np.zeros_like(rho)
        return conserved(rho, zero, zero, zero, p, gamma)
    return fn, nrm


def sample_cells(ncells, count, seed=7):
    """Distinct sorted random cell indices (always including the first and
    last cell so that periodic wrap faces are exercised)."""
    rng = np.random.default_rng(seed)
    count = min(count, ncells)
    pick = rng.choice(ncells, size=count, replace=False)
    ends = ([0, ncells - 1] if ncells > 1 else [0])[:count]
    out = np.unique(np.concatenate([ends, pick[len(ends):]]))
    # an end cell that was also drawn leaves the sample short: top it up with
    # the draws the end cells replaced (distinct from everything kept)
    extra = [c for c in pick[:len(ends)] if c not in out][:count - len(out)]
    return np.unique(np.concatenate([out, extra])).astype(np.int64)
