"""Pins of the oracle's turbulence diagnostics (Sect. 4.1 rms Mach number,
Sect. 4.2 injected energy): closed forms on uniform and piecewise-uniform
states, the zero work of a zero-mean force on uniform momentum, and the
injected power of a single driving mode acting on a velocity wave of the same
wave vector, (V/2) rho0 Re(a . conj(b)), approached at the superconvergent
rate of the L2-projected state."""
import math

import numpy as np
import pytest

import oracle
import synthetic as syn

G = syn.GAMMA


def uniform_state(o, rho, v, p):
    w = np.zeros(o.state_shape)
    w[..., 0, 0] = rho
    w[..., 1:4, 0] = rho * np.asarray(v)
    w[..., 4, 0] = p / (G - 1) + 0.5 * rho * np.dot(v, v)
    return w


def test_uniform_state_mach_and_kinetic_energy():
    o = oracle.Oracle((4, 3, 5), 2, G, L=(1.0, 0.5, 2.0))
    rho, v, p = 1.7, np.array([0.3, -0.4, 0.12]), 0.8
    d = o.diagnostics(uniform_state(o, rho, v, p))
    V = 1.0 * 0.5 * 2.0
    assert abs(d[0] - np.linalg.norm(v) / math.sqrt(G * p / rho)) <= 1e-14
    assert abs(d[1] - 0.5 * rho * np.dot(v, v) * V) <= 1e-14
    assert d[2] == 0.0  # no forcing modes


def test_piecewise_uniform_mach_is_volume_weighted_rms():
    """Two halves of the box with different uniform velocities: the rms Mach
    number is sqrt((M1^2 + M2^2) / 2)."""
    o = oracle.Oracle((4, 2, 2), 1, G)
    w = uniform_state(o, 1.0, np.array([0.2, 0.0, 0.0]), 1.0)
    w2 = uniform_state(o, 2.0, np.array([0.0, -0.6, 0.0]), 0.5)
    w[:, :, 2:] = w2[:, :, 2:]  # x index >= 2
    m1 = 0.2 / math.sqrt(G * 1.0 / 1.0)
    m2 = 0.6 / math.sqrt(G * 0.5 / 2.0)
    d = o.diagnostics(w)
    assert abs(d[0] - math.sqrt(0.5 * (m1 ** 2 + m2 ** 2))) <= 1e-14
    assert abs(d[1] - (0.5 * 0.5 * 1.0 * 0.04 + 0.5 * 0.5 * 2.0 * 0.36)) <= 1e-14


def test_zero_mean_force_does_no_work_on_uniform_momentum():
    o = oracle.Oracle((6, 5, 4), 2, G)
    nv = syn.driving_modes(1.0, 2.0)
    o.set_forcing(nv, np.random.default_rng(3).normal(size=(len(nv), 6)))
    d = o.diagnostics(uniform_state(o, 1.2, np.array([0.3, 0.1, -0.2]), 1.0))
    assert abs(d[2]) <= 1e-13


def _wave_power(n, k):
    o = oracle.Oracle((n, n, n), k, G)
    nv = np.array([[1, 2, 0]], dtype=np.int32)
    ah = np.array([[0.3, -0.2, 0.5, 0.1, 0.4, -0.3]])
    o.set_forcing(nv, ah)
    b = np.array([0.2 + 0.1j, 0.05 - 0.3j, -0.1 + 0.2j])
    rho0, p0 = 1.3, 1.0

    def fn(x, y, z):
        th = 2 * np.pi * (x + 2 * y)
        v = [np.real(b[d] * np.exp(1j * th)) for d in range(3)]
        E = p0 / (G - 1) + 0.5 * rho0 * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
        return np.stack([rho0 + 0 * x, rho0 * v[0], rho0 * v[1], rho0 * v[2], E])

    exact = rho0 * 0.5 * np.real(np.sum((ah[0, :3] + 1j * ah[0, 3:]) * np.conj(b)))
    return o.diagnostics(o.project_fn(fn))[2], exact


def test_injected_power_of_a_driving_mode_on_a_velocity_wave():
    p8, exact = _wave_power(8, 2)
    p16, _ = _wave_power(16, 2)
    e8, e16 = abs(p8 - exact) / abs(exact), abs(p16 - exact) / abs(exact)
    assert e16 <= 3e-5, (e8, e16)
    assert e8 / e16 >= 32.0, (e8, e16)  # rate >= 5 (L2 projection superconvergence)
