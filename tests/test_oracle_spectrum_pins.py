"""Pins of the oracle's velocity power spectrum (Sect. 3.3): Parseval
(the shells sum to the mean square of the sampled velocity, computed
directly), a uniform flow puts all its power in shell 0, and a single
Fourier mode of the velocity puts its power, half its squared amplitude, in
the shell of its wave number."""
import numpy as np

import oracle
import synthetic as syn

G = syn.GAMMA


def test_parseval_and_uniform_flow():
    n, k, sub = (6, 6, 6), 2, 3
    o = oracle.Oracle(n, k, G)
    w = syn.random_state(n, o.N, G, seed=61, high=0.05)
    E = o.velocity_spectrum(w, sub)
    ms = np.mean([np.mean(o.sample_velocity(w, sub, c) ** 2) for c in range(3)]) * 3
    assert abs(E.sum() - ms) <= 1e-12 * ms
    u = np.zeros(o.state_shape)
    u[..., 0, 0] = 1.3
    u[..., 1:4, 0] = 1.3 * np.array([0.2, -0.1, 0.4])
    u[..., 4, 0] = 2.0
    E = o.velocity_spectrum(u, sub)
    assert abs(E[0] - 0.21) <= 1e-14 and np.abs(E[1:]).max() <= 1e-28


def test_single_mode_lands_in_its_shell():
    n, k, sub = (8, 8, 8), 3, 4
    o = oracle.Oracle(n, k, G)
    b = np.array([0.1 + 0.05j, -0.08j, 0.03])

    def fn(x, y, z):
        th = 2 * np.pi * (x + 2 * y)  # n = (1, 2, 0), |n| = 2.24 -> shell 2
        v = [np.real(b[d] * np.exp(1j * th)) for d in range(3)]
        rho = 1.0 + 0 * x
        return syn.conserved(rho, v[0], v[1], v[2], 1.0 + 0 * x, G)

    E = o.velocity_spectrum(o.project_fn(fn), sub)
    total = 0.5 * np.sum(np.abs(b) ** 2)
    assert E[2] >= 0.999 * E.sum()
    assert abs(E.sum() - total) <= 1e-3 * total
