"""The seeded input generators (synthetic/) produce what the input recipe
states: the warm-start turbulence is divergence free with rms |v| = M c and
rho = 1, p = 1/gamma; the mode sets of the inputs and of the host driving
agree; OU draws are reproducible; the Sod tube splits the box in halves;
random modal states keep their cell means in the stated ranges; the cell
sample holds both wrap cells."""
import numpy as np

import synthetic as syn
from paper_1602_09079_gb300.forcing import half_space_modes

G = syn.GAMMA


def grid(M):
    g = np.arange(M) / M
    return np.meshgrid(g, g, g, indexing="ij")


def primitives(U, gamma=G):
    rho = U[0]
    v = U[1:4] / rho
    p = (gamma - 1) * (U[4] - 0.5 * rho * np.sum(v * v, axis=0))
    return rho, v, p


def test_warm_start_is_solenoidal_at_the_target_mach():
    M = 16  # resolves |v|^2 (wave numbers up to 4 per axis) exactly
    X, Y, Z = grid(M)
    for seed, mach in ((1234, 0.3), (7, 0.5)):
        rho, v, p = primitives(syn.solenoidal_velocity(seed=seed, mach=mach)(X, Y, Z))
        assert np.max(np.abs(rho - 1)) <= 1e-15 and np.max(np.abs(p - 1 / G)) <= 1e-12
        c = np.sqrt(G * (1 / G) / 1.0)
        rms = np.sqrt(np.mean(np.sum(v * v, axis=0)))
        assert abs(rms - mach * c) <= 1e-12
        # spectral divergence: sum_d k_d v_hat_d = 0 on every wave vector
        k = np.fft.fftfreq(M, 1.0 / M)
        KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
        vh = [np.fft.fftn(v[d]) for d in range(3)]
        div = KX * vh[0] + KY * vh[1] + KZ * vh[2]
        assert np.max(np.abs(div)) <= 1e-10 * np.max(np.abs(vh[0]))
        # all power on 1 <= |n| <= 2
        power = sum(np.abs(h) ** 2 for h in vh)
        kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
        assert power[(kk < 1 - 1e-9) | (kk > 2 + 1e-9)].sum() <= 1e-20 * power.sum()


def test_mode_sets_agree():
    a = syn.driving_modes(1.0, 2.0)
    b = half_space_modes(1.0, 2.0)
    assert sorted(map(tuple, a)) == sorted(map(tuple, b)) and len(a) == 16


def test_ou_noise_is_reproducible():
    z = syn.ou_noise(1234, 5, 16)
    assert z.shape == (5, 16, 6)
    assert np.array_equal(z, syn.ou_noise(1234, 5, 16))
    # a longer stream starts with the same draws
    assert np.array_equal(syn.ou_noise(1234, 9, 16)[:5], z)
    assert not np.array_equal(syn.ou_noise(1235, 5, 16), z)


def test_sod_tube_halves():
    X, Y, Z = grid(64)
    for seed in (1, 2, 3):
        fn, nrm = syn.sod_tube(seed)
        rho, v, p = primitives(fn(X, Y, Z))
        assert abs(np.linalg.norm(nrm) - 1) <= 1e-15
        assert set(np.unique(rho)) == {1.0, 0.125} and np.max(np.abs(v)) == 0.0
        assert np.array_equal(p == 1.0, rho == 1.0) and np.all((p == 1.0) | (np.abs(p - 0.1) <= 1e-15))
        # the planes are tilted against the periodic box, so the split is
        # near, not at, one half
        assert 0.3 <= np.mean(rho == 1.0) <= 0.7


def test_random_state_means_and_positivity():
    n, N = (5, 4, 3), 10
    w = syn.random_state(n, N, G, seed=3, high=0.02)
    assert w.shape == (3, 4, 5, 5, N)
    rho, v, p = primitives(np.moveaxis(w[..., 0], -1, 0))
    assert np.all((rho >= 0.8) & (rho <= 1.2)) and np.all(p > 0)
    assert np.array_equal(w, syn.random_state(n, N, G, seed=3, high=0.02))


def test_sample_cells():
    c = syn.sample_cells(1000, 50, seed=4)
    assert c[0] == 0 and c[-1] == 999 and len(c) == 50
    assert np.all(np.diff(c) > 0)
    assert np.array_equal(syn.sample_cells(10, 50), np.arange(10))
    for nc, cnt in ((1, 5), (2, 5), (7, 1), (7, 2), (7, 3), (128 ** 3, 8192)):
        c = syn.sample_cells(nc, cnt)
        assert len(c) == min(nc, cnt) and len(np.unique(c)) == len(c) and c[0] == 0
        if min(nc, cnt) > 1:
            assert c[-1] == nc - 1
