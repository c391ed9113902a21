"""FP64 numpy oracle of the learned troubled-cell indicator.

TEST INFRASTRUCTURE ONLY (see the package docstring): the reference the
GPU's BF16 feature, forward and backward kernels are checked against.

No counterpart in the paper: the paper's only limiter is the positivity
limiter of Sect. 2.5, whose indicator (the polynomial leaves the positive
set somewhere on S) provides the labels. The indicator network reads, per
cell:
  own   w_{i,l} / s_i for l >= 1, i = 0..4 (variable-major), with scales
        s_rho = |rho|, s_m = sqrt(|rho E|) for the three momenta, s_E = |E|
        from the cell means;
  extra log(rho_mean) and the mean Mach number |m|/rho / c;
  bound sum_{l>=1} |w_{i,l}| max_S |phi_l| / s_i for i = 0..4, the largest
        excursion of each variable's polynomial from its mean over the
        positivity point set S (Sect. 2.5), relative to the scale s_i;
  nbr   (mean_i(neighbour) - mean_i(cell)) / s_i for the 26 neighbours of
        the 3x3x3 block, offsets (dz, dy, dx) in lexicographic order of
        {-1, 0, 1}^3 without (0,0,0), variable-minor;
zero-padded to a multiple of 32 features. Network: 2 hidden layers of 64
ReLU units, one logit, sigmoid; loss: class-weighted binary cross entropy.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64


def n_features(k: int) -> int:
    N = (k + 1) * (k + 2) * (k + 3) // 6
    return 5 * (N - 1) + 2 + 5 + 26 * 5


def n_features_padded(k: int) -> int:
    f = n_features(k)
    return (f + 31) // 32 * 32


def neighbour_offsets():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dz, dy, dx) != (0, 0, 0)]


def max_abs_basis_on_S(k):
    """max over the positivity point set S of |phi_l|, from the oracle's own
    Gauss/GLL rules and basis."""
    import oracle
    Q, m = k + 1, oracle.gll_count(k)
    xg, _ = oracle.gauss(Q)
    xh, _ = oracle.gll(m)
    best = np.zeros(oracle.nmodes(k))
    for al in range(3):
        others = [o for o in range(3) if o != al]
        for r in xh:
            for a in xg:
                for b in xg:
                    xi = np.zeros(3)
                    xi[al], xi[others[0]], xi[others[1]] = r, a, b
                    phi, _ = oracle.basis(k, xi)
                    best = np.maximum(best, np.abs(phi))
    return best


def features(w, k, gamma):
    """w: canonical state [nz][ny][nx][5][N] -> X [n_cells][F_padded]."""
    w = np.asarray(w, dtype=np.float64)
    nz, ny, nx, _, N = w.shape
    mean = w[..., :, 0]
    rho, m, E = mean[..., 0], mean[..., 1:4], mean[..., 4]
    sm = np.sqrt(np.abs(rho * E))
    s = np.stack([np.abs(rho), sm, sm, sm, np.abs(E)], axis=-1)
    own = (w[..., :, 1:] / s[..., :, None]).reshape(nz, ny, nx, 5 * (N - 1))
    m2 = np.sum(m * m, axis=-1)
    p = (gamma - 1.0) * (E - 0.5 * m2 / rho)
    c = np.sqrt(gamma * p / rho)
    mach = np.sqrt(m2) / rho / c
    extra = np.stack([np.log(rho), mach], axis=-1)
    M = max_abs_basis_on_S(k)
    bound = (np.abs(w[..., :, 1:]) @ M[1:]) / s
    nbr = []
    for dz, dy, dx in neighbour_offsets():
        shifted = np.roll(mean, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        nbr.append((shifted - mean) / s)
    nbr = np.concatenate(nbr, axis=-1)
    X = np.concatenate([own, extra, bound, nbr], axis=-1).reshape(-1, n_features(k))
    out = np.zeros((X.shape[0], n_features_padded(k)))
    out[:, : X.shape[1]] = X
    return out


def init_params(f_in, seed):
    """He-uniform initial weights (the random draws both sides start from)."""
    rng = np.random.default_rng(seed)

    def he(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=shape)

    return {
        "W1": he(f_in, (HIDDEN, f_in)), "b1": np.zeros(HIDDEN),
        "W2": he(HIDDEN, (HIDDEN, HIDDEN)), "b2": np.zeros(HIDDEN),
        "w3": he(HIDDEN, (HIDDEN,)), "b3": np.zeros(1),
    }


def forward(P, X):
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    logit = h2 @ P["w3"] + P["b3"][0]
    return {"z1": z1, "h1": h1, "z2": z2, "h2": h2, "logit": logit}


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def loss(logit, y, pos_weight):
    """-(1/B) sum [a y log s(z) + (1 - y) log(1 - s(z))], in the stable form
    log s(z) = -softplus(-z), log(1 - s(z)) = -softplus(z)."""
    sp_neg = np.logaddexp(0.0, -logit)
    sp_pos = np.logaddexp(0.0, logit)
    return float(np.mean(pos_weight * y * sp_neg + (1.0 - y) * sp_pos))


def backward(P, X, cache, y, pos_weight):
    """Gradients of loss() with respect to every parameter, by the chain
    rule through the two ReLU layers."""
    B = X.shape[0]
    s = sigmoid(cache["logit"])
    dlogit = (s * (pos_weight * y + 1.0 - y) - pos_weight * y) / B
    g = {}
    g["w3"] = cache["h2"].T @ dlogit
    g["b3"] = np.array([dlogit.sum()])
    dz2 = np.outer(dlogit, P["w3"]) * (cache["z2"] > 0)
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"]) * (cache["z1"] > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return g
