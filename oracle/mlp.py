"""FP64 reference of the learned surrogate: the per-cell quantity it replaces, its
input features, and the 8 -> 128 -> 128 -> 1 SiLU network with its analytic
gradients.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only tests and the benchmark's
CPU legs use it; the CUDA library never does.

What the network replaces (Sect. 2.3, Eqs. 17, 28-32 and 36): along a ray, a cell
whose dust column before it is N_in and whose own column is dN absorbs
    acc = sum_i (F_i / F_max) exp(-kappa_i N_in) (1 - exp(-kappa_i dN))
of the power R*^2 F_max dOmega entering the ray, so q_abs = Gq acc with
Gq = 3 R*^2 F_max / (r+^3 - r-^3), and a_rad = q_abs / (rho c). The network learns
    g = acc / (kappa_550 dN)   (finite as dN -> 0: sum_i (F_i/F_max) kappa_i/kappa_550 e^{-kappa_i N_in}),
so that q_abs = Gq g kappa_550 dN and a_rad = Gq (dr / c) g kappa_550 (no division
by the density). Its output y is ln g standardised: ln g = mu + sigma y.
"""
from __future__ import annotations

import math

import numpy as np

NF = 8          # input features
H = 128         # hidden width

REF_NU = tuple(1e11 * 10.0 ** m for m in range(6))   # reference frequencies of the tau features (Hz)
NU_550 = 2.99792458e10 / 550e-7                      # 550 nm (Hz)
TAU_FLOOR = 2.0 ** -20                               # floors inside the logarithms of the features
DTAU_FLOOR = 2.0 ** -30


def nearest_bin(nu_mid, nu):
    """Index of the bin whose mid-frequency is nearest to nu in |ln nu| (first on ties)."""
    lg = np.log(np.asarray(nu_mid, dtype=np.float64))
    return int(np.argmin(np.abs(lg - math.log(nu))))


def reference_kappas(nu_mid, kappa):
    """(kappa at the six reference frequencies, kappa at 550 nm), nearest bins."""
    k = np.asarray(kappa, dtype=np.float64)
    return np.array([k[nearest_bin(nu_mid, nu)] for nu in REF_NU]), float(k[nearest_bin(nu_mid, NU_550)])


def acc_exact(n_in, dn, kappa, f_bin):
    """acc(N_in, dN) for arrays of cells; kappa, f_bin: all bins (transparent ones add 0)."""
    n_in = np.asarray(n_in, dtype=np.float64)[..., None]
    dn = np.asarray(dn, dtype=np.float64)[..., None]
    k = np.asarray(kappa, dtype=np.float64)
    w = np.asarray(f_bin, dtype=np.float64) / np.max(f_bin)
    return np.sum(w * np.exp(-k * n_in) * (-np.expm1(-k * dn)), axis=-1)


def g_exact(n_in, dn, kappa, f_bin, k550):
    """g = acc / (kappa_550 dN), with its dN -> 0 limit where dN == 0."""
    n_in = np.asarray(n_in, dtype=np.float64)
    dn = np.asarray(dn, dtype=np.float64)
    k = np.asarray(kappa, dtype=np.float64)
    w = np.asarray(f_bin, dtype=np.float64) / np.max(f_bin)
    x = k * dn[..., None]
    # phi(x) = (1 - e^-x) / x, phi(0) = 1
    phi = np.where(x > 0, -np.expm1(-x) / np.where(x > 0, x, 1.0), 1.0)
    return np.sum(w * (k / k550) * np.exp(-k * n_in[..., None]) * phi, axis=-1)


def features(n_in, dn, tdust, kref, k550):
    """The eight inputs: log2 of tau_in at the six reference frequencies / 16, the dust
    temperature (T/1000 - 0.8), and log2 of the cell's own optical depth at 550 nm / 16."""
    n_in = np.asarray(n_in, dtype=np.float64)
    x = np.zeros(n_in.shape + (NF,))
    for m in range(6):
        x[..., m] = np.log2(kref[m] * n_in + TAU_FLOOR) / 16.0
    x[..., 6] = np.asarray(tdust, dtype=np.float64) / 1000.0 - 0.8
    x[..., 7] = np.log2(k550 * np.asarray(dn, dtype=np.float64) + DTAU_FLOOR) / 16.0
    return x


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


class Params:
    """W1 [NF][H], b1 [H], W2 [H][H], b2 [H], w3 [H], b3: z1 = x W1 + b1, h1 = silu(z1),
    z2 = h1 W2 + b2, h2 = silu(z2), y = h2 . w3 + b3."""

    def __init__(self, W1, b1, W2, b2, w3, b3):
        self.W1, self.b1, self.W2, self.b2, self.w3 = (np.asarray(a, dtype=np.float64) for a in
                                                       (W1, b1, W2, b2, w3))
        self.b3 = float(b3)

    @staticmethod
    def from_flat(p):
        p = np.asarray(p, dtype=np.float64)
        assert p.size == N_PARAMS
        o = 0

        def take(n):
            nonlocal o
            v = p[o:o + n]
            o += n
            return v
        W1 = take(NF * H).reshape(NF, H)
        b1 = take(H)
        W2 = take(H * H).reshape(H, H)
        b2 = take(H)
        w3 = take(H)
        b3 = take(1)[0]
        return Params(W1, b1, W2, b2, w3, b3)

    def flat(self):
        return np.concatenate([self.W1.ravel(), self.b1, self.W2.ravel(), self.b2, self.w3, [self.b3]])


N_PARAMS = NF * H + H + H * H + H + H + 1


def forward(p: Params, x):
    """x [B][NF] -> y [B] and the activations the backward pass needs."""
    z1 = x @ p.W1 + p.b1
    h1 = silu(z1)
    z2 = h1 @ p.W2 + p.b2
    h2 = silu(z2)
    y = h2 @ p.w3 + p.b3
    return y, (z1, h1, z2, h2)


def loss_and_grad(p: Params, x, t):
    """Mean squared error of y against t, and its gradient with respect to every
    parameter (a flat vector in the Params.flat order), by the chain rule."""
    x = np.asarray(x, dtype=np.float64)
    y, (z1, h1, z2, h2) = forward(p, x)
    B = x.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    dw3 = h2.T @ dy
    db3 = dy.sum()
    dz2 = np.outer(dy, p.w3) * silu_grad(z2)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ p.W2.T) * silu_grad(z1)
    dW1 = x.T @ dz1
    db1 = dz1.sum(axis=0)
    return loss, Params(dW1, db1, dW2, db2, dw3, db3).flat()


def init_params(seed):
    """Uniform fan-in initialisation (|w| <= 1/sqrt(fan_in)), zero biases; for tests."""
    rng = np.random.default_rng(seed)
    u = lambda shape, fan: rng.uniform(-1.0, 1.0, shape) / math.sqrt(fan)
    return Params(u((NF, H), NF), np.zeros(H), u((H, H), H), np.zeros(H), u(H, H), 0.0)
