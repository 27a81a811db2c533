"""Pins of the surrogate's FP64 reference (oracle/mlp.py) against things other than
itself: the pinned FP64 tracer, closed forms checked by quadrature, and central
finite differences of the network's loss."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import mlp
import synth


def test_acc_reproduces_the_tracer_oracle():
    """Eqs. 17, 28-32, 36: Gq * acc(N_in, dN), with N_in the masked column summed
    along each ray, equals the FP64 tracer's q_abs in every cell."""
    w = synth.disk3d(24, 8, 4, n_nu=16, tau550=10.0, seed=5)
    orc = oracle.irradiate_workload(w)
    g = w.grid
    rho = w.rho32().astype(np.float64)
    td = w.tdust32().astype(np.float64)
    dr = np.diff(g.r_if)
    dn = np.where(td <= w.t_sub, rho * dr, 0.0)
    n_in = np.cumsum(dn, axis=-1) - dn
    f = oracle.planck_bins(w.t_star, w.nu)
    gq = 3.0 * w.r_star ** 2 * f.max() / (g.r_if[1:] ** 3 - g.r_if[:-1] ** 3)
    q = gq * mlp.acc_exact(n_in, dn, w.kappa, f)
    big = orc.q_abs > 1e-300
    np.testing.assert_allclose(q[big], orc.q_abs[big], rtol=1e-11)
    assert np.all(q[~big] == 0.0)


@pytest.mark.parametrize("kn,kd", [(0.0, 1e-6), (0.3, 0.01), (2.0, 1.5), (7.0, 30.0)])
def test_g_single_bin_is_the_column_average(kn, kd):
    """One gray bin (w = 1, kappa_550 = kappa): g is the mean over the cell's column
    of the attenuation, (1/dN) int_0^dN exp(-kappa (N_in + s)) ds (Eq. 17 averaged
    through the cell)."""
    kappa = 3.0
    n_in, dn = kn / kappa, kd / kappa
    ref, _ = integrate.quad(lambda s: math.exp(-kappa * (n_in + s)), 0.0, dn, epsabs=0, epsrel=1e-13)
    ref /= dn
    got = mlp.g_exact(np.array([n_in]), np.array([dn]), [kappa], [1.0], kappa)[0]
    assert abs(got / ref - 1) < 1e-12


def test_g_limit_and_consistency():
    """g kappa_550 dN = acc; g is continuous at dN -> 0, where it is the
    frequency-weighted opacity ratio (the rho -> 0 force limit)."""
    nu = synth.nu_bins(79)
    kap = synth.kappa_synth(nu)
    f = oracle.planck_bins(synth.T_STAR_K, nu)
    kref, k550 = mlp.reference_kappas(nu, kap)
    n_in = np.array([0.0, 1e-4, 3e-3, 0.05])
    for dn in (1e-3, 1e-6):
        g = mlp.g_exact(n_in, np.full(4, dn), kap, f, k550)
        np.testing.assert_allclose(g * k550 * dn, mlp.acc_exact(n_in, np.full(4, dn), kap, f), rtol=1e-12)
    g0 = mlp.g_exact(n_in, np.zeros(4), kap, f, k550)
    g1 = mlp.g_exact(n_in, np.full(4, 1e-14), kap, f, k550)
    np.testing.assert_allclose(g0, g1, rtol=1e-9)
    ref0 = np.sum(f / f.max() * kap / k550)
    assert abs(g0[0] / ref0 - 1) < 1e-13


def test_reference_bins_of_the_disk_table():
    """The six reference frequencies 1e11..1e16 Hz and 550 nm fall on bins
    0, 16, 31, 47, 62, 78 and 58 of the 79-bin log grid."""
    nu = synth.nu_bins(79)
    assert [mlp.nearest_bin(nu, v) for v in mlp.REF_NU] == [0, 16, 31, 47, 62, 78]
    assert mlp.nearest_bin(nu, mlp.NU_550) == 58


def test_features_encoding():
    kref = np.array([1e-3, 1e-1, 1.0, 10.0, 100.0, 1e4])
    x = mlp.features(np.array([1.0, 0.0]), np.array([0.5, 0.0]), np.array([300.0, 1500.0]), kref, 2.0)
    np.testing.assert_allclose(x[0, :6], np.log2(kref + 2.0 ** -20) / 16, rtol=1e-15)
    np.testing.assert_allclose(x[1, :6], -20.0 / 16)           # N_in = 0 sits on the floor
    assert x[0, 6] == pytest.approx(-0.5) and x[1, 6] == pytest.approx(0.7)
    assert x[0, 7] == pytest.approx(np.log2(1.0 + 2.0 ** -30) / 16)
    assert x[1, 7] == pytest.approx(-30.0 / 16)


def test_gradient_matches_finite_differences():
    """Backward pass (chain rule) against central differences of the FP64 loss,
    on every parameter tensor (a dropped or transposed term fails here)."""
    p = mlp.init_params(3)
    rng = np.random.default_rng(4)
    p.b1 = rng.normal(0, 0.3, mlp.H)
    p.b2 = rng.normal(0, 0.3, mlp.H)
    p.b3 = 0.2
    x = rng.normal(0, 1, (16, mlp.NF))
    t = rng.normal(0, 1, 16)
    _, g = mlp.loss_and_grad(p, x, t)
    flat = p.flat()
    # a sample of indices from every tensor
    sizes = [mlp.NF * mlp.H, mlp.H, mlp.H * mlp.H, mlp.H, mlp.H, 1]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    idx = np.concatenate([o + rng.choice(s, min(s, 12), replace=False) for o, s in zip(offs[:-1], sizes)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        lp, _ = mlp.loss_and_grad(mlp.Params.from_flat(flat + e), x, t)
        lm, _ = mlp.loss_and_grad(mlp.Params.from_flat(flat - e), x, t)
        fd = (lp - lm) / (2 * h)
        # central-difference rounding on a loss of order 1 is ~1e-10 absolute
        assert abs(fd - g[i]) <= 1e-6 * abs(fd) + 1e-9, (i, fd, g[i])


def test_forward_special_cases():
    """With W2 = 0 the output is silu(b2) . w3 + b3 for every input; silu(z) =
    z / (1 + e^-z) has silu(0) = 0, silu(z) -> z for large z and -> 0 for z -> -inf."""
    p = mlp.init_params(1)
    p.W2[:] = 0.0
    p.b2 = np.linspace(-3, 3, mlp.H)
    x = np.random.default_rng(0).normal(0, 1, (5, mlp.NF))
    y, _ = mlp.forward(p, x)
    ref = np.sum(p.b2 / (1 + np.exp(-p.b2)) * p.w3) + p.b3
    np.testing.assert_allclose(y, ref, rtol=1e-14)
    assert mlp.silu(0.0) == 0.0
    assert abs(mlp.silu(40.0) - 40.0) < 1e-15 * 40 * 1e3
    assert abs(mlp.silu(-40.0)) < 1e-15
