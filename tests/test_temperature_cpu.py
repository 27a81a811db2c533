"""Pins of the FP64 oracle's Planck mean and dust-temperature solve (Sect. 2.2,
Eq. 16 in the frequency-dependent form of Sect. 2.3) against closed forms and the
pinned tracer oracle."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import special

import oracle
import synth
from tests import _pins

SIGMA = oracle.sigma_sb()   # pinned to the printed CODATA value in test_oracle_pins
A_RAD = 4.0 * SIGMA / _pins.C


def test_planck_mean_of_one_bin_is_its_opacity():
    """One bin spans 0..inf, so its Planck mean is its opacity at any temperature."""
    for t in (3.0, 300.0, 5800.0, 4e4):
        assert oracle.planck_mean(t, [5e14], [7.5]) == pytest.approx(7.5, rel=1e-14)


@pytest.mark.parametrize("t", [300.0, 3000.0])
def test_planck_mean_of_a_power_law(t):
    """kappa = k0 (nu/nu0)^b averaged over B_nu(T) is k0 (kT/(h nu0))^b
    Gamma(4+b) zeta(4+b) / (Gamma(4) zeta(4)); 128 log bins over 1e11..1e16 Hz
    reproduce it to the binning error (~1e-3)."""
    nu = np.geomspace(1e11, 1e16, 128)
    k0, nu0, b = 2.0, 1e14, 1.5
    kap = k0 * (nu / nu0) ** b
    got = oracle.planck_mean(t, nu, kap)
    x = _pins.K_B * t / (_pins.H * nu0)
    ref = k0 * x ** b * special.gamma(4 + b) * special.zeta(4 + b) / (special.gamma(4) * special.zeta(4))
    assert abs(got / ref - 1) < 2e-3


def test_radiation_only_closed_form():
    """a_rad = 0: a T^4 = E_R."""
    e = np.array([1e-8, 3e-3, 42.0])
    t = oracle.dust_temperature(np.zeros(3), e, synth.nu_bins(16), synth.kappa_synth(synth.nu_bins(16)))
    np.testing.assert_allclose(t, (e / A_RAD) ** 0.25, rtol=1e-13)
    assert oracle.dust_temperature(np.zeros(1), np.zeros(1), [5e14], [1.0])[0] == 0.0


def test_solution_satisfies_eq16():
    nu = synth.nu_bins(40)
    kap = synth.kappa_synth(nu)
    rng = np.random.default_rng(0)
    ar = 10 ** rng.uniform(-8, 2, 50)
    er = 10 ** rng.uniform(-12, -2, 50)
    t = oracle.dust_temperature(ar, er, nu, kap)
    for i in range(50):
        kp = oracle.planck_mean(min(max(t[i], 1.0), 1e5), nu, kap)
        assert abs(A_RAD * t[i] ** 4 / (er[i] + ar[i] / kp) - 1) < 1e-12


def test_gray_thin_sphere_equilibrium():
    """Eq. 16 fed by the tracer oracle's a_rad in the optically thin limit of a gray
    (one-bin) table: a T^4 kappa = kappa F over the cell, F = sigma T*^4 (R*/r)^2, so
    T^4 = T*^4 R*^2 3 dr / (4 (r+^3 - r-^3)) -- at a point, T = T* sqrt(R* / 2r)."""
    g = synth.log_grid(12, 2, 1)
    kap = 0.7
    rho = np.full(g.shape, 1e-40)
    res = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, synth.T_STAR_K, synth.R_STAR_CM, [5e14], [kap], 1500.0,
                           rho, np.full(g.shape, 50.0))
    t = oracle.dust_temperature(res.a_rad, None, [5e14], [kap], t_lo=1e-3, t_hi=1e6)
    r0, r1 = g.r_if[:-1], g.r_if[1:]
    ref = synth.T_STAR_K * (synth.R_STAR_CM ** 2 * 3 * (r1 - r0) / (4 * (r1 ** 3 - r0 ** 3))) ** 0.25
    np.testing.assert_allclose(t[0, 0], ref, rtol=1e-12)
    # the point form T* sqrt(R*/(2r)) at the cell's volume-mean 1/r^2
    rm = ((r1 ** 3 - r0 ** 3) / (3 * (r1 - r0))) ** 0.5
    np.testing.assert_allclose(t[0, 0], synth.T_STAR_K * np.sqrt(synth.R_STAR_CM / (2 * rm)), rtol=1e-12)


def test_gray_and_frequency_agree_when_thin():
    """With kappa_P(T*) as the gray opacity the absorbed stellar power of a thin cell
    is sum_i kappa_i F_i in both, so the dust temperatures agree (Eq. 16, Eq. 19)."""
    g = synth.log_grid(8, 2, 1)
    nu = synth.nu_bins(79)
    kap = synth.kappa_synth(nu)
    rho = np.full(g.shape, 1e-40)
    td = np.full(g.shape, 50.0)
    kp = oracle.planck_mean(synth.T_STAR_K, nu, kap)
    rf = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, synth.T_STAR_K, synth.R_STAR_CM, nu, kap, 1500.0, rho, td)
    rg = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, synth.T_STAR_K, synth.R_STAR_CM, [5e14], [kp], 1500.0, rho, td)
    np.testing.assert_allclose(rf.a_rad, rg.a_rad, rtol=1e-12)
    tf = oracle.dust_temperature(rf.a_rad, None, nu, kap)
    np.testing.assert_allclose(tf, oracle.dust_temperature(rg.a_rad, None, nu, kap), rtol=1e-12)


def test_planck_mean_is_held_outside_the_table_range():
    """kappa_P is evaluated at T clamped to [t_lo, t_hi]: a cell whose solution lies
    below t_lo solves a T^4 = a_rad / kappa_P(t_lo) exactly, one above t_hi
    a T^4 = a_rad / kappa_P(t_hi)."""
    nu = synth.nu_bins(24)
    kap = synth.kappa_synth(nu)
    t_lo, t_hi = 20.0, 400.0
    kp_lo = oracle.planck_mean(t_lo, nu, kap)
    kp_hi = oracle.planck_mean(t_hi, nu, kap)
    assert kp_lo != pytest.approx(kp_hi, rel=1e-3)
    # a_rad chosen so the clamped solutions are 5 K and 2000 K
    ar = np.array([A_RAD * 5.0 ** 4 * kp_lo, A_RAD * 2000.0 ** 4 * kp_hi])
    t = oracle.dust_temperature(ar, None, nu, kap, t_lo=t_lo, t_hi=t_hi)
    np.testing.assert_allclose(t, [5.0, 2000.0], rtol=1e-12)
