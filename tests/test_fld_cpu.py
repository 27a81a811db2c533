"""Pins of the FP64 flux-limited-diffusion reference (oracle/fld.py; Sect. 2.1,
Eqs. 7-15) against closed forms, conservation of the discrete step, and the
analytic steady state of spherical diffusion."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import special

import oracle
from oracle import fld
import synth
from tests import _pins


def test_limiter_limits():
    """lambda -> 1/3 in the diffusion limit (R -> 0) and lambda R -> 1 in the
    free-streaming limit (R -> inf), Eq. 12; D -> c/(3 kappa rho) and c E/|grad E|."""
    assert fld.limiter(0.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert fld.limiter(1e8) * 1e8 == pytest.approx(1.0, rel=1e-7)
    assert fld.diffusion_coefficient(2.0, 0.0) == pytest.approx(fld.C / 6.0, rel=1e-15)
    assert fld.diffusion_coefficient(0.0, 4.0) == pytest.approx(fld.C / 4.0, rel=1e-15)
    R = 3.7
    assert fld.diffusion_coefficient(0.5, R * 0.5) == pytest.approx(fld.limiter(R) * fld.C / 0.5, rel=1e-14)


@pytest.mark.parametrize("t", [30.0, 300.0, 3000.0])
def test_rosseland_mean_of_a_power_law(t):
    """1/kappa_R = int kappa^-1 dB/dT / int dB/dT; for kappa = k0 (nu/nu0)^b,
    kappa_R = k0 (kT/(h nu0))^b Gamma(5) zeta(4) / (Gamma(5 - b) zeta(4 - b)),
    reached by 2048 log bins to 1e-4."""
    nu = np.geomspace(1e9, 1e18, 2048)
    k0, nu0, b = 2.0, 1e14, 1.5
    got = oracle.rosseland_mean(t, nu, k0 * (nu / nu0) ** b)
    x = _pins.K_B * t / (_pins.H * nu0)
    ref = k0 * x ** b * special.gamma(5) * special.zeta(4) / (special.gamma(5 - b) * special.zeta(4 - b))
    assert abs(got / ref - 1) < 1e-4
    assert oracle.rosseland_mean(t, [5e14], [3.0]) == pytest.approx(3.0, rel=1e-14)


def _disk_case(nr=10, nth=6, nph=4):
    w = synth.disk3d(nr, nth, nph, n_nu=16, tau550=10.0, seed=3)
    g = w.grid
    rho = w.rho32().astype(np.float64)
    t = np.full(g.shape, 40.0) + 200.0 * np.random.default_rng(1).random(g.shape)
    return w, g, rho, t


def test_uniform_background_is_stationary():
    w, g, rho, _ = _disk_case()
    t_bg = 20.0
    t = np.full(g.shape, t_bg)
    e0 = np.full(g.shape, fld.radiation_constant() * t_bg ** 4)
    e1 = fld.fld_step(g.r_if, g.theta_if, g.phi_if, rho, t, np.zeros(g.shape), e0, 1e8, 1e8, t_bg, w.nu, w.kappa)
    np.testing.assert_allclose(e1, e0, rtol=1e-12)


def test_discrete_energy_balance():
    """Summing the step over the cells, every interior face cancels: the storage
    change sum V (E' - E)/(dt f_c) equals sum V q minus the flux through the outer
    boundary, w_out (E' - a T_bg^4)."""
    w, g, rho, t = _disk_case()
    geo = fld.Geometry(g.r_if, g.theta_if, g.phi_if)
    a = fld.radiation_constant()
    e0 = a * t ** 4
    q = 1e-14 * np.random.default_rng(2).random(g.shape)
    dt, c_v, t_bg = 3e9, 1e8, 10.0
    kr = np.array([oracle.rosseland_mean(tt, w.nu, w.kappa) for tt in t.ravel()]).reshape(g.shape)
    e1 = fld.fld_step(g.r_if, g.theta_if, g.phi_if, rho, t, q, e0, dt, c_v, t_bg, w.nu, w.kappa, kappa_r=kr)
    d, fc = fld.cell_coefficients(geo, rho, t, e0, kr, c_v)
    w_out = d[..., -1] * geo.dom * g.r_if[-1] ** 2 / (g.r_if[-1] - geo.rc[-1])
    lhs = np.sum(geo.vol * (e1 - e0) / (dt * fc))
    rhs = np.sum(geo.vol * q) - np.sum(w_out * (e1[..., -1] - a * t_bg ** 4))
    scale = np.sum(np.abs(geo.vol * (e1 - e0) / (dt * fc))) + np.sum(np.abs(geo.vol * q))
    assert abs(lhs - rhs) <= 1e-9 * scale


@pytest.mark.parametrize("n", [40])
def test_spherical_steady_state_converges(n):
    """One gray, optically thick shell (D = c/(3 s) constant), luminosity L released
    in the innermost cell, E = E_bg at the outer edge, dt -> infinity: outside the
    source E(r) = E_bg + L / (4 pi D) (1/r - 1/R). The finite-volume solution
    converges to it at second order in the radial spacing."""
    r_in, r_out = 1.0, 10.0
    s, L = 1e3, 1e4
    e_bg = 1e-5
    t_bg = (e_bg / fld.radiation_constant()) ** 0.25
    errs = []
    for m in (n, 2 * n, 4 * n):
        r_if = np.linspace(r_in, r_out, m + 1)
        geo = fld.Geometry(r_if, [0.0, math.pi], [0.0, 2 * math.pi])
        rho = np.ones((1, 1, m))
        q = np.zeros((1, 1, m))
        q[0, 0, 0] = L / geo.vol[0, 0, 0]
        e_guess = np.full((1, 1, m), e_bg)
        t = np.full((1, 1, m), 100.0)
        e = fld.fld_step(r_if, [0.0, math.pi], [0.0, 2 * math.pi], rho, t, q, e_guess, 1e300, 1.0, t_bg,
                         [5e14], [s], kappa_r=np.full((1, 1, m), s))
        D = fld.C / (3 * s) * (2 * s + 0.0) / (2 * s)   # g << s: the diffusion limit
        rc = geo.rc
        exact = e_bg + L / (4 * math.pi * D) * (1 / rc - 1 / r_out)
        sel = rc > r_in + 2 * (r_out - r_in) / n
        errs.append(np.max(np.abs(e[0, 0, sel] / exact[sel] - 1)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[0] / errs[2] > 10.0      # second order: ~16x for 4x the cells
    assert errs[2] < 1e-3


def test_row_residuals_vanish_at_the_solution():
    """row_residuals rebuilds single rows independently of assemble: at the direct
    solution every row balances to rounding, and a 1e-3 perturbation of one cell
    shows up in its row and its neighbours' rows only."""
    w, g, rho, t = _disk_case(nr=9, nth=5, nph=4)
    a = fld.radiation_constant()
    e0 = a * t ** 4 * (1.0 + 0.3 * np.random.default_rng(4).random(g.shape))
    q = 1e-13 * np.random.default_rng(5).random(g.shape)
    kr_of_t = lambda tt: oracle.rosseland_mean(tt, w.nu, w.kappa)
    kr = np.array([kr_of_t(tt) for tt in t.ravel()]).reshape(t.shape)
    args = (g.r_if, g.theta_if, g.phi_if, rho, t, q, e0)
    e1 = fld.fld_step(*args, 1e9, 1e8, 15.0, w.nu, w.kappa, kappa_r=kr)
    cells = [(l, j, k) for l in range(4) for j in range(5) for k in range(9)]
    res = fld.row_residuals(*args, e1, 1e9, 1e8, 15.0, kr_of_t, cells)
    assert res.max() < 1e-10
    e2 = e1.copy()
    e2[1, 2, 4] *= 1.001
    res2 = fld.row_residuals(*args, e2, 1e9, 1e8, 15.0, kr_of_t, cells).reshape(4, 5, 9)
    hit = res2 > 1e-8
    assert hit[1, 2, 4] and hit[1, 2, 3] and hit[1, 2, 5] and hit[1, 1, 4] and hit[0, 2, 4] and hit[2, 2, 4]
    assert hit.sum() == 7
