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


def test_rosseland_mean_of_a_transparent_window():
    """1/kappa_R is the dB/dT-weighted mean of 1/kappa: a bin with kappa = 0 and
    nonzero weight makes kappa_R = 0, and two bins of opacities k1, k2 give the
    weighted harmonic mean, k1 k2 (W1 + W2) / (W1 k2 + W2 k1)."""
    nu = np.array([1e13, 1e14])
    assert oracle.rosseland_mean(300.0, nu, [4.0, 0.0]) == 0.0
    k1, k2 = 2.0, 8.0
    got = oracle.rosseland_mean(300.0, nu, [k1, k2])
    # the weights from the single-bin means: W1 / (W1 + W2) from kappa = (1, inf-like)
    w1 = 1.0 / oracle.rosseland_mean(300.0, nu, [1.0, 1e300])
    assert got == pytest.approx(k1 * k2 / (w1 * k2 + (1.0 - w1) * k1), rel=1e-12)
    assert min(k1, k2) < got < max(k1, k2)


def test_geometry_tiles_the_shell():
    """The cells' solid angles and volumes add up to the whole region: 4 pi and
    4 pi (R^3 - r^3) / 3 on the full sphere, (phi range) (cos theta_0 - cos theta_1)
    (R^3 - r^3) / 3 on a wedge; every radial face area is dOmega r^2."""
    r_if = np.geomspace(1.0, 50.0, 13)
    full = fld.Geometry(r_if, np.linspace(0.0, math.pi, 8), np.linspace(0.0, 2 * math.pi, 6))
    assert full.dom.sum() == pytest.approx(4 * math.pi, rel=1e-14)
    assert full.vol.sum() == pytest.approx(4 * math.pi * (50.0 ** 3 - 1.0) / 3, rel=1e-14)
    th = np.linspace(0.3, 1.2, 5)
    wedge = fld.Geometry(r_if, th, np.linspace(0.0, 0.7, 4))
    ref = 0.7 * (math.cos(0.3) - math.cos(1.2)) * (50.0 ** 3 - 1.0) / 3
    assert wedge.vol.sum() == pytest.approx(ref, rel=1e-14)
    # the volume of one cell is the integral of r^2 sin(theta) over it (midpoint rule, 400^2 points)
    m = 400
    r = r_if[3] + (np.arange(m) + 0.5) / m * (r_if[4] - r_if[3])
    t = th[1] + (np.arange(m) + 0.5) / m * (th[2] - th[1])
    quad = (r ** 2).sum() * np.sin(t).sum() * (r_if[4] - r_if[3]) / m * (th[2] - th[1]) / m * (0.7 / 3)
    assert wedge.vol[1, 1, 3] == pytest.approx(quad, rel=1e-5)
    assert wedge.dr2[3] == pytest.approx(r.sum() * (r_if[4] - r_if[3]) / m, rel=1e-12)


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


@pytest.mark.parametrize("case", ["uniform", "layered"])
def test_spherical_steady_state_converges(case):
    """A gray, optically thick shell (D = c/(3 s), g << s), luminosity L released in
    the innermost cell, E = E_bg at the outer edge, dt -> infinity: outside the
    source the flux L / (4 pi r^2) = -D dE/dr gives
    E(r) = E_bg + L / (4 pi) int_r^R dr' / (D(r') r'^2).
    'uniform': one D, a linear radial grid, E = E_bg + L / (4 pi D) (1/r - 1/R).
    'layered': s jumps tenfold at the middle face of a logarithmic radial grid, so
    the face between the layers takes the harmonic mean of the two D and the
    centre distances differ from the cell widths. The finite-volume solution
    converges to the exact one at second order in the radial spacing."""
    r_in, r_out, n = 1.0, 10.0, 40
    s1, L = 1e3, 1e4
    e_bg = 1e-5
    t_bg = (e_bg / fld.radiation_constant()) ** 0.25
    contrast = 10.0 if case == "layered" else 1.0
    errs = []
    for m in (n, 2 * n, 4 * n):
        r_if = np.geomspace(r_in, r_out, m + 1) if case == "layered" else np.linspace(r_in, r_out, m + 1)
        r_j = r_if[m // 2]
        geo = fld.Geometry(r_if, [0.0, math.pi], [0.0, 2 * math.pi])
        rc = geo.rc
        s = np.where(rc < r_j, s1, contrast * s1)[None, None, :]
        rho = np.ones((1, 1, m))
        q = np.zeros((1, 1, m))
        q[0, 0, 0] = L / geo.vol[0, 0, 0]
        e = fld.fld_step(r_if, [0.0, math.pi], [0.0, 2 * math.pi], rho, np.full((1, 1, m), 100.0), q,
                         np.full((1, 1, m), e_bg), 1e300, 1.0, t_bg, [5e14], [s1], kappa_r=s)
        d1, d2 = fld.C / (3 * s1), fld.C / (3 * contrast * s1)
        outer = e_bg + L / (4 * math.pi * d2) * (1 / rc - 1 / r_out)
        inner = e_bg + L / (4 * math.pi * d1) * (1 / rc - 1 / r_j) + L / (4 * math.pi * d2) * (1 / r_j - 1 / r_out)
        exact = np.where(rc >= r_j, outer, inner)
        sel = rc > r_in + 2 * (r_out - r_in) / n
        errs.append(np.max(np.abs(e[0, 0, sel] / exact[sel] - 1)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[0] / errs[2] > 10.0      # second order: ~16x for 4x the cells
    assert errs[2] < 1e-3


def _shell_step(r_if, th_if, ph_if, e_old, dt, s):
    """One step on a shell of cells with kappa_R rho = s everywhere, f_c = 1 (c_V = 0),
    no source, and the background at the mean of e_old's modes (E = 1)."""
    shp = e_old.shape
    t_bg = (1.0 / fld.radiation_constant()) ** 0.25
    return fld.fld_step(r_if, th_if, ph_if, np.ones(shp), np.full(shp, 100.0), np.zeros(shp), e_old, dt, 0.0,
                        t_bg, [5e14], [s], kappa_r=np.full(shp, s))


def _angular_rate_error(n, direction):
    """Relative error of the discrete decay-rate gap of two angular modes against the
    continuum Laplacian on a thin shell (r = 2 .. 2.02). Backward Euler multiplies an
    eigenmode of rate mu by 1 / (1 + dt (beta + mu)); beta, the loss through the outer
    boundary, is the same for every mode, so the gap (1/rho_2 - 1/rho_1) / dt is
    D (mu_2 - mu_1): l(l+1) <1/r^2> for the even Legendre modes P_l(cos theta) on
    the half range 0 .. pi/2 (zero slope at the equator, where the partial range
    ends without flux), m^2 <1/r^2> <1/sin^2 theta> for cos(m (phi - 0.3)) (not
    symmetric about the periodic seam) on a thin equatorial band; <.> are volume
    averages over the cell."""
    r_if = np.array([2.0, 2.02])
    s = 1e10                                   # R = g / s ~ 1e-13: D = c / (3 s)
    d_coef = fld.C / (3.0 * s)
    d3 = (r_if[1] ** 3 - r_if[0] ** 3) / 3.0
    inv_r2 = (r_if[1] - r_if[0]) / d3
    beta = d_coef * r_if[1] ** 2 / (0.5 * (r_if[1] - r_if[0]) * d3)
    dt, eps = 1.0 / beta, 1e-3
    inv = []
    if direction == "theta":
        th_if, ph_if = np.linspace(0.0, 0.5 * math.pi, n + 1), [0.0, 2.0 * math.pi]
        thc = 0.5 * (th_if[1:] + th_if[:-1])
        wgt = np.cos(th_if[:-1]) - np.cos(th_if[1:])
        modes = (2, 4)
        for l in modes:
            pl = special.eval_legendre(l, np.cos(thc))
            e1 = _shell_step(r_if, th_if, ph_if, (1.0 + eps * pl)[None, :, None], dt, s)[0, :, 0]
            inv.append(np.sum(wgt * pl * pl) * eps / np.sum(wgt * pl * (e1 - 1.0)))
        ref = d_coef * (modes[1] * (modes[1] + 1) - modes[0] * (modes[0] + 1)) * inv_r2
    else:
        h = 0.005
        th_if, ph_if = [0.5 * math.pi - h, 0.5 * math.pi + h], np.linspace(0.0, 2.0 * math.pi, n + 1)
        phc = 0.5 * (ph_if[1:] + ph_if[:-1])
        inv_s2 = math.log(math.tan(th_if[1] / 2) / math.tan(th_if[0] / 2)) / (math.cos(th_if[0]) - math.cos(th_if[1]))
        modes = (1, 3)
        for m in modes:
            cm = np.cos(m * (phc - 0.3))
            e1 = _shell_step(r_if, th_if, ph_if, (1.0 + eps * cm)[:, None, None], dt, s)[:, 0, 0]
            inv.append(np.sum(cm * cm) * eps / np.sum(cm * (e1 - 1.0)))
        ref = d_coef * (modes[1] ** 2 - modes[0] ** 2) * inv_r2 * inv_s2
    return abs((inv[1] - inv[0]) / dt / ref - 1.0)


@pytest.mark.parametrize("direction", ["theta", "phi"])
def test_angular_modes_decay_at_the_continuum_rate(direction):
    """The theta and phi couplings (face areas, distances, the periodic wrap) converge
    to the angular part of div(D grad E) at second order: halving the angular
    spacing cuts the error of the decay-rate gap of two modes by 4."""
    errs = [_angular_rate_error(n, direction) for n in (32, 64, 128)]
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5
    assert errs[2] < 3e-3


def test_gradient_of_a_quadratic_field_converges():
    """|grad E| for E = x^2 + 2 y z + 10 z (gradient (2x, 2z, 2y + 10), never 0 on
    the shell 1 <= r <= 2) at the cell centres converges at second order away from
    the one-sided r and theta ends."""
    errs = []
    for n in (16, 32, 64):
        geo = fld.Geometry(np.linspace(1.0, 2.0, n + 1), np.linspace(0.3, math.pi - 0.3, n + 1),
                           np.linspace(0.0, 2.0 * math.pi, n + 1))
        r = geo.rc[None, None, :]
        st, ct = np.sin(geo.thc)[None, :, None], np.cos(geo.thc)[None, :, None]
        sp_, cp_ = np.sin(geo.phc)[:, None, None], np.cos(geo.phc)[:, None, None]
        x, y, z = r * st * cp_, r * st * sp_, r * ct
        e = x * x + 2 * y * z + 10 * z
        exact = np.sqrt((2 * x) ** 2 + (2 * z) ** 2 + (2 * y + 10) ** 2)
        got = fld.gradient_norm(geo, e)
        errs.append(np.max(np.abs(got / exact - 1.0)[:, 1:-1, 1:-1]))
    assert 3.5 < errs[0] / errs[1] and 3.5 < errs[1] / errs[2]
    assert errs[2] < 2e-3


def test_diffusion_coefficient_limits_per_cell():
    """From the cell state (Eqs. 10-13): optically thick cells diffuse with
    D = c / (3 kappa_R rho); in optically thin cells the flux D |grad E| reaches the
    free-streaming value c E."""
    w, g, rho, t = _disk_case()
    geo = fld.Geometry(g.r_if, g.theta_if, g.phi_if)
    e = 1e-5 * (1.0 + 0.5 * np.random.default_rng(7).random(g.shape))
    grad = fld.gradient_norm(geo, e)
    d_thick, _ = fld.cell_coefficients(geo, rho, t, e, 1e30 / rho, 1e8)
    np.testing.assert_allclose(d_thick, fld.C / 3e30, rtol=1e-12)
    d_thin, _ = fld.cell_coefficients(geo, rho, t, e, 1e-40 / rho, 1e8)
    np.testing.assert_allclose(d_thin * grad, fld.C * e, rtol=1e-12)


def test_injected_energy_splits_between_gas_and_radiation():
    """With no transport (D -> 0) the step keeps gas and radiation in equilibrium:
    of the energy q dt injected per volume, the radiation takes dE and the gas
    c_V rho dT with dE = 4 a T^3 dT (E = a T^4 linearised), so dE (1 + c_V rho /
    (4 a T^3)) = q dt: the split that f_c of Eq. 9 expresses."""
    w, g, rho, t = _disk_case()
    a = fld.radiation_constant()
    e0 = a * t ** 4
    q = 1e-12 * (1.0 + np.random.default_rng(8).random(g.shape))
    dt, c_v = 1e5, 1e8
    e1 = fld.fld_step(g.r_if, g.theta_if, g.phi_if, rho, t, q, e0, dt, c_v, 20.0, w.nu, w.kappa,
                      kappa_r=np.full(g.shape, 1e40) / rho)
    de = e1 - e0
    d_temp = de / (4.0 * a * t ** 3)
    np.testing.assert_allclose(de + c_v * rho * d_temp, q * dt, rtol=1e-9)


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
