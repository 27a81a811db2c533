"""Pins of the FP64 oracle against things other than itself.

Each test names the passage it follows. Together they are chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign, an off-by-one in
the optical-depth scan, transposed theta/phi, the wrong bin edge) fails at
least one of them; ``test_oracle_mutants.py`` checks that claim by planting
such slips in copies of the oracle.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import _pins

T_STAR = synth.T_STAR_K
R_STAR = synth.R_STAR_CM
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_grid(nr=8, nth=3, nph=2, stretch=True):
    if stretch:
        return synth.stretched_grid(nr, nth, nph, stretch=1.1)
    return synth.log_grid(nr, nth, nph)


# --------------------------------------------------------------------------
# Eq. 18 / Eq. 20: stellar boundary flux
# --------------------------------------------------------------------------
def test_sigma_is_a_c_over_4():
    """Eq. 18: sigma_SB = a c / 4, against the printed CODATA values."""
    s = oracle.sigma_sb()
    assert abs(s / _pins.SIGMA_PRINTED - 1) < 2e-10
    assert abs(s / (0.25 * _pins.A_RAD_PRINTED * _pins.C) - 1) < 2e-9


@pytest.mark.parametrize("n_nu", [1, 2, 5, 32, 79])
def test_planck_bins_against_quadrature(n_nu):
    """Eq. 20: each bin flux equals pi * int B_nu over [mid(i-1,i), mid(i,i+1)],
    outer edges 0 and infinity, computed here by adaptive quadrature."""
    nu = synth.nu_bins(n_nu)
    f = oracle.planck_bins(T_STAR, nu)
    ref = _pins.bin_fluxes_quad(T_STAR, nu)
    big = ref > 1e-20 * ref.sum()
    np.testing.assert_allclose(f[big], ref[big], rtol=2e-11)
    np.testing.assert_allclose(f[~big], ref[~big], atol=1e-20 * ref.sum())
    # the bins tile the whole spectrum: sum = sigma T^4 (Eq. 18)
    assert abs(f.sum() / (_pins.SIGMA_PRINTED * T_STAR ** 4) - 1) < 2e-10


@pytest.mark.parametrize("t", [300.0, 5800.0, 40000.0])
def test_planck_bins_other_temperatures(t):
    nu = synth.nu_bins(16)
    f = oracle.planck_bins(t, nu)
    ref = _pins.bin_fluxes_quad(t, nu)
    big = ref > 1e-14 * ref.sum()
    np.testing.assert_allclose(f[big], ref[big], rtol=2e-11)
    assert abs(f.sum() / (_pins.SIGMA_PRINTED * t ** 4) - 1) < 2e-10


def test_planck_split_is_continuous():
    """The small-x series and the large-x series meet: H(x) + G(x) = pi^4/15."""
    for x in [0.3, 0.8, 1.0, 1.5]:
        tot = oracle.planck_band(0.0, x) + oracle.planck_band(x, math.inf)
        assert abs(tot / (math.pi ** 4 / 15) - 1) < 1e-14


# --------------------------------------------------------------------------
# Eq. 17 with tau = 0: the optically thin limit
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["rho0", "sublimated"])
def test_thin_limit(mode):
    """Eq. 17 with tau = 0: F(r) = L*/(4 pi r^2); nothing absorbed, all escapes.
    The force per unit mass tends to sum_i kappa_i F_i(r)/c averaged over the cell."""
    g = small_grid(10, 4, 3)
    nu = synth.nu_bins(12)
    kap = synth.kappa_synth(nu)
    rho = np.full(g.shape, 1e-18) if mode == "sublimated" else np.zeros(g.shape)
    td = np.full(g.shape, 2000.0) if mode == "sublimated" else np.full(g.shape, 50.0)
    r = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, T_STAR, R_STAR, nu, kap, 1500.0,
                         rho, td, want_flux=True)
    lstar = 4 * math.pi * R_STAR ** 2 * _pins.SIGMA_PRINTED * T_STAR ** 4
    thin = lstar / (4 * math.pi * g.r_if ** 2)
    np.testing.assert_allclose(r.flux_if, np.broadcast_to(thin, r.flux_if.shape), rtol=1e-9)
    assert np.all(r.q_abs == 0.0)
    assert r.e_abs == 0.0
    assert abs(r.e_esc / lstar - 1) < 1e-9
    f_bin = _pins.bin_fluxes_quad(T_STAR, nu)
    dr = np.diff(g.r_if)
    expect_a = (np.sum(kap * f_bin) * R_STAR ** 2 * dr / (_pins.shell_volumes(g.r_if) * _pins.C))
    if mode == "sublimated":
        assert np.all(r.a_rad == 0.0)
    else:
        np.testing.assert_allclose(r.a_rad, np.broadcast_to(expect_a, r.a_rad.shape), rtol=1e-10)


# --------------------------------------------------------------------------
# uniform gray sphere: analytic exp(-kappa rho (r - r_min))
# --------------------------------------------------------------------------
def test_uniform_gray_sphere_closed_form():
    """Eqs. 17 + 19 with one bin and constant kappa rho, tau(r_min) = 0:
    P_k = L* dOmega/(4 pi) [exp(-kr (r_- - r_min)) - exp(-kr (r_+ - r_min))],
    evaluated at 40 digits so the difference does not cancel."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    g = small_grid(16, 3, 2)
    kap = np.array([300.0])
    nu = np.array([synth.NU_550NM_HZ])
    # total optical depth 6 along every ray
    rho_val = 6.0 / (kap[0] * (g.r_if[-1] - g.r_if[0]))
    rho = np.full(g.shape, rho_val)
    r = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, T_STAR, R_STAR, nu, kap, 1500.0,
                         rho, np.full(g.shape, 100.0))
    lstar = 4 * math.pi * R_STAR ** 2 * _pins.SIGMA_PRINTED * T_STAR ** 4
    dom = _pins.solid_angles(g.theta_if, g.phi_if)
    kr = mpmath.mpf(kap[0]) * mpmath.mpf(rho_val)
    rmin = mpmath.mpf(g.r_if[0])
    ref = np.empty(g.nr)
    for k in range(g.nr):
        ref[k] = float(mpmath.exp(-kr * (mpmath.mpf(g.r_if[k]) - rmin)) -
                       mpmath.exp(-kr * (mpmath.mpf(g.r_if[k + 1]) - rmin)))
    expect = lstar / (4 * math.pi) * dom[:, :, None] * ref[None, None, :]
    np.testing.assert_allclose(r.p_abs, expect, rtol=3e-10)  # sigma printed to 10 digits
    # same thing relative to the oracle's own L*, to full precision
    np.testing.assert_allclose(r.p_abs / r.l_star * 4 * math.pi,
                               dom[:, :, None] * ref[None, None, :], rtol=1e-13)
    # a_rad = q/(rho c) for rho > 0 (Sect. 5)
    np.testing.assert_allclose(r.a_rad, r.q_abs / (rho_val * _pins.C), rtol=1e-13)
    esc = float(mpmath.exp(-kr * (mpmath.mpf(g.r_if[-1]) - rmin)))
    assert abs(r.e_esc / (r.l_star * esc) - 1) < 1e-13


# --------------------------------------------------------------------------
# brute-force quadrature of Eq. 27/28 on tiny grids
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1])
def test_brute_force_quadrature(seed):
    """Cell-integrated absorption and force (Eqs. 27-32 carried to spherical shells,
    Eq. 36) against adaptive quadrature of kappa rho F(r) r^2 across every cell,
    with F from Eq. 17 and a continuous tau(r); bin fluxes from quadrature too."""
    rng = np.random.default_rng(seed)
    g = small_grid(6, 3, 2)
    nu = synth.nu_bins(3)
    kap = np.array([0.5, 40.0, 3000.0])
    # per-cell optical depths 1e-4 .. 5 at the middle bin
    dr = np.diff(g.r_if)
    dtau = 10 ** rng.uniform(-4, 0.7, size=g.shape)
    rho = dtau / (kap[1] * dr[None, None, :])
    td = rng.uniform(20, 1600, size=g.shape)
    td[0, 1, 2] = 1500.0                # exactly at t_sub: dust survives
    r = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, T_STAR, R_STAR, nu, kap, 1500.0, rho, td)
    P, A = _pins.brute_force_cells(g.r_if, g.theta_if, g.phi_if, T_STAR, R_STAR, nu, kap,
                                   1500.0, rho, td)
    tiny = P.max() * 1e-30
    np.testing.assert_allclose(r.p_abs, P, rtol=1e-10, atol=tiny)
    vol = _pins.solid_angles(g.theta_if, g.phi_if)[:, :, None] * _pins.shell_volumes(g.r_if)
    np.testing.assert_allclose(r.a_rad, A / (vol * _pins.C), rtol=1e-10,
                               atol=1e-30 * np.max(A / vol))
    assert np.all(r.q_abs[td > 1500.0] == 0.0) and np.all(r.a_rad[td > 1500.0] == 0.0)


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------
@pytest.mark.parametrize("wl", ["disk2d", "disk3d_small", "thick"])
def test_energy_conservation(wl):
    """Eqs. 33-35 (flux difference telescopes along a ray): absorbed plus escaped
    power equals the stellar luminosity into the grid, to 1e-12."""
    if wl == "disk2d":
        w = synth.disk2d()
    elif wl == "disk3d_small":
        w = synth.disk3d(48, 16, 8, n_nu=24, tau550=10.0, seed=5)
    else:
        w = synth.disk2d(48, 24, 40, tau550=100.0)
    r = oracle.irradiate_workload(w)
    assert abs(r.rel_err) < 1e-12
    assert r.e_abs > 0 and r.e_esc > 0
    lstar = 4 * math.pi * w.r_star ** 2 * _pins.SIGMA_PRINTED * w.t_star ** 4
    assert abs(r.l_star / lstar - 1) < 3e-10


def test_flux_difference_form():
    """Eq. 33/36: the absorbed power equals dOmega (r_-^2 F(r_-) - r_+^2 F(r_+)),
    the flux-divergence form, where that difference does not cancel."""
    w = synth.disk3d(40, 12, 4, n_nu=16, tau550=30.0, seed=2)
    r = oracle.irradiate_workload(w, want_flux=True)
    g = w.grid
    dom = _pins.solid_angles(g.theta_if, g.phi_if)
    r2f = r.flux_if * g.r_if[None, None, :] ** 2
    diff = dom[:, :, None] * (r2f[:, :, :-1] - r2f[:, :, 1:])
    ok = diff > 1e-3 * dom[:, :, None] * r2f[:, :, :-1]
    assert ok.sum() > 50
    np.testing.assert_allclose(r.p_abs[ok], diff[ok], rtol=1e-10)
    # escaping power is the flux through the outer interface
    np.testing.assert_allclose(r.p_esc, dom * r2f[:, :, -1], rtol=1e-12)


def test_gray_equivalence():
    """Sect. 2.3 reduces to Eqs. 17-19 when kappa(nu) is one constant: the
    frequency-summed result equals the one-bin (gray) run."""
    w = synth.disk3d(32, 8, 3, n_nu=20, tau550=20.0, seed=4)
    g = w.grid
    kap = np.full(len(w.nu), 250.0)
    many = oracle.irradiate_workload(w, kappa=kap)
    one = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, w.t_star, w.r_star,
                           np.array([5e14]), np.array([250.0]), w.t_sub,
                           w.rho32().astype(np.float64), w.tdust32().astype(np.float64))
    m = one.p_abs > 1e-30 * one.p_abs.max()
    np.testing.assert_allclose(many.q_abs[m], one.q_abs[m], rtol=1e-12)
    np.testing.assert_allclose(many.a_rad, one.a_rad, rtol=1e-12, atol=0)


def test_scalings():
    """q and a scale with R*^2 at fixed T* (Eq. 17); doubling rho while halving
    kappa keeps every optical depth, so q is unchanged and a = q/(rho c) halves."""
    w = synth.disk3d(24, 6, 2, n_nu=10, tau550=5.0, seed=9)
    base = oracle.irradiate_workload(w)
    g = w.grid
    rho = w.rho32().astype(np.float64)
    td = w.tdust32().astype(np.float64)
    big = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, w.t_star, 2 * w.r_star, w.nu,
                           w.kappa, w.t_sub, rho, td)
    np.testing.assert_allclose(big.q_abs, 4 * base.q_abs, rtol=1e-14)
    np.testing.assert_allclose(big.a_rad, 4 * base.a_rad, rtol=1e-14)
    swap = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, w.t_star, w.r_star, w.nu,
                            0.5 * w.kappa, w.t_sub, 2 * rho, td)
    np.testing.assert_allclose(swap.q_abs, base.q_abs, rtol=1e-13)
    np.testing.assert_allclose(swap.a_rad, 0.5 * base.a_rad, rtol=1e-13)


def test_sublimated_cells_are_transparent():
    """Evaporated dust has no opacity: a cell above t_sub absorbs nothing, exerts
    no force, and attenuates nothing for the cells behind it."""
    w = synth.disk3d(24, 6, 2, n_nu=10, tau550=5.0, seed=11)
    g = w.grid
    rho = w.rho32().astype(np.float64)
    td = w.tdust32().astype(np.float64)
    hot = td > w.t_sub
    assert hot.any()
    r = oracle.irradiate_workload(w)
    rho0 = np.where(hot, 0.0, rho)
    cold = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, w.t_star, w.r_star, w.nu, w.kappa,
                            1e30, rho0, td)
    assert np.all(r.q_abs[hot] == 0) and np.all(r.a_rad[hot] == 0)
    np.testing.assert_allclose(r.q_abs[~hot], cold.q_abs[~hot], rtol=1e-14)
    np.testing.assert_allclose(r.a_rad[~hot], cold.a_rad[~hot], rtol=1e-14)


def test_layout_theta_phi_distinct():
    """Fields are [nphi][ntheta][nr]: a ray's solid angle follows its theta row.
    An equatorial ray and a polar ray of a uniform medium differ only by dOmega."""
    g = small_grid(5, 4, 3)
    nu = synth.nu_bins(4)
    rho = np.full(g.shape, 1e-24)
    td = np.full(g.shape, 50.0)
    # make only phi-slab 1, theta-row 2 opaque
    rho[1, 2, :] = 1e-16
    r = oracle.irradiate(g.r_if, g.theta_if, g.phi_if, T_STAR, R_STAR, nu,
                         synth.kappa_synth(nu), 1500.0, rho, td)
    dom = _pins.solid_angles(g.theta_if, g.phi_if)
    per_sr = r.p_abs.sum(axis=2) / dom
    others = np.delete(per_sr.ravel(), 1 * g.ntheta + 2)
    np.testing.assert_allclose(others, others[0], rtol=1e-12)
    assert per_sr[1, 2] > 10 * others[0]


# --------------------------------------------------------------------------
# the density generator against the paper's table (Sect. 3.1.1)
# --------------------------------------------------------------------------
def _golden_table():
    rows = []
    with open(os.path.join(GOLDEN, "disk_normalisation.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def test_density_total_mass_matches_paper():
    """Integrating rho0 f1 f2 over the 1-1000 AU sphere reproduces the printed
    total gas masses (two significant figures) at the printed rho0."""
    from scipy import integrate
    tab = _golden_table()
    for tau, rho0, mtot in tab:
        def integrand(th, r):
            rc, z = r * math.sin(th), r * math.cos(th)
            rho = synth.disk_density(np.array([max(rc, 1e-300)]), np.array([z]), rho0)[0]
            return rho * 2 * math.pi * r * r * math.sin(th)
        au = synth.AU_CM
        # integrate in log r for accuracy
        val, _ = integrate.dblquad(lambda th, u: integrand(th, math.exp(u)) * math.exp(u),
                                   math.log(au), math.log(1000 * au), 0.0, math.pi,
                                   epsrel=1e-6)
        m = val / synth.M_SUN_G
        assert round(m, -int(math.floor(math.log10(m))) + 1) == pytest.approx(mtot, rel=1e-9), (tau, m)


def test_density_normalisation_linear_in_tau():
    """The printed rho0 are proportional to tau550 (ratio 1000 for 100/0.1), as the
    midplane integral normalisation implies; and both rows imply the same 550 nm
    opacity."""
    tab = _golden_table()
    (t1, r1, _), (t2, r2, _) = tab
    assert r2 / r1 == pytest.approx(t2 / t1, rel=1e-9)
    k1 = t1 / (r1 * synth.R_D_AU * synth.AU_CM * math.log(1000.0))
    k2 = t2 / (r2 * synth.R_D_AU * synth.AU_CM * math.log(1000.0))
    assert k1 == pytest.approx(k2, rel=1e-9)
    assert synth.rho0_for_tau550(t2, k2) == pytest.approx(r2, rel=1e-12)


def test_generator_is_counter_based():
    """Any cell of a workload regenerates from (seed, stream, index) alone."""
    idx = np.arange(1000, dtype=np.uint64)
    a = synth.hash_u01(3, 1, idx)
    b = synth.hash_u01(3, 1, idx[::-1])[::-1]
    assert np.array_equal(a, b)
    assert 0.0 < a.min() and a.max() <= 1.0
    g = synth.hash_normal(1, 1, np.arange(200000, dtype=np.uint64))
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
