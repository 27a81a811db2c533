"""Pins of the oracle with temperature-dependent opacity tables (kappa_i linear in
T between grid points; the scan of Eq. 19 with every cell's own kappa)."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth


def _grid_fields(nr=20, nth=4, nph=3, seed=2):
    w = synth.disk3d(nr, nth, nph, n_nu=16, tau550=10.0, seed=seed)
    return w, w.rho32().astype(np.float64), w.tdust32().astype(np.float64)


def _run_tdep(w, tg, kt, rho, td):
    g = w.grid
    return oracle.irradiate_tdep(g.r_if, g.theta_if, g.phi_if, w.t_star, w.r_star, w.nu, tg, kt, w.t_sub, rho, td)


def test_constant_table_is_the_plain_tracer():
    """A table constant in T reproduces the temperature-independent oracle exactly."""
    w, rho, td = _grid_fields()
    tg = synth.t_grid(8)
    kt = np.repeat(w.kappa[:, None], len(tg), axis=1)
    a = _run_tdep(w, tg, kt, rho, td)
    b = oracle.irradiate_workload(w)
    assert np.array_equal(a.q_abs, b.q_abs) and np.array_equal(a.a_rad, b.a_rad)
    assert a.e_abs == b.e_abs and a.e_esc == b.e_esc


@pytest.mark.parametrize("t_u", [5.0, 10.0, 97.0, 150.0, 1499.0])
def test_uniform_temperature_uses_the_interpolated_row(t_u):
    """With one dust temperature everywhere every cell's kappa is the table at t_u:
    linear between the bracketing points (the ends beyond the grid)."""
    w, rho, _ = _grid_fields()
    tg = synth.t_grid(12)
    kt = synth.kappa_synth_t(w.nu, tg)
    td = np.full(w.grid.shape, t_u)
    a = _run_tdep(w, tg, kt, rho, td)
    if t_u <= tg[0]:
        k_u = kt[:, 0]
    else:
        j = int(np.searchsorted(tg, t_u, side="right") - 1)
        wgt = (t_u - tg[j]) / (tg[j + 1] - tg[j])
        k_u = kt[:, j] + (kt[:, j + 1] - kt[:, j]) * wgt
    b = oracle.irradiate_workload(w, rho=rho, tdust=td, kappa=k_u)
    np.testing.assert_allclose(a.q_abs, b.q_abs, rtol=1e-14, atol=0)
    np.testing.assert_allclose(a.a_rad, b.a_rad, rtol=1e-14, atol=0)


def test_two_zone_gray_ray():
    """One gray bin, dust at T_a in the inner cells and T_b in the outer ones: the
    optical depth in front of cell k sums each cell's own kappa (Eq. 19), and the
    absorbed power of cell k is L dOmega/(4 pi) (e^{-tau_-} - e^{-tau_+})."""
    g = synth.log_grid(10, 1, 1)
    tg = np.array([100.0, 200.0])
    kt = np.array([[2.0, 0.5]])          # kappa(100 K) = 2, kappa(200 K) = 0.5
    rho = np.full(g.shape, 3e-14)
    td = np.where(np.arange(10) < 4, 100.0, 200.0)[None, None, :]
    res = oracle.irradiate_tdep(g.r_if, g.theta_if, g.phi_if, 5800.0, synth.R_STAR_CM, [5e14], tg, kt, 1500.0,
                                rho, td)
    dtau = np.where(np.arange(10) < 4, 2.0, 0.5) * 3e-14 * np.diff(g.r_if)
    tau = np.concatenate([[0.0], np.cumsum(dtau)])
    lum = 4 * math.pi * synth.R_STAR_CM ** 2 * oracle.sigma_sb() * 5800.0 ** 4
    p = lum * (np.exp(-tau[:-1]) - np.exp(-tau[1:]))
    np.testing.assert_allclose(res.p_abs[0, 0], p, rtol=1e-12)


def test_energy_is_conserved():
    w, rho, td = _grid_fields(nr=32, seed=6)
    tg = synth.t_grid(24)
    res = _run_tdep(w, tg, synth.kappa_synth_t(w.nu, tg), rho, td)
    assert abs(res.rel_err) < 1e-12
