"""The flux-limited-diffusion step (Sect. 2.1, Eqs. 7-15) and the Rosseland mean on
the GPU against the FP64 oracle: every cell of small grids against the direct
sparse solve, and at the full 256x128x256 size sampled rows of the implicit
system plus the global energy balance of the step."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import fld
import synth

pytestmark = pytest.mark.gpu

# Per-cell tolerance against the FP64 direct solve. The FP32 coefficients (about
# ten rounded operations each, ~1e-6 relative) and the cubic ln T interpolation of
# ln kappa_R (< 1e-6) move the solution by ~1e-8 (the step is well conditioned in
# its coefficients); the refinement stops once a pass changes no cell by more than
# TOL, after which the error is about TOL times the inner solver's reduction.
# The bound is TOL with a factor 3 for the FP32 rounding of E' itself.
RTOL_E = 3e-5
TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _tracer(g, nu, kappa, t_grid=None):
    from paper_1001_3301_gb300 import Tracer
    tr = Tracer.from_grid(g)
    if t_grid is None:
        tr.set_opacity_table(nu, kappa, synth.T_SUB_K)
    else:
        tr.set_opacity_table_t(nu, t_grid, kappa, synth.T_SUB_K)
    tr.set_star(synth.T_STAR_K, synth.R_STAR_CM)
    return tr


def _cuda(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("t", [1.0, 10.0, 150.0, 1500.0, 3e4, 1e5])
def test_rosseland_mean_matches_oracle(torch, t):
    w = synth.disk2d(16, 8, 79)
    tr = _tracer(w.grid, w.nu, w.kappa)
    got = tr.rosseland_mean_opacity(t)
    ref = oracle.rosseland_mean(t, w.nu, w.kappa)
    assert abs(got / ref - 1) < 1e-12, (got, ref)
    tr.close()


def _kappa_rows_at(kt, tg, t):
    """kappa_i(T): linear in T between the table's temperatures, the end values beyond."""
    return np.array([np.interp(t, tg, row) for row in kt])


@pytest.mark.parametrize("t", [5.0, 40.0, 149.0, 151.0, 900.0, 3000.0])
def test_rosseland_mean_of_a_temperature_table(torch, t):
    g = synth.log_grid(8, 4, 1)
    nu = synth.nu_bins(32)
    tg = synth.t_grid(24)
    kt = synth.kappa_synth_t(nu, tg)
    tr = _tracer(g, nu, kt, tg)
    got = tr.rosseland_mean_opacity(t)
    ref = oracle.rosseland_mean(t, nu, _kappa_rows_at(kt, tg, t))
    assert abs(got / ref - 1) < 1e-12, (got, ref)
    tr.close()


def _step_pair(torch, g, nu, kappa, rho, t, q, e0, dt, c_v, t_bg, t_grid=None):
    """(GPU E', oracle E', GPU stats) on the same FP32-rounded inputs."""
    rho, t, q, e0 = (np.asarray(a, dtype=np.float32) for a in (rho, t, q, e0))
    tr = _tracer(g, nu, kappa, t_grid)
    e1, st = tr.fld_step(_cuda(torch, rho), _cuda(torch, t), _cuda(torch, q), _cuda(torch, e0), dt, c_v, t_bg,
                         tol=TOL, max_iter=5000)
    got = e1.double().cpu().numpy()
    tr.close()
    if t_grid is None:
        kr_of_t = lambda tt: oracle.rosseland_mean(tt, nu, kappa)
    else:
        kr_of_t = lambda tt: oracle.rosseland_mean(tt, nu, _kappa_rows_at(kappa, t_grid, tt))
    t64 = t.astype(np.float64)
    uniq, inv = np.unique(t64, return_inverse=True)
    kr = np.array([kr_of_t(float(x)) for x in uniq])[inv].reshape(t.shape)
    ref = fld.fld_step(g.r_if, g.theta_if, g.phi_if, rho, t64, q, e0, dt, c_v, t_bg, nu, kappa, kappa_r=kr)
    return got, ref, st


CASES = [
    # (nr, ntheta, nphi), dt (s): storage-dominated, mixed, steady state; grids above
    # 512 cells take the multigrid-preconditioned path, smaller ones Jacobi
    ((20, 12, 8), 1e4),     # the paper's FLD time step
    ((20, 12, 8), 1e6),
    ((20, 12, 8), 1e10),
    ((20, 12, 8), 1e300),
    ((37, 9, 5), 3e9),      # ragged sizes
    ((33, 7, 1), 1e10),     # axisymmetric
    ((16, 6, 2), 1e10),     # two phi cells: both faces between the same pair
    ((24, 1, 1), 1e10),     # one theta cell: radial only
    ((40, 24, 16), 1e4),    # three multigrid levels, four-cell kernels
    ((41, 23, 9), 1e4),     # three multigrid levels, odd sizes (one-cell aggregates at the ends)
    ((48, 24, 1), 1e4),     # multigrid on an axisymmetric grid (no phi aggregation)
    ((3000, 1, 1), 1e4),    # multigrid along r only (four levels)
]


@pytest.mark.parametrize("shape,dt", CASES)
def test_fld_step_matches_oracle(torch, shape, dt):
    nr, nth, nph = shape
    w = synth.disk3d(nr, nth, nph, n_nu=32, tau550=10.0, seed=5)
    t, e0, q = synth.fld_fields(w.grid, seed=2)
    got, ref, st = _step_pair(torch, w.grid, w.nu, w.kappa, w.rho, t, q, e0, dt, 1e8, 15.0)
    rel = np.abs(got / ref - 1)
    assert st["rel_change"] < TOL
    assert (st["levels"] > 1) == (nr * nth * nph > 512)
    assert rel.max() < RTOL_E, (rel.max(), st)


def test_fld_step_with_the_tracer_source(torch):
    """The irradiation's q_abs (oracle tracer, Eq. 15) as the source of one step."""
    w = synth.disk3d(24, 10, 4, n_nu=32, tau550=1.0, seed=9)
    res = oracle.irradiate_workload(w)
    t, e0, _ = synth.fld_fields(w.grid, seed=3)
    got, ref, st = _step_pair(torch, w.grid, w.nu, w.kappa, w.rho, t, res.q_abs, e0, 3e9, 1e8, 10.0)
    assert np.abs(got / ref - 1).max() < RTOL_E


def test_fld_step_with_a_temperature_table(torch):
    g = synth.log_grid(20, 8, 4)
    nu = synth.nu_bins(32)
    tg = synth.t_grid(24)
    kt = synth.kappa_synth_t(nu, tg)
    rho = synth.density(g, 10.0, envelope=True)
    t, e0, q = synth.fld_fields(g, seed=4)
    got, ref, st = _step_pair(torch, g, nu, kt, rho, t, q, e0, 1e10, 1e8, 15.0, t_grid=tg)
    # ln kappa_R(T) has kinks at the table's temperatures, which the cubic
    # interpolation of the tabulated mean smooths over one node spacing
    assert np.abs(got / ref - 1).max() < 1e-3


def test_uniform_background_is_stationary(torch):
    w = synth.disk3d(16, 8, 4, n_nu=32, tau550=10.0, seed=1)
    t_bg = 20.0
    t = np.full(w.grid.shape, t_bg)
    e0 = np.full(w.grid.shape, fld.radiation_constant() * t_bg ** 4)
    tr = _tracer(w.grid, w.nu, w.kappa)
    e1, st = tr.fld_step(_cuda(torch, w.rho), _cuda(torch, t), _cuda(torch, np.zeros(w.grid.shape)),
                         _cuda(torch, e0), 1e9, 1e8, t_bg, tol=TOL)
    assert np.abs(e1.double().cpu().numpy() / e0.astype(np.float32) - 1).max() < 1e-5
    tr.close()


def test_invalid_input_and_iteration_limit(torch):
    from paper_1001_3301_gb300 import RtError
    w = synth.disk3d(12, 6, 2, n_nu=16, tau550=1.0, seed=1)
    t, e0, q = synth.fld_fields(w.grid)
    tr = _tracer(w.grid, w.nu, w.kappa)
    r_, q_, e_ = _cuda(torch, w.rho), _cuda(torch, q), _cuda(torch, e0)
    bad_t = t.copy()
    bad_t[1, 2, 3] = 0.0
    with pytest.raises(RtError, match="NONFINITE"):
        tr.fld_step(r_, _cuda(torch, bad_t), q_, e_, 1e9, 1e8, 10.0)
    with pytest.raises(RtError, match="TIMEOUT"):
        tr.fld_step(r_, _cuda(torch, t), q_, e_, 1e12, 1e8, 10.0, tol=1e-30, max_iter=3)
    with pytest.raises(RtError, match="INVALID"):
        tr.fld_step(r_, _cuda(torch, t), q_, e_, -1.0, 1e8, 10.0)
    # the context stays usable
    _, st = tr.fld_step(r_, _cuda(torch, t), q_, e_, 1e9, 1e8, 10.0, tol=1e-6)
    assert st["rel_change"] < 1e-6
    tr.close()


def test_full_size_rows_and_energy_balance(torch):
    """256x128x256 (8.4M cells): 96 sampled rows of the implicit system rebuilt by
    the oracle in FP64, and the global balance sum V (E' - E)/(dt f_c) =
    sum V q - sum_outer w_out (E' - a T_bg^4), in which every interior face cancels."""
    w = synth.disk3d(256, 128, 256, n_nu=79, tau550=1.0, seed=1)
    g = w.grid
    t, e0, q = synth.fld_fields(g, seed=1)
    rho32, t32, q32, e32 = (a.astype(np.float32) for a in (w.rho, t, q, e0))
    dt, c_v, t_bg = 1e10, 1e8, 15.0
    tr = _tracer(g, w.nu, w.kappa)
    e1, st = tr.fld_step(_cuda(torch, rho32), _cuda(torch, t32), _cuda(torch, q32), _cuda(torch, e32), dt, c_v,
                         t_bg, tol=TOL, max_iter=20000)
    got = e1.double().cpu().numpy()
    tr.close()
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    cache = {}

    def kr_of_t(tt):
        if tt not in cache:
            cache[tt] = oracle.rosseland_mean(tt, w.nu, w.kappa)
        return cache[tt]

    rng = np.random.default_rng(11)
    cells = [(int(rng.integers(g.nphi)), int(rng.integers(g.ntheta)), int(rng.integers(g.nr))) for _ in range(80)]
    cells += [(0, 0, 0), (g.nphi - 1, g.ntheta - 1, g.nr - 1), (0, 64, g.nr - 1), (5, 0, 100), (7, 127, 3)]
    f64 = [a.astype(np.float64) for a in (rho32, t32, q32, e32)]
    res = fld.row_residuals(g.r_if, g.theta_if, g.phi_if, *f64, got, dt, c_v, t_bg, kr_of_t, cells)
    assert res.max() < 1e-4, res.max()
    # global balance
    geo = fld.Geometry(g.r_if, g.theta_if, g.phi_if)
    a = fld.radiation_constant()
    rho, tt, qq, ee = f64
    fc = 1.0 / (c_v * rho / (4.0 * a * tt ** 3) + 1.0)
    store = geo.vol * (got - ee) / (dt * fc)
    d_out = np.empty((g.nphi, g.ntheta))
    for l in range(g.nphi):
        for j in range(g.ntheta):
            s = kr_of_t(float(tt[l, j, -1])) * rho[l, j, -1]
            gn = fld._grad_at(geo, ee, l, j, g.nr - 1) / ee[l, j, -1]
            d_out[l, j] = fld.diffusion_coefficient(s, gn)
    w_out = d_out * geo.dom * g.r_if[-1] ** 2 / (g.r_if[-1] - geo.rc[-1])
    lhs = store.sum()
    flux_out = w_out * (got[..., -1] - a * t_bg ** 4)
    rhs = (geo.vol * qq).sum() - flux_out.sum()
    # what per-cell relative errors of RTOL_E in E' can move each term by
    scale = ((geo.vol * (np.abs(got) + ee) / (dt * fc)).sum() + (geo.vol * qq).sum() +
             (w_out * (np.abs(got[..., -1]) + a * t_bg ** 4)).sum())
    assert abs(lhs - rhs) < RTOL_E * scale, (lhs, rhs, scale)
