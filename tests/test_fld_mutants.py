"""Plant plausible slips in copies of the flux-limited-diffusion reference
(``oracle/fld.py``, Sect. 2.1, Eqs. 7-15) on the CPU and check that the pins in
``test_fld_cpu.py`` catch every one of them: a dropped factor, a face quantity
taken at the cell centre, an arithmetic instead of a harmonic mean, a lost
periodic wrap, a one-sided difference.

Each mutant is a text edit of the module written to a temporary directory and
loaded as a sibling of ``oracle.fld``; the pins run with that module in place of
the real one. The real oracle is never modified. Every slip in the step itself
must fail a pin built on a closed form, a convergence rate or a conservation law,
not only the single-row check (which codes the same rows a second time).
"""
from __future__ import annotations

import importlib.util
import os

import pytest

from oracle import fld
from tests import test_fld_cpu as pins

SRC = fld.__file__

# (name, original text, mutated text)
MUTANTS = [
    # Eqs. 10-13: limiter and diffusion coefficient
    ("limiter_denominator", "return (2.0 + R) / (6.0 + 3.0 * R + R * R)", "return (2.0 + R) / (6.0 + 3.0 * R + R)"),
    ("d_cross_term", "den = 6.0 * s * s + 3.0 * s * g + g * g", "den = 6.0 * s * s + 2.0 * s * g + g * g"),
    ("d_without_c", "return np.where(num > 0.0, C * num / np.where(num > 0.0, den, 1.0), 0.0)",
     "return np.where(num > 0.0, num / np.where(num > 0.0, den, 1.0), 0.0)"),
    ("r_not_normalised_by_e", "g = gradient_norm(geo, e) / np.asarray(e, dtype=np.float64)",
     "g = gradient_norm(geo, e)"),
    # Eq. 9
    ("fc_dropped", "fc = 1.0 / (c_v * np.asarray(rho, dtype=np.float64) / (4.0 * a * t ** 3) + 1.0)",
     "fc = np.ones_like(t)"),
    ("fc_t4", "/ (4.0 * a * t ** 3) + 1.0)", "/ (4.0 * a * t ** 4) + 1.0)"),
    # gradients for R
    ("gradient_r_one_sided", "gr[..., 1:-1] = (e[..., 2:] - e[..., :-2]) / (rc[2:] - rc[:-2])",
     "gr[..., 1:-1] = (e[..., 2:] - e[..., 1:-1]) / (rc[2:] - rc[1:-1])"),
    ("gradient_theta_without_r", "gt[:, 1:-1, :] = (e[:, 2:, :] - e[:, :-2, :]) / (rr * (thc[2:] - thc[:-2])[None, :, None])",
     "gt[:, 1:-1, :] = (e[:, 2:, :] - e[:, :-2, :]) / ((thc[2:] - thc[:-2])[None, :, None])"),
    ("gradient_phi_without_sin", "scale = rc[None, None, :] * np.sin(thc)[None, :, None] * dphi[:, None, None]",
     "scale = rc[None, None, :] * dphi[:, None, None]"),
    # finite-volume geometry and faces
    ("half_volume", "d3 = (self.r_if[1:] ** 3 - self.r_if[:-1] ** 3) / 3.0",
     "d3 = (self.r_if[1:] ** 3 - self.r_if[:-1] ** 3) / 2.0"),
    ("arithmetic_face_mean", "df = np.where(pos, 2.0 * da * db / np.where(pos, da + db, 1.0), 0.0)",
     "df = np.where(pos, 0.5 * (da + db), 0.0)"),
    ("radial_area_at_centre", "area = geo.dom[:, :, None] * (geo.r_if[1:-1] ** 2)[None, None, :]",
     "area = geo.dom[:, :, None] * (geo.rc[:-1] ** 2)[None, None, :]"),
    ("radial_distance_cell_width", "dist = np.broadcast_to((geo.rc[1:] - geo.rc[:-1])[None, None, :], area.shape)",
     "dist = np.broadcast_to((geo.r_if[2:] - geo.r_if[1:-1])[None, None, :], area.shape)"),
    ("theta_area_at_centre", "np.sin(geo.th_if[1:-1])[None, :, None] * geo.dr2[None, None, :]",
     "np.sin(geo.thc[1:])[None, :, None] * geo.dr2[None, None, :]"),
    ("theta_distance_without_r", "dist = geo.rc[None, None, :] * (geo.thc[1:] - geo.thc[:-1])[None, :, None]",
     "dist = (geo.thc[1:] - geo.thc[:-1])[None, :, None] + 0.0 * geo.rc[None, None, :]"),
    ("phi_area_without_r", "area = np.broadcast_to(dth[None, :, None] * geo.dr2[None, None, :], shape)",
     "area = np.broadcast_to(dth[None, :, None] * np.diff(geo.r_if)[None, None, :], shape)"),
    ("phi_not_periodic", "faces(idx, np.roll(idx, -1, axis=0), d, np.roll(d, -1, axis=0), area, dist)",
     "faces(idx[:-1], idx[1:], d[:-1], d[1:], area[:-1], dist[:-1])"),
    ("one_sided_diagonal", "np.add.at(diag, cols, ws)\n", "\n"),
    ("off_diagonal_sign", "np.concatenate([diag, -ws, -ws])", "np.concatenate([diag, ws, ws])"),
    # storage, source and the outer boundary (Eqs. 8, 15)
    ("storage_times_fc", "diag = (geo.vol / (dt * fc)).ravel().copy()", "diag = (geo.vol * fc / dt).ravel().copy()"),
    ("source_without_volume", "+ (geo.vol * q).ravel() + bnd", "+ q.ravel() + bnd"),
    ("outer_boundary_full_cell", "w_out = d[..., -1] * geo.dom * geo.r_if[-1] ** 2 / (geo.r_if[-1] - geo.rc[-1])",
     "w_out = d[..., -1] * geo.dom * geo.r_if[-1] ** 2 / (geo.r_if[-1] - geo.r_if[-2])"),
    ("outer_boundary_without_a", "bnd[idx[..., -1].ravel()] = (w_out * a * t_bg ** 4).ravel()",
     "bnd[idx[..., -1].ravel()] = (w_out * t_bg ** 4).ravel()"),
    # the single-row check used at sizes the direct solve cannot reach
    ("row_radial_face_inner", "rf = geo.r_if[max(k, kk)]", "rf = geo.r_if[min(k, kk)]"),
    ("row_harmonic_dropped", "return 2.0 * x * y / (x + y) if x > 0.0 and y > 0.0 else 0.0",
     "return 0.5 * (x + y)"),
]

PIN_CALLS = [
    ("limits", lambda: pins.test_limiter_limits()),
    ("geometry", lambda: pins.test_geometry_tiles_the_shell()),
    ("stationary", lambda: pins.test_uniform_background_is_stationary()),
    ("balance", lambda: pins.test_discrete_energy_balance()),
    ("spherical", lambda: pins.test_spherical_steady_state_converges("uniform")),
    ("layered", lambda: pins.test_spherical_steady_state_converges("layered")),
    ("theta_modes", lambda: pins.test_angular_modes_decay_at_the_continuum_rate("theta")),
    ("phi_modes", lambda: pins.test_angular_modes_decay_at_the_continuum_rate("phi")),
    ("gradient", lambda: pins.test_gradient_of_a_quadratic_field_converges()),
    ("d_limits", lambda: pins.test_diffusion_coefficient_limits_per_cell()),
    ("energy_split", lambda: pins.test_injected_energy_splits_between_gas_and_radiation()),
    ("rows", lambda: pins.test_row_residuals_vanish_at_the_solution()),
]


def _load_mutant(path, name):
    spec = importlib.util.spec_from_file_location(f"oracle._fld_mutant_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_fld_pins_catch_mutant(name, orig, mut, tmp_path, monkeypatch):
    src = open(SRC).read()
    assert orig in src, f"mutation anchor for {name} not found in the reference"
    path = os.path.join(tmp_path, f"fld_{name}.py")
    with open(path, "w") as fh:
        fh.write(src.replace(orig, mut, 1))
    monkeypatch.setattr(pins, "fld", _load_mutant(path, name))
    caught = []
    for pin_name, call in PIN_CALLS:
        try:
            call()
        except AssertionError:
            caught.append(pin_name)
    assert caught, f"mutant {name} passed every pin"
    if not name.startswith("row_"):
        # a slip in the step itself must also fail a pin that does not rest on
        # row_residuals, the second coding of the same rows
        assert set(caught) - {"rows"}, f"mutant {name} is caught only by the row check"


def test_unmutated_copy_passes_every_pin(tmp_path, monkeypatch):
    """The loading route itself is sound: an unedited copy passes all pins."""
    path = os.path.join(tmp_path, "fld_copy.py")
    with open(path, "w") as fh:
        fh.write(open(SRC).read())
    monkeypatch.setattr(pins, "fld", _load_mutant(path, "copy"))
    for _, call in PIN_CALLS:
        call()
