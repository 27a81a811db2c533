"""Plant plausible slips in copies of the oracle (on the CPU) and check that the
pins in ``test_oracle_pins.py`` (tracer), ``test_temperature_cpu.py`` (Planck mean,
Eq. 16), ``test_fld_cpu.py`` (Rosseland mean) and ``test_tdep_cpu.py`` (kappa(nu, T)
tables) catch every one of them.

A pin set that lets a dropped term, a wrong sign, an off-by-one or a transposed
index through would not be pinning anything; this test makes that claim
checkable. The mutants are built from text edits of ``oracle/rt_oracle.c`` into
a temporary directory; the real oracle is never modified.
"""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

import oracle
from tests import test_fld_cpu as fld_pins
from tests import test_oracle_pins as pins
from tests import test_tdep_cpu as tdep_pins
from tests import test_temperature_cpu as temp_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rt_oracle.c")

# (name, original text, mutated text)
MUTANTS = [
    ("tau_inclusive", "const double att = exp(-tau);", "const double att = exp(-(tau + dtau));"),
    ("linearised_absorption", "P[k] += lum * att * (-expm1(-dtau));", "P[k] += lum * att * dtau;"),
    ("wrong_sign_expm1", "P[k] += lum * att * (-expm1(-dtau));", "P[k] += lum * att * expm1(dtau);"),
    ("outer_interface_dilution", "Fif[k] += f_bin[i] * (r2 / (r_if[k] * r_if[k])) * att;",
     "Fif[k] += f_bin[i] * (r2 / (r_if[k + 1] * r_if[k + 1])) * att;"),
    ("transposed_ray_index", "const int it = (int)(j % ntheta);\n        const int ip = (int)(j / ntheta);",
     "const int it = (int)(j / nphi);\n        const int ip = (int)(j % nphi);"),
    ("geometric_bin_edge", "double lo = (i == 0) ? 0.0 : 0.5 * (nu_mid[i - 1] + nu_mid[i]);",
     "double lo = (i == 0) ? 0.0 : sqrt(nu_mid[i - 1] * nu_mid[i]);"),
    ("finite_top_edge", "double hi = (i == n_nu - 1) ? INFINITY :", "double hi = (i == n_nu - 1) ? 2.0 * nu_mid[i] :"),
    ("strict_sublimation", "(t_ray[k] <= t_sub)", "(t_ray[k] < t_sub)"),
    ("force_without_phi", "A[k] += lum * att * kap * dr * rto_phi(dtau);", "A[k] += lum * att * kap * dr;"),
    ("half_volume", "(pow(r_if[k + 1], 3) - pow(r_if[k], 3)) / 3.0", "(pow(r_if[k + 1], 3) - pow(r_if[k], 3)) / 2.0"),
    ("bernoulli_sign", "-691.0 / 2730.0", "691.0 / 2730.0"),
    ("series_term_dropped", "3.0 * x * x / (dm * dm)", "0.0 * x * x / (dm * dm)"),
    ("escape_lost", "rto_add(&esc, lum * exp(-tau));", "rto_add(&esc, lum * exp(-tau) * 0.999);"),
    ("no_mask_on_force", "A[k] += lum * att * kap * dr * rto_phi(dtau);",
     "A[k] += lum * att * kappa[i] * dr * rto_phi(dtau);"),
    # Planck and Rosseland means (Eqs. 11, 16)
    ("planck_unweighted", "num += kappa[i] * f[i];\n        den += f[i];", "num += kappa[i];\n        den += 1.0;"),
    ("rosseland_arithmetic", "if (kappa[i] > 0.0) num += w / kappa[i];", "if (kappa[i] > 0.0) num += w * kappa[i];"),
    ("rosseland_planck_weight", "const double w = ea - eb + 4.0 * rto_planck_band(a, b);",
     "const double w = rto_planck_band(a, b);"),
    ("rosseland_boundary_sign", "const double w = ea - eb + 4.0 * rto_planck_band(a, b);",
     "const double w = eb - ea + 4.0 * rto_planck_band(a, b);"),
    ("rosseland_window_ignored", "else if (w > 0.0) opaque_gap = 1;", "else if (w > 0.0) opaque_gap = 0;"),
    # dust temperature (Eq. 16)
    ("temperature_without_er", "const double f = a_rad_const * tt * tt * tt * tt - er - ar / kp;",
     "const double f = a_rad_const * tt * tt * tt * tt - ar / kp;"),
    ("temperature_kappa_times", "- er - ar / kp;", "- er - ar * kp;"),
    ("temperature_no_clamp", "const double tk = tt < t_lo ? t_lo : (tt > t_hi ? t_hi : tt);",
     "const double tk = tt;"),
    # kappa(nu, T) tables: linear in T between grid points, held beyond the ends
    ("kappa_at_left_row", "return row[j] + (row[j + 1] - row[j]) * w;", "return row[j];"),
    ("kappa_at_weight_flipped", "const double w = (t - t_grid[j]) / (t_grid[j + 1] - t_grid[j]);",
     "const double w = (t_grid[j + 1] - t) / (t_grid[j + 1] - t_grid[j]);"),
    ("kappa_at_extrapolated_below", "if (n_t == 1 || t <= t_grid[0]) return row[0];", "if (n_t == 1) return row[0];"),
]

PIN_CALLS = [
    ("sigma", lambda: pins.test_sigma_is_a_c_over_4()),
    ("bins79", lambda: pins.test_planck_bins_against_quadrature(79)),
    ("bins5", lambda: pins.test_planck_bins_against_quadrature(5)),
    ("bins_hot", lambda: pins.test_planck_bins_other_temperatures(40000.0)),
    ("thin_rho0", lambda: pins.test_thin_limit("rho0")),
    ("thin_sub", lambda: pins.test_thin_limit("sublimated")),
    ("brute0", lambda: pins.test_brute_force_quadrature(0)),
    ("energy", lambda: pins.test_energy_conservation("disk3d_small")),
    ("fluxdiff", lambda: pins.test_flux_difference_form()),
    ("layout", lambda: pins.test_layout_theta_phi_distinct()),
    ("sublimated", lambda: pins.test_sublimated_cells_are_transparent()),
    ("planck_one_bin", lambda: temp_pins.test_planck_mean_of_one_bin_is_its_opacity()),
    ("planck_power_law", lambda: temp_pins.test_planck_mean_of_a_power_law(300.0)),
    ("t_radiation_only", lambda: temp_pins.test_radiation_only_closed_form()),
    ("t_eq16", lambda: temp_pins.test_solution_satisfies_eq16()),
    ("t_thin_sphere", lambda: temp_pins.test_gray_thin_sphere_equilibrium()),
    ("t_clamp", lambda: temp_pins.test_planck_mean_is_held_outside_the_table_range()),
    ("rosseland_power_law", lambda: fld_pins.test_rosseland_mean_of_a_power_law(300.0)),
    ("rosseland_window", lambda: fld_pins.test_rosseland_mean_of_a_transparent_window()),
    ("tdep_constant", lambda: tdep_pins.test_constant_table_is_the_plain_tracer()),
    ("tdep_row_below", lambda: tdep_pins.test_uniform_temperature_uses_the_interpolated_row(5.0)),
    ("tdep_row_inside", lambda: tdep_pins.test_uniform_temperature_uses_the_interpolated_row(97.0)),
    ("tdep_two_zone", lambda: tdep_pins.test_two_zone_gray_ray()),
]


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    return tmp_path_factory.mktemp("mutants")


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, orig, mut, mutant_dir):
    src = open(SRC).read()
    assert orig in src, f"mutation anchor for {name} not found in the oracle"
    cpath = os.path.join(mutant_dir, f"{name}.c")
    with open(cpath, "w") as fh:
        fh.write(src.replace(orig, mut, 1))
    so = os.path.join(mutant_dir, f"lib{name}.so")
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", cpath, "-o", so, "-lm"],
                   check=True, capture_output=True)
    caught = []
    with oracle.use_library(so):
        for pin_name, call in PIN_CALLS:
            try:
                call()
            except AssertionError:
                caught.append(pin_name)
    assert caught, f"mutant {name} passed every pin"
