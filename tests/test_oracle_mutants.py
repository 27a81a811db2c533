"""Plant plausible slips in copies of the oracle (on the CPU) and check that the
pins in ``test_oracle_pins.py`` catch every one of them.

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
from tests import test_oracle_pins as pins

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
