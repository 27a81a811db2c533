"""The synthetic input recipe as stated: frequency grid, dust temperatures, the
lognormal density perturbation, the counter-based normal deviates, and the ranges of
the uneven 96-grid batch."""
from __future__ import annotations

import math

import numpy as np
import pytest

import synth


def test_frequency_grid():
    nu = synth.nu_bins(79)
    assert nu[0] == pytest.approx(1e11, rel=1e-15) and nu[-1] == pytest.approx(1e16, rel=1e-14)
    ratios = nu[1:] / nu[:-1]
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-12)   # log-spaced, end points included


def test_normal_deviates():
    g = synth.hash_normal(5, 3, np.arange(2_000_000, dtype=np.uint64))
    assert abs(g.mean()) < 3e-3 and abs(g.std() - 1.0) < 3e-3
    assert abs(np.mean(g ** 3)) < 1e-2 and abs(np.mean(g ** 4) - 3.0) < 2e-2


def test_dust_temperatures_and_sublimated_fraction():
    """T_dust i.i.d. uniform on 20..1600 K: a fraction 100/1580 = 6.33 % above 1500 K."""
    g = synth.log_grid(256, 128, 16)
    t = synth.tdust_random(g, 20.0, 1600.0, seed=1)
    assert t.min() >= 20.0 and t.max() <= 1600.0
    assert np.mean(t > synth.T_SUB_K) == pytest.approx(100.0 / 1580.0, abs=1.5e-3)


def test_lognormal_perturbation():
    """rho = base exp(ln(1.2) g): the log ratio to the unperturbed field has mean 0 and
    standard deviation ln 1.2, and no correlation between neighbouring cells."""
    g = synth.log_grid(128, 64, 8)
    base = synth.density(g, 1.0, envelope=True)
    pert = synth.density(g, 1.0, envelope=True, perturb_sigma=math.log(1.2), seed=1)
    ok = base > 1e-90 * base.max()
    x = np.log(pert[ok] / base[ok])
    assert abs(x.mean()) < 2e-3 and x.std() == pytest.approx(math.log(1.2), rel=5e-3)
    lr = np.log(pert / base)
    c = np.corrcoef(lr[..., 1:].ravel(), lr[..., :-1].ravel())[0, 1]
    assert abs(c) < 5e-3


def test_batch_ranges():
    specs = synth.batch_specs(96, seed=3)
    assert len(specs) == 96
    assert all(64 <= s["nr"] <= 512 and 32 <= s["ntheta"] <= 256 for s in specs)
    assert {s["nphi"] for s in specs} <= {1, 64, 128} and {s["n_nu"] for s in specs} <= {32, 79, 128}
    assert all(0.1 <= s["tau550"] <= 100.0 for s in specs)
    assert len({s["seed"] for s in specs}) == 96
