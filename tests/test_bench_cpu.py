"""Host-side measurement logic of bench.py: the count of exponentials the tracer
cannot replace by its thin-ray series (the MUFU floor of the roofline), checked
against a brute-force count over warps, rays and bins on small grids."""
from __future__ import annotations

import numpy as np
import pytest

import bench
import synth


def _brute(w, shape):
    """Per warp of R = 32 / G rays: bins with kappa_i N_max > THIN_X, times the
    warp's rays' cells; every (cell, bin) for the tile kernel."""
    g = w.grid
    kap = w.kappa[w.kappa > 0]
    if shape[0] != 1:
        return g.ncells * len(kap)
    c = shape[1]
    lanes = 8 if 8 * c >= g.nr else (16 if 16 * c >= g.nr else 32)
    r = 32 // lanes
    rho = w.rho32().astype(np.float64).reshape(-1, g.nr)
    td = w.tdust32().reshape(-1, g.nr)
    dr = np.diff(g.r_if)
    total = 0
    nrays = rho.shape[0]
    for first in range(0, nrays, r):
        rays = range(first, min(first + r, nrays))
        nmax = max(sum(rho[j, k] * dr[k] for k in range(g.nr) if td[j, k] <= w.t_sub) for j in rays)
        exact = sum(1 for kk in kap if kk * nmax > bench.THIN_X)
        total += exact * len(rays) * g.nr
    return total


@pytest.mark.parametrize("tau,shape", [(10.0, (1, 8, 4, 6)), (100.0, (1, 4, 4, 8)), (1.0, (1, 16, 4, 3)),
                                       (10.0, (0, 8, 4, 6))])
def test_exact_exp_ops_matches_brute_force(tau, shape):
    w = synth.disk3d(40, 6, 5, n_nu=16, tau550=tau, seed=4)   # 30 rays: a partial last warp
    assert bench.exact_exp_ops(w, shape) == _brute(w, shape)


def test_exact_exp_ops_limits():
    """No dust column: the series takes every bin; a column far above 1/kappa_min:
    no bin is thin."""
    w = synth.disk3d(32, 4, 3, n_nu=12, tau550=1.0, seed=2)
    w0 = synth.Workload(w.name, w.grid, w.nu, w.kappa, np.zeros_like(w.rho), w.tdust, tau550=0.0)
    assert bench.exact_exp_ops(w0, (1, 8, 4, 6)) == 0
    big = synth.Workload(w.name, w.grid, w.nu, w.kappa, w.rho * 1e30, w.tdust, tau550=1e30)
    nbins = int(np.count_nonzero(w.kappa > 0))
    assert bench.exact_exp_ops(big, (1, 8, 4, 6)) == w.grid.ncells * nbins


def test_roofline_summary_picks_the_binding_floor():
    """HBM binds when its time per launch is the larger one, MUFU otherwise; frac is the
    binding floor's time over the launch time, and the two other bases ride along."""
    # 134 MB at 6678 GB/s = 20.1 us against 1e8 ex2 at 1e4 Gop/s = 10 us: HBM binds
    r = bench.roofline_summary(bytes_per_launch=134217728, exact_ops=1e8, cell_nu_per_launch=6.627e8,
                               avg_launch_s=80e-6, hbm_peak_gbs=6678.0, ex2_peak_gops=1e4, ex2_basis="x")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(134217728 / 6678e9 / 80e-6)
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])
    assert r["mufu"]["frac"] == pytest.approx(1e8 / 1e13 / 80e-6)
    assert r["one_ex2_per_cell_nu"]["frac"] == pytest.approx(6.627e8 / 80e-6 / 1e13)
    # three times the exponentials: MUFU binds
    r = bench.roofline_summary(bytes_per_launch=134217728, exact_ops=3e8, cell_nu_per_launch=6.627e8,
                               avg_launch_s=80e-6, hbm_peak_gbs=6678.0, ex2_peak_gops=1e4, ex2_basis="x")
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(3e8 / 1e13 / 80e-6)
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])


def test_thin_bound_matches_the_library():
    """bench.THIN_X mirrors the tracer's kThinX (rt_internal.cuh): the count of
    exponentials above is only right while the two agree."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(bench.__file__), "paper_1001_3301_gb300", "csrc",
                            "rt_internal.cuh")).read()
    m = re.search(r"constexpr float kThinX = ([0-9.eE+-]+)f;", src)
    assert m and float(m.group(1)) == bench.THIN_X


def test_cpu_baseline_samples_every_grid_of_the_step():
    ws = [synth.disk3d(32, 8, 4, n_nu=16, tau550=t, seed=1) for t in (0.1, 100.0)]
    r = bench.cpu_baseline(ws, target_s=0.05)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1
    assert "tau550=0.1" in r["sample"] and "tau550=100" in r["sample"]
