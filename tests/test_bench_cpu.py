"""Host-side measurement logic of bench.py: the count of exponentials the tracer
cannot replace by its thin-ray series (the MUFU floor of the roofline), checked
against a brute-force count over warps, rays and bins on small grids."""
from __future__ import annotations

import numpy as np
import pytest

import bench
import synth


def _brute_warps(w, shape):
    """Per warp of R = 32 / G rays (G lanes of C cells per ray): its cells, the bins
    its thin series takes (kappa_i N_max <= THIN_X, N_max the largest ray total) and
    the end of its tier (kappa_i c_max <= THIN_X, c_max the largest column of one
    lane's C cells; used if it adds bins and a thin row exists or it adds >= 4)."""
    g = w.grid
    kap = sorted(w.kappa[w.kappa > 0])
    c = shape[1]
    rho = w.rho32().astype(np.float64).reshape(-1, g.nr)
    td = w.tdust32().reshape(-1, g.nr)
    dr = np.diff(g.r_if)
    col = lambda j, k: rho[j, k] * dr[k] if td[j, k] <= w.t_sub else 0.0
    out = []
    nrays = rho.shape[0]
    if shape[0] == 2:   # chunked: 4 rays of 8 lanes per warp, chunks of 8 c cells
        L = 8 * c
        for first in range(0, nrays, 4):
            slots = range(first, first + 4)          # ray slots past the last ray hold nothing
            for k0 in range(0, g.nr, L):
                def lane_start(j, l):
                    return sum(col(j, k) for k in range(min(k0 + l * c, g.nr))) if j < nrays else 0.0
                nmax = max(lane_start(j, 8) for j in slots)
                cmax = max(sum(col(j, k) for k in range(k0 + l * c, min(k0 + (l + 1) * c, g.nr))) if j < nrays else 0.0
                           for j in slots for l in range(8))
                n0min = min(lane_start(j, l) for j in slots for l in range(8))
                bt = sum(1 for kk in kap if kk * nmax <= bench.THIN_X)
                bc = sum(1 for kk in kap if kk * cmax <= bench.THIN_X)
                bt2 = bc if (bc > bt and (bt > 0 or bc >= 4)) else bt
                na = sum(1 for kk in kap if kk * n0min <= 127.0 * np.log(2.0))
                cells = sum(1 for j in slots if j < nrays for k in range(k0, min(k0 + L, g.nr)))
                out.append((cells, bt, bt2, na))
        return out
    if 32 * c < g.nr:   # two warps per ray, each 32 c of its cells
        for j in range(nrays):
            nmax = sum(col(j, k) for k in range(g.nr))
            for h in range(2):
                k0, k1 = 32 * c * h, min(32 * c * (h + 1), g.nr)
                cmax = max(sum(col(j, k) for k in range(a, min(a + c, k1))) for a in range(k0, k0 + 32 * c, c))
                bt = sum(1 for kk in kap if kk * nmax <= bench.THIN_X)
                bc = sum(1 for kk in kap if kk * cmax <= bench.THIN_X)
                bt2 = bc if (bc > bt and (bt > 0 or bc >= 4)) else bt
                out.append((k1 - k0, bt, bt2, len(kap)))
        return out
    lanes = 8 if 8 * c >= g.nr else (16 if 16 * c >= g.nr else 32)
    r = 32 // lanes
    for first in range(0, nrays, r):
        rays = range(first, min(first + r, nrays))
        nmax = max(sum(col(j, k) for k in range(g.nr)) for j in rays)
        cmax = max(sum(col(j, k) for k in range(l * c, min((l + 1) * c, g.nr)))
                   for j in rays for l in range(lanes))
        bt = sum(1 for kk in kap if kk * nmax <= bench.THIN_X)
        bc = sum(1 for kk in kap if kk * cmax <= bench.THIN_X)
        bt2 = bc if (bc > bt and (bt > 0 or bc >= 4)) else bt
        out.append((len(rays) * g.nr, bt, bt2, len(kap)))
    return out


def _brute(w, shape):
    """One exponential per (cell, bin) beyond the tier, one per (lane, bin) of the
    tier; every (cell, bin) for the tile kernel."""
    if shape[0] not in (1, 2):
        return w.grid.ncells * int(np.count_nonzero(w.kappa > 0))
    return sum(max(na - bt2, 0) * cells + 32 * (bt2 - bt) for cells, bt, bt2, na in _brute_warps(w, shape))


@pytest.mark.parametrize("tau,shape", [(10.0, (1, 8, 4, 6)), (100.0, (1, 4, 4, 8)), (1.0, (1, 16, 4, 3)),
                                       (1e3, (1, 2, 4, 8)), (10.0, (0, 8, 4, 6))])
def test_exact_exp_ops_matches_brute_force(tau, shape):
    w = synth.disk3d(40, 6, 5, n_nu=16, tau550=tau, seed=4)   # 30 rays: a partial last warp
    assert bench.exact_exp_ops(w, shape) == _brute(w, shape)


@pytest.mark.parametrize("tau", [1.0, 100.0])
def test_exact_exp_ops_two_warps_per_ray(tau):
    """Rays of 80 cells with 2 cells per lane: two warps share each ray."""
    w = synth.disk3d(80, 4, 3, n_nu=16, tau550=tau, seed=5)
    shape = (1, 2, 4, 8)
    assert bench.exact_exp_ops(w, shape) == _brute(w, shape)
    assert bench.series_fma_ops(w, shape) == _brute_fma(w, shape)


@pytest.mark.parametrize("tau,shape", [(10.0, (2, 8, 4, 6)), (1e3, (2, 4, 4, 8)), (1e5, (2, 2, 4, 8))])
def test_chunked_ops_match_brute_force(tau, shape):
    """The chunked kernel: 150-cell rays in chunks of 8 c cells (a ragged last chunk),
    30 rays (a partial last warp), thick enough for bins to underflow."""
    w = synth.disk3d(150, 6, 5, n_nu=16, tau550=tau, seed=6)
    assert bench.exact_exp_ops(w, shape) == _brute(w, shape)
    assert bench.series_fma_ops(w, shape) == _brute_fma(w, shape)


def test_exact_exp_ops_limits():
    """No dust column: the series takes every bin; a column far above 1/kappa_min:
    no bin is thin."""
    w = synth.disk3d(32, 4, 3, n_nu=12, tau550=1.0, seed=2)
    w0 = synth.Workload(w.name, w.grid, w.nu, w.kappa, np.zeros_like(w.rho), w.tdust, tau550=0.0)
    assert bench.exact_exp_ops(w0, (1, 8, 4, 6)) == 0
    big = synth.Workload(w.name, w.grid, w.nu, w.kappa, w.rho * 1e30, w.tdust, tau550=1e30)
    nbins = int(np.count_nonzero(w.kappa > 0))
    assert bench.exact_exp_ops(big, (1, 8, 4, 6)) == w.grid.ncells * nbins


def _brute_fma(w, shape):
    """Series FMAs per cell in every warp that sums some bin in the series, plus
    EXACT_FMA_PER_PAIR per (cell, bin) traced bin by bin."""
    if shape[0] not in (1, 2):
        return bench.EXACT_FMA_PER_PAIR * _brute(w, shape)
    return sum(bench.SERIES_FMA_PER_CELL * cells * (bt2 > 0) + bench.EXACT_FMA_PER_PAIR * max(na - bt2, 0) * cells
               for cells, bt, bt2, na in _brute_warps(w, shape))


@pytest.mark.parametrize("tau,shape", [(10.0, (1, 8, 4, 6)), (1e4, (1, 4, 4, 8)), (0.3, (0, 8, 4, 6))])
def test_series_fma_ops_matches_brute_force(tau, shape):
    w = synth.disk3d(40, 6, 5, n_nu=16, tau550=tau, seed=4)
    assert bench.series_fma_ops(w, shape) == _brute_fma(w, shape)


def _grid(launch_s, ex2, fma=0.0, nbytes=134217728):
    return {"bytes": nbytes, "ex2": ex2, "fma": fma, "cell_nu": 6.627e8, "launch_s": launch_s}


def test_roofline_summary_headline_and_floors():
    """The headline is HBM (16 B per cell over the launch time, against the measured
    copy bandwidth) whatever binds; the binding floor per grid is the largest of the
    HBM, MUFU and FP32 times, summed over the step against the summed launch time."""
    peaks = dict(hbm_peak_gbs=6678.0, ex2_peak_gops=1e4, ffma_peak_gops=4e4, ex2_basis="x", ffma_basis="y")
    # grid 1: 134 MB at 6678 GB/s = 20.1 us against 1e8 ex2 at 1e4 Gop/s = 10 us (HBM binds);
    # grid 2: 3e8 ex2 = 30 us (MUFU binds); grid 3: 1.2e9 FMA at 4e4 Gop/s = 30 us (FP32 binds)
    r = bench.roofline_summary([_grid(80e-6, 1e8), _grid(100e-6, 3e8), _grid(60e-6, 0.0, 1.2e9)], **peaks)
    t_h = 134217728 / 6678e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(3 * t_h / 240e-6)
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])
    assert r["binding_floor"]["per_grid"] == ["hbm", "mufu", "fp32"]
    assert r["binding_floor"]["frac"] == pytest.approx((t_h + 30e-6 + 30e-6) / 240e-6)
    assert r["mufu"]["frac"] == pytest.approx(4e8 / 1e13 / 240e-6)
    assert r["fp32"]["frac"] == pytest.approx(1.2e9 / 4e13 / 240e-6)
    assert r["one_ex2_per_cell_nu"]["frac"] == pytest.approx(3 * 6.627e8 / 240e-6 / 1e13)
    assert r["target_frac"] == bench.ROOFLINE_TARGET
    assert r["target_met"] == (r["binding_floor"]["frac"] >= bench.ROOFLINE_TARGET)


def test_series_fma_constants_match_the_library():
    """SERIES_FMA_PER_CELL is the paired Horner form's 2 K + 1 operations for the
    library's kThinTerms = K."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(bench.__file__), "paper_1001_3301_gb300", "csrc",
                            "rt_internal.cuh")).read()
    m = re.search(r"constexpr int kThinTerms = ([0-9]+);", src)
    assert m and 2 * int(m.group(1)) + 1 == bench.SERIES_FMA_PER_CELL


def test_workloads_and_reference_config():
    """The default step is the 512 x 256 x 512 grid at tau550 = 1 and 100 (seed 2);
    the reference arm names the same workload."""
    spec = bench.WORKLOADS["c3"]
    assert (spec["nr"], spec["ntheta"], spec["nphi"], spec["n_nu"]) == (512, 256, 512, 79)
    assert spec["taus"] == (1.0, 100.0) and spec["seed"] == 2
    name = bench.workload_name(spec, spec["taus"])
    assert "512x256x512" in name and "tau550 in {1,100}" in name


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
