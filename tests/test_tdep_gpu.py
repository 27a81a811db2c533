"""The tracer with temperature-dependent opacity tables against the FP64 oracle: a
table that separates, kappa_i(T) = kappa_i b(T) (the one-column tracer with each
cell's column weighted by b(T)), two-, three- and four-species tables of rank two to
four (that many columns per ray) and a full-rank table (per-bin scans of Eq. 19 with
every cell's own kappa)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import _parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _oracle(w, tg, kt):
    g = w.grid
    return oracle.irradiate_tdep(g.r_if, g.theta_if, g.phi_if, w.t_star, w.r_star, w.nu, tg, kt, w.t_sub,
                                 w.rho32().astype(np.float64), w.tdust32().astype(np.float64), nthreads=8)


def _run(w, tg, kt, shape=None, precision="fp32_kahan", kind=None):
    import torch
    from paper_1001_3301_gb300 import Tracer
    tr = Tracer.from_grid(w.grid, precision)
    tr.set_opacity_table_t(w.nu, tg, kt, w.t_sub)
    tr.set_star(w.t_star, w.r_star)
    if kind is not None:
        assert tr.table_kind() == kind
    if shape is not None:
        tr.set_tuning(*shape)
    r = torch.from_numpy(w.rho32()).cuda()
    t = torch.from_numpy(w.tdust32()).cuda()
    q, a, e = tr.irradiate(r, t, energy=True)
    out = q.double().cpu().numpy(), a.double().cpu().numpy(), e, tr.tunings()
    tr.close()
    return out


TABLES = {"separable": synth.kappa_synth_t, "two-species": synth.kappa_synth_t2,
          "three-species": synth.kappa_synth_t3, "four-species": synth.kappa_synth_t4,
          "full-rank": synth.kappa_synth_t_full}


def _tg(n):
    """The synthetic temperature grid as float32 values: the form the device holds
    (like the float32 fields, both sides see the same points)."""
    return synth.t_grid(n).astype(np.float32).astype(np.float64)


def _separates(kt):
    """kappa_i(T_j) = kmax_i b_j to 1e-12 of every entry, b the row of the largest kmax."""
    kmax = kt.max(axis=1)
    iref = int(np.argmax(kmax))
    if kmax[iref] == 0.0:
        return True
    want = np.outer(kmax, kt[iref] / kmax[iref])
    return bool(np.all(np.abs(kt - want) <= 1e-12 * np.maximum(np.abs(kt), np.abs(want))))


def _rank_two(kt):
    """Every column a non-negative combination of the two columns of extreme angle in
    the plane of the columns, to 1e-10 of every entry."""
    n = np.linalg.norm(kt, axis=0)
    j1 = int(np.argmax(n))
    if n[j1] == 0.0:
        return False
    u = kt[:, j1] / n[j1]
    pu = u @ kt
    r = kt - np.outer(u, pu)
    rn = np.linalg.norm(r, axis=0)
    j2 = int(np.argmax(rn))
    if not rn[j2] > 1e-12 * n[j1]:
        return False
    pv = (r[:, j2] / rn[j2]) @ kt
    th = np.where(n > 0, np.arctan2(pv, pu), np.nan)
    lo, hi = int(np.nanargmin(th)), int(np.nanargmax(th))
    det = pu[lo] * pv[hi] - pu[hi] * pv[lo]
    if lo == hi or det == 0.0:
        return False
    x = np.maximum((pu * pv[hi] - pu[hi] * pv) / det, 0.0)
    y = np.maximum((pu[lo] * pv - pu * pv[lo]) / det, 0.0)
    want = np.outer(kt[:, lo], x) + np.outer(kt[:, hi], y)
    return bool(np.all(np.abs(kt - want) <= 1e-10 * np.maximum(np.abs(kt), np.abs(want))))


def _low_rank(kt, r):
    """The leading r right singular vectors reproduce every entry to 1e-10 of its row's
    largest value."""
    if r > kt.shape[1]:
        return False
    vr = np.linalg.svd(kt, full_matrices=False)[2][:r].T
    want = (kt @ vr) @ vr.T
    rowmax = np.abs(kt).max(axis=1, keepdims=True)
    return bool(np.all(np.abs(kt - want) <= 1e-10 * rowmax))


def _kind(kt, nr, precision="fp32_kahan"):
    """The path the library takes: the one-column tracer with the column weight where
    the table separates and the rays fit its shapes, else the two-column kernel where
    the table is of rank two with non-negative factors, else the three- or four-column
    kernel where it is of rank three or four, else the per-bin scans (FP32 arithmetic
    in every path)."""
    from paper_1001_3301_gb300._lib import (RT_TABLE_NU_T, RT_TABLE_NU_T_LOW_RANK, RT_TABLE_NU_T_RANK2,
                                            RT_TABLE_NU_T_SEPARABLE)
    if precision == "fp64":
        return RT_TABLE_NU_T
    if _separates(kt):
        return RT_TABLE_NU_T_SEPARABLE if nr <= 512 else RT_TABLE_NU_T
    if _rank_two(kt):
        return RT_TABLE_NU_T_RANK2
    return RT_TABLE_NU_T_LOW_RANK if (_low_rank(kt, 3) or _low_rank(kt, 4)) else RT_TABLE_NU_T


def test_synthetic_tables_take_their_kernels():
    """The synthetic tables on the bench's 79 bins: one per path."""
    from paper_1001_3301_gb300._lib import (RT_TABLE_NU_T, RT_TABLE_NU_T_LOW_RANK, RT_TABLE_NU_T_RANK2,
                                            RT_TABLE_NU_T_SEPARABLE)
    nu = synth.disk3d(8, 2, 2, n_nu=79, tau550=1.0, seed=1).nu
    tg = _tg(24)
    assert _kind(synth.kappa_synth_t(nu, tg), 256) == RT_TABLE_NU_T_SEPARABLE
    assert _kind(synth.kappa_synth_t2(nu, tg), 256) == RT_TABLE_NU_T_RANK2
    assert _kind(synth.kappa_synth_t3(nu, tg), 256) == RT_TABLE_NU_T_LOW_RANK
    assert _kind(synth.kappa_synth_t4(nu, tg), 256) == RT_TABLE_NU_T_LOW_RANK
    assert _kind(synth.kappa_synth_t_full(nu, tg), 256) == RT_TABLE_NU_T


@pytest.mark.parametrize("table", sorted(TABLES))
@pytest.mark.parametrize("tau", [0.1, 1.0, 100.0])
def test_disk_against_oracle(torch, tau, table):
    w = synth.disk3d(96, 24, 8, n_nu=79, tau550=tau, seed=11)
    tg = _tg(24)
    kt = TABLES[table](w.nu, tg)
    orc = _oracle(w, tg, kt)
    q, a, e, _ = _run(w, tg, kt, kind=_kind(kt, w.grid.nr))
    _parity.assert_parity(w, q, a, e, orc, label=f"tdep {table} tau {tau}")


@pytest.mark.parametrize("table", sorted(TABLES))
@pytest.mark.parametrize("dims", [(1, 1, 1, 1), (7, 3, 2, 5), (33, 5, 3, 17), (65, 4, 2, 40), (200, 3, 2, 79),
                                  (300, 3, 2, 24), (513, 2, 2, 32), (1024, 2, 1, 16)],
                         ids=lambda d: "x".join(map(str, d)))
def test_ragged_all_shapes(torch, dims, table):
    nr, nth, nph, nnu = dims
    w = synth.disk3d(nr, nth, nph, n_nu=nnu, tau550=10.0, seed=nr + nth)
    tg = _tg(9)
    kt = TABLES[table](w.nu, tg)
    orc = _oracle(w, tg, kt)
    _, _, _, shapes = _run(w, tg, kt, kind=_kind(kt, nr))
    assert shapes and all(s[0] == 1 for s in shapes)
    for shape in shapes:
        q, a, e, _ = _run(w, tg, kt, shape=shape)
        _parity.assert_parity(w, q, a, e, orc, label=f"tdep {table} {dims} {shape}")


def test_separable_weight_edges(torch):
    """A separable table whose temperature factor is zero above 1000 K (dust that
    stays but stops absorbing: the column weight 0, the force 0) and temperatures
    beyond both ends of its grid (the end values hold); every precision mode, the
    FP64 one through the per-bin kernel."""
    w = synth.disk3d(128, 12, 4, n_nu=32, tau550=30.0, seed=9)
    tg = np.array([40.0, 100.0, 300.0, 600.0, 1000.0, 1200.0])
    b = np.array([0.6, 1.0, 0.8, 0.5, 0.0, 0.0])
    kt = np.outer(w.kappa, b)
    td = w.tdust32().copy()
    td.reshape(-1)[::7] = 15.0                    # below the grid
    orc = oracle.irradiate_tdep(w.grid.r_if, w.grid.theta_if, w.grid.phi_if, w.t_star, w.r_star, w.nu, tg, kt,
                                w.t_sub, w.rho32().astype(np.float64), td.astype(np.float64), nthreads=8)
    ww = synth.Workload(w.name, w.grid, w.nu, w.kappa, w.rho, td, tau550=w.tau550)
    # (an FP64 context takes the per-bin kernel, whose arithmetic is FP32: the same 1e-5)
    for precision, rtol in (("fp32_kahan", 1e-5), ("fp32_plain", 1e-5), ("fp64", 1e-5)):
        q, a, e, _ = _run(ww, tg, kt, precision=precision, kind=_kind(kt, 128, precision))
        _parity.assert_parity(ww, q, a, e, orc, rtol_q=rtol, rtol_a=rtol, label=f"edges {precision}")
        hot = (td > 1000.0) & (td <= w.t_sub)
        assert hot.any() and np.all(q[hot] == 0.0) and np.all(a[hot] == 0.0)


@pytest.mark.parametrize("table", ["two-species", "four-species"])
def test_low_rank_edges(torch, table):
    """The two- and four-species tables through the two- and four-column kernels with
    zero-density dust cells (the rho -> 0 limit of a_rad, kappa_i(T) from every column),
    cells hotter than the sublimation temperature, temperatures beyond both ends of the
    grid, and species whose weight is zero above 400 K; both FP32 scans."""
    from paper_1001_3301_gb300._lib import RT_TABLE_NU_T_LOW_RANK
    w = synth.disk3d(160, 12, 4, n_nu=48, tau550=30.0, seed=5)
    tg = np.array([12.0, 20.0, 60.0, 140.0, 160.0, 400.0, 900.0])
    kt = TABLES[table](w.nu, tg)
    kt[:, 5:] = np.outer(synth.kappa_synth(w.nu), [0.7, 0.7])   # the ices gone, silicate at 0.7
    rho = w.rho32().copy()
    td = w.tdust32().copy()
    rho.reshape(-1)[::11] = 0.0                   # zero density, dust present
    td.reshape(-1)[::7] = 5.0                     # below the grid
    td.reshape(-1)[3::13] = 1200.0                # above the grid, below t_sub
    assert (td > w.t_sub).any()
    orc = oracle.irradiate_tdep(w.grid.r_if, w.grid.theta_if, w.grid.phi_if, w.t_star, w.r_star, w.nu, tg, kt,
                                w.t_sub, rho.astype(np.float64), td.astype(np.float64), nthreads=8)
    ww = synth.Workload(w.name, w.grid, w.nu, w.kappa, rho, td, tau550=w.tau550)
    from paper_1001_3301_gb300._lib import RT_TABLE_NU_T_RANK2
    kind = RT_TABLE_NU_T_RANK2 if table == "two-species" else RT_TABLE_NU_T_LOW_RANK
    assert _kind(kt, 160) == kind
    for precision in ("fp32_kahan", "fp32_plain"):
        q, a, e, shapes = _run(ww, tg, kt, precision=precision, kind=kind)
        _parity.assert_parity(ww, q, a, e, orc, label=f"{table} edges {precision}")
        zc = (rho == 0.0) & (td <= w.t_sub)
        assert zc.any() and np.all(q[zc] == 0.0) and np.all(a[zc] >= 0.0) and (a[zc] > 0.0).any()
        for shape in shapes:
            q, a, e, _ = _run(ww, tg, kt, shape=shape, precision=precision)
            _parity.assert_parity(ww, q, a, e, orc, label=f"{table} edges {precision} {shape}")


def test_constant_table_matches_plain_tracer(torch):
    w = synth.disk3d(64, 16, 4, n_nu=32, tau550=10.0, seed=2)
    tg = _tg(4)
    kt = np.repeat(w.kappa[:, None], 4, axis=1)
    q, a, e, _ = _run(w, tg, kt)
    q0, a0, e0 = _parity.run_gpu(w)
    mq, _ = _parity.masks(w, _parity.oracle_for(w))
    np.testing.assert_allclose(q[mq], q0[mq], rtol=2e-5)
    assert abs(e.e_abs / e0.e_abs - 1) < 1e-6


def test_planck_mean_uses_kappa_of_t(torch):
    from paper_1001_3301_gb300 import Tracer
    w = synth.disk2d(16, 8, 40)
    tg = _tg(12)
    kt = synth.kappa_synth_t(w.nu, tg)
    tr = Tracer.from_grid(w.grid)
    tr.set_opacity_table_t(w.nu, tg, kt, w.t_sub)
    tr.set_star(w.t_star, w.r_star)
    for t in (20.0, 150.0, 400.0):
        j = int(np.searchsorted(tg, t, side="right") - 1)
        k = kt[:, j] + (kt[:, j + 1] - kt[:, j]) * (t - tg[j]) / (tg[j + 1] - tg[j])
        f = oracle.planck_bins(t, w.nu)
        assert abs(tr.planck_mean_opacity(t) / (np.sum(k * f) / np.sum(f)) - 1) < 1e-12
    tr.close()


def test_unsupported_paths_refuse(torch):
    from paper_1001_3301_gb300 import Batch, RtError, Tracer
    w = synth.disk3d(16, 4, 2, n_nu=8, tau550=1.0, seed=1)
    tg = _tg(4)
    tr = Tracer.from_grid(w.grid)
    tr.set_opacity_table_t(w.nu, tg, synth.kappa_synth_t(w.nu, tg), w.t_sub)
    tr.set_star(w.t_star, w.r_star)
    with pytest.raises(RtError):
        Batch([tr])
    r = torch.from_numpy(w.rho32()).cuda()
    t = torch.from_numpy(w.tdust32()).cuda()
    with pytest.raises(RtError):
        tr.surrogate_train([r], [t], steps=10)
    tr.close()
    w2 = synth.disk3d(1025, 1, 1, n_nu=4, tau550=1.0, seed=1)
    tr2 = Tracer.from_grid(w2.grid)
    tr2.set_opacity_table_t(w2.nu, tg, synth.kappa_synth_t(w2.nu, tg), w2.t_sub)
    tr2.set_star(w2.t_star, w2.r_star)
    with pytest.raises(RtError):
        tr2.irradiate(torch.from_numpy(w2.rho32()).cuda(), torch.from_numpy(w2.tdust32()).cuda())
    tr2.close()
