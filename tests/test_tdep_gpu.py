"""The tracer with temperature-dependent opacity tables (per-bin scans of Eq. 19 with
every cell's own kappa) against the FP64 oracle."""
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


def _run(w, tg, kt, shape=None):
    import torch
    from paper_1001_3301_gb300 import Tracer
    tr = Tracer.from_grid(w.grid)
    tr.set_opacity_table_t(w.nu, tg, kt, w.t_sub)
    tr.set_star(w.t_star, w.r_star)
    if shape is not None:
        tr.set_tuning(*shape)
    r = torch.from_numpy(w.rho32()).cuda()
    t = torch.from_numpy(w.tdust32()).cuda()
    q, a, e = tr.irradiate(r, t, energy=True)
    out = q.double().cpu().numpy(), a.double().cpu().numpy(), e, tr.tunings()
    tr.close()
    return out


@pytest.mark.parametrize("tau", [0.1, 1.0, 100.0])
def test_disk_against_oracle(torch, tau):
    w = synth.disk3d(96, 24, 8, n_nu=79, tau550=tau, seed=11)
    tg = synth.t_grid(24)
    kt = synth.kappa_synth_t(w.nu, tg)
    orc = _oracle(w, tg, kt)
    q, a, e, _ = _run(w, tg, kt)
    _parity.assert_parity(w, q, a, e, orc, label=f"tdep tau {tau}")


@pytest.mark.parametrize("dims", [(1, 1, 1, 1), (7, 3, 2, 5), (33, 5, 3, 17), (65, 4, 2, 40), (200, 3, 2, 79),
                                  (513, 2, 2, 32), (1024, 2, 1, 16)],
                         ids=lambda d: "x".join(map(str, d)))
def test_ragged_all_shapes(torch, dims):
    nr, nth, nph, nnu = dims
    w = synth.disk3d(nr, nth, nph, n_nu=nnu, tau550=10.0, seed=nr + nth)
    tg = synth.t_grid(9)
    kt = synth.kappa_synth_t(w.nu, tg)
    orc = _oracle(w, tg, kt)
    _, _, _, shapes = _run(w, tg, kt)
    assert shapes and all(s[0] == 1 for s in shapes)
    for shape in shapes:
        q, a, e, _ = _run(w, tg, kt, shape=shape)
        _parity.assert_parity(w, q, a, e, orc, label=f"tdep {dims} {shape}")


def test_constant_table_matches_plain_tracer(torch):
    w = synth.disk3d(64, 16, 4, n_nu=32, tau550=10.0, seed=2)
    tg = synth.t_grid(4)
    kt = np.repeat(w.kappa[:, None], 4, axis=1)
    q, a, e, _ = _run(w, tg, kt)
    q0, a0, e0 = _parity.run_gpu(w)
    mq, _ = _parity.masks(w, _parity.oracle_for(w))
    np.testing.assert_allclose(q[mq], q0[mq], rtol=2e-5)
    assert abs(e.e_abs / e0.e_abs - 1) < 1e-6


def test_planck_mean_uses_kappa_of_t(torch):
    from paper_1001_3301_gb300 import Tracer
    w = synth.disk2d(16, 8, 40)
    tg = synth.t_grid(12)
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
    tg = synth.t_grid(4)
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
