"""The lookup-table comparator of the per-bin sum (rt_lut_build, rt_irradiate_lut)
against the FP64 oracle: within the table's tolerance where it answers, the exact
1e-5 where every square is flagged (every warp-slot then takes the per-bin sum), and
its refusals."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from tests import _parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _tracer(w, precision="fp32_kahan"):
    from paper_1001_3301_gb300 import Tracer
    tr = Tracer.from_grid(w.grid, precision)
    tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
    tr.set_star(w.t_star, w.r_star)
    return tr


def _fields(torch, w):
    return torch.from_numpy(w.rho32()).cuda(), torch.from_numpy(w.tdust32()).cuda()


@pytest.mark.parametrize("tau", [1.0, 100.0])
@pytest.mark.parametrize("shape", [(1, 8, 4, 6), (1, 16, 4, 4)])
def test_lut_within_tolerance(torch, tau, shape):
    """Every masked cell within 1e-3 of the oracle (q_abs and a_rad), energies too."""
    w = synth.disk3d(256, 48, 8, n_nu=79, tau550=tau, seed=4)
    orc = _parity.oracle_for(w)
    tr = _tracer(w)
    tr.set_tuning(*shape)
    tr.lut_build(1e-3)
    r, t = _fields(torch, w)
    q, a, e, fb = tr.irradiate_lut(r, t, energy=True, stats=True)
    q, a = q.double().cpu().numpy(), a.double().cpu().numpy()
    mq, ma = _parity.masks(w, orc)
    rq = np.abs(q[mq] - orc.q_abs[mq]) / orc.q_abs[mq]
    ra = np.abs(a[ma] - orc.a_rad[ma]) / np.abs(orc.a_rad[ma])
    assert rq.max() <= 1e-3 and ra.max() <= 1e-3, (rq.max(), ra.max(), fb)
    assert np.all(q[orc.q_abs == 0.0] == 0.0)
    assert abs(e.e_abs - orc.e_abs) <= 1e-3 * orc.l_star and abs(e.e_esc - orc.e_esc) <= 1e-6 * orc.l_star
    rays_per_warp = 1 if shape[1] * 32 >= 256 and shape[1] * 16 < 256 else 2
    assert fb is not None and fb < 48 * 8 // rays_per_warp // 2   # most warp-slots answered by the table
    tr.close()


def test_lut_every_square_flagged_is_the_tracer(torch):
    """A tolerance no bilinear square meets: every warp-slot takes the per-bin sum, so
    the result is the tracer's (the 1e-5 of the parity tests), including the rho -> 0
    force limit of the density-floor cells."""
    w = synth.disk2d(64, 32, 16, tau550=100.0)
    assert (w.rho32() == 0).any()
    orc = _parity.oracle_for(w)
    tr = _tracer(w)
    tr.set_tuning(1, 8, 4, 6)          # 8 cells per lane: 8 lanes per 64-cell ray, 4 rays per warp
    tr.lut_build(1e-12)
    r, t = _fields(torch, w)
    q, a, e, fb = tr.irradiate_lut(r, t, energy=True, stats=True)
    _parity.assert_parity(w, q.double().cpu().numpy(), a.double().cpu().numpy(), e, orc, label="all flagged")
    assert fb == (w.grid.ntheta * w.grid.nphi + 3) // 4
    tr.close()


def test_lut_refusals(torch):
    from paper_1001_3301_gb300 import RtError, Tracer
    w = synth.disk3d(64, 8, 4, n_nu=16, tau550=1.0, seed=3)
    r, t = _fields(torch, w)
    tr = _tracer(w)
    with pytest.raises(RtError):      # no table yet
        tr.irradiate_lut(r, t)
    with pytest.raises(RtError):
        tr.lut_build(0.0)
    tr.lut_build(1e-3)
    tr.set_star(6000.0, w.r_star)     # the table belonged to the old star
    with pytest.raises(RtError):
        tr.irradiate_lut(r, t)
    tr.close()
    t64 = _tracer(w, "fp64")
    with pytest.raises(RtError):
        t64.lut_build(1e-3)
    t64.close()
    tg = synth.t_grid(4)
    tt = Tracer.from_grid(w.grid)
    tt.set_opacity_table_t(w.nu, tg, synth.kappa_synth_t(w.nu, tg), w.t_sub)
    tt.set_star(w.t_star, w.r_star)
    with pytest.raises(RtError):
        tt.lut_build(1e-3)
    tt.close()
