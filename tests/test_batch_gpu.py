"""The multi-grid batch (one persistent launch, CUDA graph) against the oracle
and against tracing every grid on its own."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth
from tests import _parity, _pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _make(specs):
    ws = [synth.disk3d(s["nr"], s["ntheta"], s["nphi"], n_nu=s["n_nu"], tau550=s["tau550"], seed=s["seed"])
          for s in specs]
    return ws


def _tracers(ws, precision="fp32_kahan"):
    from paper_1001_3301_gb300 import Tracer
    trs = []
    for w in ws:
        tr = Tracer.from_grid(w.grid, precision)
        tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
        tr.set_star(w.t_star, w.r_star)
        trs.append(tr)
    return trs


def _fields(torch, ws):
    rho = [torch.from_numpy(w.rho32()).cuda() for w in ws]
    td = [torch.from_numpy(w.tdust32()).cuda() for w in ws]
    q = [torch.full_like(r, float("nan")) for r in rho]
    a = [torch.full_like(r, float("nan")) for r in rho]
    return rho, td, q, a


SMALL = [dict(nr=nr, ntheta=nt, nphi=np_, n_nu=nn, tau550=t, seed=i)
         for i, (nr, nt, np_, nn, t) in enumerate([
             (64, 8, 1, 32, 0.1), (65, 9, 3, 79, 1.0), (200, 5, 4, 128, 30.0), (33, 31, 2, 32, 100.0),
             (512, 4, 3, 79, 3.0), (129, 17, 1, 128, 0.5), (300, 6, 5, 79, 10.0), (1, 7, 3, 5, 1.0),
             (97, 12, 2, 32, 60.0), (256, 8, 8, 79, 2.0), (7, 3, 2, 16, 5.0), (480, 3, 2, 128, 100.0)])]


def test_batch_against_oracle_every_shape(torch):
    from paper_1001_3301_gb300 import Batch
    ws = _make(SMALL)
    trs = _tracers(ws)
    rho, td, q, a = _fields(torch, ws)
    orcs = [_parity.oracle_for(w) for w in ws]
    with Batch(trs) as b:
        b.run(rho, td, q, a)
        es = b.energy()
        for w, o, qq, aa, e in zip(ws, orcs, q, a, es):
            _parity.assert_parity(w, qq.double().cpu().numpy(), aa.double().cpu().numpy(), e, o,
                                  label=w.name)
        shape = b.autotune(rho, td, q, a, reps=2)
        assert shape[0] in (0, 1)
        for rep in range(2):  # graph replays after the autotuner rebuilt the plan
            for x in q + a:
                x.fill_(float("nan"))
            b.run(rho, td, q, a)
            es = b.energy()
            for w, o, qq, aa, e in zip(ws, orcs, q, a, es):
                _parity.assert_parity(w, qq.double().cpu().numpy(), aa.double().cpu().numpy(), e, o,
                                      label=f"{w.name} rep {rep}")
    for tr in trs:
        tr.close()


@pytest.mark.parametrize("shape", [(1, 16, 4, 3), (1, 16, 4, 4), (1, 8, 4, 6)])
def test_batch_warp_per_ray_shapes(torch, shape):
    """The warp-per-ray batch body (8, 16 or 32 lanes per ray chosen per grid)
    against the oracle; shapes whose rays cannot hold a grid are refused."""
    from paper_1001_3301_gb300 import Batch, RtError
    specs = SMALL if shape[1] == 16 else [s for s in SMALL if s["nr"] <= 256]
    ws = _make(specs)
    trs = _tracers(ws)
    rho, td, q, a = _fields(torch, ws)
    orcs = [_parity.oracle_for(w) for w in ws]
    with Batch(trs) as b:
        assert b.set_tuning(*shape) == shape
        for rep in range(2):
            for x in q + a:
                x.fill_(float("nan"))
            b.run(rho, td, q, a)
            es = b.energy()
            for w, o, qq, aa, e in zip(ws, orcs, q, a, es):
                _parity.assert_parity(w, qq.double().cpu().numpy(), aa.double().cpu().numpy(), e, o,
                                      label=f"{w.name} {shape} rep {rep}")
    if shape[1] == 8:  # the 512-cell rays do not fit 32 lanes x 8 cells
        big = _make([s for s in SMALL if s["nr"] > 256][:2])
        trs2 = _tracers(big)
        with Batch(trs2) as b2:
            with pytest.raises(RtError, match="INVALID"):
                b2.set_tuning(*shape)
        for tr in trs2:
            tr.close()
    for tr in trs:
        tr.close()


def test_batch_matches_single_grid_calls(torch):
    """Same kernel family, same arithmetic: the batch equals per-grid rt_irradiate
    up to the summation order of the tile carries."""
    from paper_1001_3301_gb300 import Batch
    ws = _make(SMALL[:6])
    trs = _tracers(ws)
    rho, td, q, a = _fields(torch, ws)
    for tr in trs:
        tr.set_tuning(0, 8, 4, 6)
    singles = [tr.irradiate(r, t, energy=True) for tr, r, t in zip(trs, rho, td)]
    with Batch(trs) as b:
        b.run(rho, td, q, a)
        es = b.energy()
    for (qs, as_, e1), qb, ab, e2 in zip(singles, q, a, es):
        qs, qb = qs.double().cpu().numpy(), qb.double().cpu().numpy()
        m = qs > 0
        assert np.max(np.abs(qb[m] - qs[m]) / qs[m]) < 1e-6
        assert abs(e1.e_abs - e2.e_abs) <= 1e-7 * e1.l_star
    for tr in trs:
        tr.close()


def test_full_96_grid_batch(torch):
    """The 96 uneven grids of the batch workload (Nr 64-512, Ntheta 32-256,
    Nphi 1/64/128, 32/79/128 bins, tau550 0.1-100): energy of every grid and
    sampled rays against the oracle."""
    from paper_1001_3301_gb300 import Batch
    specs = synth.batch_specs(96, seed=3)
    rng = np.random.default_rng(11)
    worst = 0.0
    ws = _make(specs)
    trs = _tracers(ws)
    rho, td, q, a = _fields(torch, ws)
    with Batch(trs) as b:
        b.autotune(rho, td, q, a, reps=1)
        b.run(rho, td, q, a)
        es = b.energy()
    for w, qq, aa, e in zip(ws, q, a, es):
        assert abs(e.rel_err) < 1e-6, w.name
        g = w.grid
        rays = rng.choice(g.ntheta * g.nphi, size=min(24, g.ntheta * g.nphi), replace=False)
        th = np.linspace(0.0, math.pi, len(rays) + 1)
        o = oracle.irradiate(g.r_if, th, np.array([0.0, 2 * math.pi]), w.t_star, w.r_star, w.nu,
                             w.kappa, w.t_sub, w.rho32().reshape(-1, g.nr)[rays].astype(np.float64),
                             w.tdust32().reshape(-1, g.nr)[rays].astype(np.float64))
        qs = qq.cpu().numpy().reshape(-1, g.nr)[rays].astype(np.float64)
        dom = _pins.solid_angles(g.theta_if, g.phi_if).reshape(-1)[rays]
        oq = o.q_abs.reshape(len(rays), g.nr)
        p_cell = oq * dom[:, None] * _pins.shell_volumes(g.r_if)[None, :]
        lstar = 4 * math.pi * w.r_star ** 2 * oracle.sigma_sb() * w.t_star ** 4
        m = p_cell > 1e-12 * lstar
        if m.any():
            r = np.max(np.abs(qs[m] - oq[m]) / oq[m])
            worst = max(worst, r)
            assert r <= 1e-5, w.name
    for tr in trs:
        tr.close()
    assert worst > 0
