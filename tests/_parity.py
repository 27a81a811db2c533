"""Helpers for GPU-vs-oracle parity checks.

Tolerances (from the accuracy target of the tracer):
  * q_abs: relative 1e-5 in every cell that absorbs more than 1e-12 of the
    stellar luminosity into the grid;
  * a_rad: relative 1e-5 in the same cells, plus cells with dust and rho == 0
    that see at least 1e-12 of the flux entering the grid (the rho -> 0 limit);
  * elsewhere an absolute bound of 1e-5 of the largest value (the cells outside
    the mask carry < 1e-12 L* each);
  * energy: |(E_abs + E_esc)/L* - 1| < 1e-6, and E_abs within 1e-6 of the oracle's.
"""
from __future__ import annotations

import numpy as np

import oracle

RTOL_Q = 1e-5
RTOL_A = 1e-5
MASK_FRAC = 1e-12
RTOL_ENERGY = 1e-6


def run_gpu(w, precision="fp32_kahan", shape=None, rho=None, tdust=None, kappa=None,
            kappa_bf16=False, tracer=None):
    """Trace a synth.Workload on cuda:0; returns (q, a, energy) as float64 numpy."""
    import torch
    from paper_1001_3301_gb300 import Tracer
    rho = w.rho32() if rho is None else rho.astype(np.float32)
    tdust = w.tdust32() if tdust is None else tdust.astype(np.float32)
    tr = tracer or Tracer.from_grid(w.grid, precision)
    tr.set_opacity_table(w.nu, w.kappa if kappa is None else kappa, w.t_sub, kappa_bf16)
    tr.set_star(w.t_star, w.r_star)
    if shape is not None:
        tr.set_tuning(*shape)
    r = torch.from_numpy(np.ascontiguousarray(rho)).cuda()
    t = torch.from_numpy(np.ascontiguousarray(tdust)).cuda()
    q, a, e = tr.irradiate(r, t, energy=True)
    torch.cuda.synchronize()
    out = q.double().cpu().numpy(), a.double().cpu().numpy(), e
    if tracer is None:
        tr.close()
    return out


def oracle_for(w, rho=None, tdust=None, kappa=None):
    return oracle.irradiate_workload(
        w, rho=None if rho is None else rho.astype(np.float32).astype(np.float64),
        tdust=None if tdust is None else tdust.astype(np.float32).astype(np.float64),
        kappa=kappa)


def masks(w, orc, rho=None, tdust=None):
    rho = (w.rho32() if rho is None else rho.astype(np.float32)).astype(np.float64)
    tdust = (w.tdust32() if tdust is None else tdust.astype(np.float32)).astype(np.float64)
    mq = orc.p_abs > MASK_FRAC * orc.l_star
    # rho == 0 cells with dust: the force is the flux-weighted opacity; keep those
    # whose force is within 1e-12 of the largest such value
    zero = (rho == 0.0) & (tdust <= w.t_sub)
    az = np.where(zero, orc.a_rad, 0.0)
    ma = mq | (zero & (az > MASK_FRAC * max(az.max(), 1e-300)))
    return mq, ma


def assert_parity(w, q, a, e, orc, rtol_q=RTOL_Q, rtol_a=RTOL_A, rtol_energy=RTOL_ENERGY,
                  rho=None, tdust=None, label=""):
    assert np.all(np.isfinite(q)) and np.all(np.isfinite(a)), f"{label}: non-finite output"
    mq, ma = masks(w, orc, rho, tdust)
    assert mq.sum() > 0 or orc.e_abs == 0.0
    rq = np.abs(q[mq] - orc.q_abs[mq]) / orc.q_abs[mq]
    assert rq.size == 0 or rq.max() <= rtol_q, f"{label}: q_abs rel err {rq.max():.3e} > {rtol_q}"
    if ma.any():
        ra = np.abs(a[ma] - orc.a_rad[ma]) / np.abs(orc.a_rad[ma])
        assert ra.max() <= rtol_a, f"{label}: a_rad rel err {ra.max():.3e} > {rtol_a}"
    qa = np.abs(q - orc.q_abs).max()
    assert qa <= rtol_q * max(orc.q_abs.max(), 1e-300) + 1e-300, f"{label}: q_abs abs err {qa:.3e}"
    aa = np.abs(a - orc.a_rad).max()
    assert aa <= rtol_a * max(np.abs(orc.a_rad).max(), 1e-300) + 1e-300, f"{label}: a_rad abs err {aa:.3e}"
    # where the oracle gives exactly zero (sublimated cells) the GPU does too
    z = orc.q_abs == 0.0
    assert np.all(q[z] == 0.0), f"{label}: q_abs non-zero where the oracle has zero"
    if e is not None:
        assert abs(e.rel_err) <= rtol_energy, f"{label}: energy rel err {e.rel_err:.3e}"
        assert abs(e.l_star / orc.l_star - 1) <= 1e-9, f"{label}: l_star"
        # absorbed and escaped parts each within rtol_energy of L* of the oracle's
        assert abs(e.e_abs - orc.e_abs) <= rtol_energy * orc.l_star, f"{label}: e_abs {e.e_abs} vs {orc.e_abs}"
        assert abs(e.e_esc - orc.e_esc) <= rtol_energy * orc.l_star, f"{label}: e_esc {e.e_esc} vs {orc.e_esc}"
    return dict(q_max_rel=float(rq.max()) if rq.size else 0.0, n_mask=int(mq.sum()))
