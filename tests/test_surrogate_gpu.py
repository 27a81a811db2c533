"""The learned surrogate on the GPU: training kernels against the FP64 reference
network (gradients), the tensor-core inference against the reference forward
pass, the fused ray kernel against the oracle pipeline, the exact fallback and
the gate against the FP64 tracer, and what the trained network gains over the
exact per-bin sum."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from oracle import mlp
import synth
from tests import _parity

pytestmark = pytest.mark.gpu

TOL = 1e-3   # per-cell relative error bound of q_abs the surrogate is held to


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _tracer(w):
    from paper_1001_3301_gb300 import Tracer
    tr = Tracer.from_grid(w.grid)
    tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
    tr.set_star(w.t_star, w.r_star)
    return tr


def _bf16(a):
    """Round to BF16 (nearest, ties to even), as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _rounded(p: mlp.Params) -> mlp.Params:
    """The network the tensor cores evaluate: W1, b1, W2 in BF16, the rest FP32."""
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return mlp.Params(_bf16(p.W1), _bf16(p.b1), _bf16(p.W2), f32(p.b2), f32(p.w3), float(np.float32(p.b3)))


def _random_params(seed):
    p = mlp.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    p.b1 = rng.normal(0, 0.3, mlp.H)
    p.b2 = rng.normal(0, 0.3, mlp.H)
    p.b3 = 0.1
    return p


def _rows(n, seed):
    """Feature rows in the range real cells produce."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.2, 0.6, (n, mlp.NF))
    x[:, 6] = rng.uniform(-0.8, 0.7, n)
    return x.astype(np.float32).astype(np.float64)


def test_gradient_matches_fp64_reference(torch):
    """One forward + backward of the training kernels (BF16 tensor-core products,
    FP32 accumulation) against the FP64 chain rule on the same BF16 weights,
    element by element: |g - g_ref| <= rtol |g_ref| + floor max|g_ref| in every
    entry of every tensor. The output layer and b2 are FP32 all the way (rtol 1e-4,
    floor 1e-5); W1, b1 and W2 see the BF16 rounding of dZ2 and dZ1 (2^-9 relative
    per product term, so about 2e-3 on a sum over rows whose terms do not cancel:
    rtol 1e-2), and entries whose row sums cancel keep the absolute part of that
    rounding (floor 1e-3 of the tensor's largest entry). The bound is checked to be
    tight enough that a copy of the reference with one entry, its largest, off by 3 %
    fails it."""
    w = synth.disk2d()
    tr = _tracer(w)
    p = _random_params(11)
    tr.surrogate_set_params(p.flat(), 0.0, 1.0)
    x = _rows(1000, 5)                   # not a multiple of the 256-row blocks
    t = np.random.default_rng(6).normal(0, 1, 1000)
    loss, g = tr.surrogate_grad(x, t)
    pr = _rounded(mlp.Params.from_flat(tr.surrogate_params()[0]))
    lref, gref = mlp.loss_and_grad(pr, x, t)
    assert abs(loss / lref - 1) < 1e-4
    sizes = [("W1", mlp.NF * mlp.H, 1e-2, 1e-3), ("b1", mlp.H, 1e-2, 1e-3),
             ("W2", mlp.H * mlp.H, 1e-2, 1e-3), ("b2", mlp.H, 1e-4, 1e-5),
             ("w3", mlp.H, 1e-4, 1e-5), ("b3", 1, 1e-4, 1e-5)]
    o = 0
    for name, n, rtol, floor in sizes:
        a, b = g[o:o + n].astype(np.float64), gref[o:o + n]
        bound = rtol * np.abs(b) + floor * np.abs(b).max()
        over = np.abs(a - b) > bound
        k = int(np.argmax(np.abs(a - b) / bound))
        assert not over.any(), (f"{name}: {int(over.sum())} of {n} entries outside the bound; worst entry {k}: "
                                f"{a[k]:.6e} vs {b[k]:.6e}")
        planted = b.copy()
        planted[np.argmax(np.abs(b))] *= 1.03
        assert (np.abs(planted - b) > bound).any(), f"{name}: the bound misses a 3 % error in one entry"
        o += n
    tr.close()


def test_inference_matches_fp64_forward(torch):
    """The tcgen05 inference (features and first-layer activations as sums of BF16
    parts, BF16 weights, FP32 accumulators in TMEM) against the FP64 forward pass
    of the same BF16 weights."""
    w = synth.disk2d()
    tr = _tracer(w)
    p = _random_params(21)
    tr.surrogate_set_params(p.flat(), 0.0, 1.0)
    x = _rows(5000, 7)
    y = tr.surrogate_eval(x).astype(np.float64)
    yref, _ = mlp.forward(_rounded(mlp.Params.from_flat(tr.surrogate_params()[0])), x)
    err = np.abs(y - yref)
    assert err.max() < 1e-4 * (1 + np.abs(yref).max()), err.max()
    tr.close()


def _volumes(g):
    """Cell volumes dOmega (r+^3 - r-^3) / 3 in the [nphi][ntheta][nr] layout."""
    dom = np.outer(np.diff(g.phi_if), np.cos(g.theta_if[:-1]) - np.cos(g.theta_if[1:]))
    return dom[:, :, None] * (g.r_if[1:] ** 3 - g.r_if[:-1] ** 3)[None, None, :] / 3.0


def _fields(w):
    import torch
    return (torch.from_numpy(w.rho32()).cuda(), torch.from_numpy(w.tdust32()).cuda())


def test_fallback_with_untrained_network_is_exact(torch):
    """A random network fails the trust map almost everywhere; the cells it does
    not answer take the exact per-bin sum, so the result meets the tracer's 1e-5
    bound (2e-5 here: the fallback sums in plain FP32)."""
    w = synth.disk3d(40, 16, 8, n_nu=32, tau550=10.0, seed=4)
    tr = _tracer(w)
    tr.surrogate_set_params(_random_params(3).flat(), -8.0, 4.0)
    r, t = _fields(w)
    q, a, st = tr.irradiate_surrogate(r, t, err_tol=TOL, validate=0)
    orc = _parity.oracle_for(w)
    mq, _ = _parity.masks(w, orc)
    qn = q.double().cpu().numpy()
    rel = np.abs(qn[mq] / orc.q_abs[mq] - 1)
    assert rel.max() < 2e-5, rel.max()
    assert st["n_fallback"] > 0
    tr.close()


@pytest.fixture(scope="module")
def trained(torch):
    """A surrogate trained on four optical depths of a small 3-D disk."""
    geo = dict(nr=48, ntheta=24, nphi=16, n_nu=79)
    ws = [synth.disk3d(**geo, tau550=tau, seed=30 + i) for i, tau in enumerate((0.1, 1.0, 10.0, 100.0))]
    tr = _tracer(ws[0])
    fields = [_fields(w) for w in ws]
    st = tr.surrogate_train([f[0] for f in fields], [f[1] for f in fields], n_samples=400000,
                            batch=2048, steps=4000, lr=2e-3, seed=5)
    test = synth.disk3d(**geo, tau550=3.0, seed=99)
    yield tr, st, test
    tr.close()


def test_training_converges(trained):
    tr, st, _ = trained
    h = tr.surrogate_loss_history()
    print("train stats", st, "loss first/last", h[:20].mean(), h[-40:].mean())
    assert st["n_train"] > 10000 and st["n_val"] > 100
    assert h[-40:].mean() < 0.02 * h[:20].mean()
    assert math.isfinite(st["val_rms"]) and st["val_rms"] < 0.5


def _oracle_pipeline_q(w, tr):
    """q_abs and a_rad of the trained network evaluated by the FP64 reference on the
    oracle's columns: the fused kernel's scan, features, network and outputs in one."""
    params, mu, sigma = tr.surrogate_params()
    p = _rounded(mlp.Params.from_flat(params))
    g = w.grid
    rho = w.rho32().astype(np.float64)
    td = w.tdust32().astype(np.float64)
    dr = np.diff(g.r_if)
    dust = td <= w.t_sub
    dn = np.where(dust, rho * dr, 0.0)
    n_in = np.cumsum(dn, axis=-1) - dn
    kref, k550 = mlp.reference_kappas(w.nu, w.kappa)
    x = mlp.features(n_in, dn, td, kref, k550).reshape(-1, mlp.NF)
    y, _ = mlp.forward(p, x)
    gg = np.exp(mu + sigma * y).reshape(dn.shape)
    f = oracle.planck_bins(w.t_star, w.nu)
    gq = 3.0 * w.r_star ** 2 * f.max() / (g.r_if[1:] ** 3 - g.r_if[:-1] ** 3)
    q = np.where(dust, gq * gg * k550 * dn, 0.0)
    a = np.where(dust, gq * dr / synth.C_CM_S * gg * k550, 0.0)
    return q, a, dust


def test_network_only_matches_reference_pipeline(trained):
    """validate == 2 (the network in every cell) against the FP64 pipeline on the
    same BF16 weights: scan, features, network and outputs of the fused kernel."""
    tr, _, w = trained
    r, t = _fields(w)
    q, a, _ = tr.irradiate_surrogate(r, t, validate=2)
    qref, aref, dust = _oracle_pipeline_q(w, tr)
    qn, an = q.double().cpu().numpy(), a.double().cpu().numpy()
    m = dust & (qref > 0)
    assert np.all(qn[~dust] == 0) and np.all(an[~dust] == 0)
    assert np.max(np.abs(qn[m] / qref[m] - 1)) < 5e-4
    assert np.max(np.abs(an[dust] / aref[dust] - 1)) < 5e-4


def test_validate_mode_meets_tolerance(trained):
    """validate == 1: the exact tracer judges each cell; the result is within
    err_tol of the FP64 oracle wherever a cell absorbs more than 1e-12 of L*."""
    tr, _, w = trained
    r, t = _fields(w)
    q, a, st = tr.irradiate_surrogate(r, t, err_tol=TOL, validate=1)
    orc = _parity.oracle_for(w)
    mq, _ = _parity.masks(w, orc)
    qn = q.double().cpu().numpy()
    rel = np.abs(qn[mq] / orc.q_abs[mq] - 1)
    print("validate stats", st, "fraction answered by the network",
          1 - st["n_fallback"] / max(st["n_dust"], 1))
    assert rel.max() <= TOL * (1 + 1e-3) + 2e-5
    assert st["n_judged"] > 0 and st["max_rel_err"] >= 0
    assert abs(st["rel_err"]) < TOL


def test_gate_mode_meets_tolerance(trained):
    """validate == 0: the trust map decides without the exact tracer; cells outside
    it take the exact per-bin sum. Every judged cell is within err_tol."""
    tr, _, w = trained
    r, t = _fields(w)
    q, a, st = tr.irradiate_surrogate(r, t, err_tol=TOL, validate=0)
    orc = _parity.oracle_for(w)
    mq, _ = _parity.masks(w, orc)
    qn = q.double().cpu().numpy()
    rel = np.abs(qn[mq] / orc.q_abs[mq] - 1)
    bits, _ = tr.surrogate_trust_map(TOL)
    print("gate stats", st, "trusted bins", int(bits.sum()), "max rel", rel.max())
    assert rel.max() <= TOL
    assert abs(st["rel_err"]) < TOL


def test_save_load_roundtrip(trained, tmp_path):
    from paper_1001_3301_gb300 import RtError
    tr, _, w = trained
    path = str(tmp_path / "sur.bin")
    tr.surrogate_save(path)
    tr2 = _tracer(w)
    tr2.surrogate_load(path)
    x = _rows(700, 9)
    assert np.array_equal(tr.surrogate_eval(x), tr2.surrogate_eval(x))
    p1, mu1, s1 = tr.surrogate_params()
    p2, mu2, s2 = tr2.surrogate_params()
    assert np.array_equal(p1, p2) and mu1 == mu2 and s1 == s2
    tr2.close()
    # a different sublimation temperature changes the function: refused
    from paper_1001_3301_gb300 import Tracer
    tr3 = Tracer.from_grid(w.grid)
    tr3.set_opacity_table(w.nu, w.kappa, w.t_sub + 1.0)
    tr3.set_star(w.t_star, w.r_star)
    with pytest.raises(RtError):
        tr3.surrogate_load(path)
    tr3.close()


def test_gain_over_exact_tracer(trained, torch):
    """What the trained network gains over the method without it: device time of
    the gated surrogate (validate == 0) against the exact tracer on the same grid,
    and the accuracy it keeps. The ratio is reported, not asserted: on this GPU the
    exact per-bin sum costs about one exp2 per cell and bin, the network 256 SiLU
    activations and ~19k multiply-adds per cell."""
    tr0, _, _ = trained
    w = synth.disk3d(256, 64, 64, n_nu=79, tau550=3.0, seed=98)
    tr = _tracer(w)
    path = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"sur_gain_{os.getpid()}.bin")
    tr0.surrogate_save(path)
    tr.surrogate_load(path)
    os.remove(path)
    r, t = _fields(w)
    q_ex, a_ex, _ = tr.irradiate(r, t)
    q_s, a_s, st = tr.irradiate_surrogate(r, t, err_tol=TOL, validate=0)

    def timed(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_ex = timed(lambda: tr.irradiate(r, t, q_ex, a_ex))
    t_s = timed(lambda: tr.irradiate_surrogate(r, t, q_s, a_s, err_tol=TOL, validate=0, stats=False))
    _, _, e = tr.irradiate(r, t, q_ex, a_ex, energy=True)
    qe, qs = q_ex.double().cpu().numpy(), q_s.double().cpu().numpy()
    m = qe * _volumes(w.grid) > 1e-12 * e.l_star   # cells absorbing more than 1e-12 L*
    rel = np.abs(qs[m] / qe[m] - 1)
    ncell = w.grid.ncells
    print(f"gain: exact {t_ex:.3f} ms ({ncell / t_ex / 1e6:.3e} cells/s), surrogate {t_s:.3f} ms "
          f"({ncell / t_s / 1e6:.3e} cells/s), speed-up {t_ex / t_s:.3f}, fallback "
          f"{st['n_fallback'] / max(st['n_dust'], 1):.3f}, max rel err {rel.max():.2e}")
    assert rel.max() < 2 * TOL
    tr.close()
