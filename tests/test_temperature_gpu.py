"""Planck-mean opacity and the dust-temperature update (Sect. 2.2, Eq. 16 with the
frequency-dependent fluxes of Sect. 2.3) on the GPU against the FP64 oracle, and the
gray irradiation of Eq. 19 with kappa_P(T*) against the frequency-dependent one."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

RTOL_T = 3e-6   # FP32 Newton in ln T (ulp of ln T ~ 5e-7) and the tabulated mean


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _tracer(w, nu=None, kappa=None):
    from paper_1001_3301_gb300 import Tracer
    tr = Tracer.from_grid(w.grid)
    tr.set_opacity_table(w.nu if nu is None else nu, w.kappa if kappa is None else kappa, w.t_sub)
    tr.set_star(w.t_star, w.r_star)
    return tr


@pytest.mark.parametrize("t", [1.0, 3.0, 30.0, 300.0, 1500.0, 5800.0, 3e4, 1e5])
def test_planck_mean_matches_oracle(torch, t):
    w = synth.disk2d(16, 8, 79)
    tr = _tracer(w)
    got = tr.planck_mean_opacity(t)
    ref = oracle.planck_mean(t, w.nu, w.kappa)
    assert abs(got / ref - 1) < 1e-12, (got, ref)
    tr.close()


def _fields(w, torch):
    return torch.from_numpy(w.rho32()).cuda(), torch.from_numpy(w.tdust32()).cuda()


@pytest.mark.parametrize("tau", [0.1, 10.0])
def test_dust_temperature_matches_oracle(torch, tau):
    """Tracer a_rad -> Eq. 16 on the GPU, against the oracle's bisection on the same
    a_rad (and a random E_R field), every cell of a small 3-D disk."""
    w = synth.disk3d(40, 16, 6, n_nu=79, tau550=tau, seed=7)
    tr = _tracer(w)
    r, t = _fields(w, torch)
    _, a, _ = tr.irradiate(r, t)
    rng = np.random.default_rng(3)
    e = (10 ** rng.uniform(-14, -4, w.grid.shape)).astype(np.float32)
    for er in (None, e):
        td = tr.dust_temperature(a, None if er is None else torch.from_numpy(er).cuda())
        got = td.double().cpu().numpy()
        ref = oracle.dust_temperature(a.double().cpu().numpy(), None if er is None else er.astype(np.float64),
                                      w.nu, w.kappa)
        inside = (ref > 1.0) & (ref < 1e5)
        assert inside.mean() > 0.9
        rel = np.abs(got[inside] / ref[inside] - 1)
        assert rel.max() < RTOL_T, rel.max()
        assert np.all(np.isfinite(got)) and np.all(got >= 0)
    tr.close()


@pytest.mark.parametrize("table", ["disk", "step"])
def test_dust_temperature_whole_range(torch, table):
    """E_R = 0 over the whole range of a_rad: temperatures from 0.3 K to 3e5 K (beyond
    both ends of the tabulated mean, and densely around them, where the inverse table
    bends), for the disk's opacities and for a table that steps by 1e3 at 30 micron
    (a steep Planck mean). Every cell against the oracle's FP64 bisection."""
    w = synth.disk3d(40, 25, 20, n_nu=79, tau550=1.0, seed=1)   # 20,000 cells, one per temperature
    kappa = w.kappa if table == "disk" else np.where(w.nu > synth.C_CM_S / 30e-4, 1e3, 1.0)
    tr = _tracer(w, kappa=kappa)
    a_const = 4 * 5.670374419e-5 / 2.99792458e10
    rng = np.random.default_rng(11)
    t_want = np.concatenate([10 ** rng.uniform(np.log10(0.3), np.log10(3e5), 16_000),
                             10 ** rng.uniform(-0.05, 0.05, 2_000), 1e5 * 10 ** rng.uniform(-0.05, 0.05, 2_000)])
    kp = np.array([oracle.planck_mean(min(max(t, 1.0), 1e5), w.nu, kappa) for t in np.geomspace(0.3, 3e5, 64)])
    kp_i = np.exp(np.interp(np.log(t_want), np.log(np.geomspace(0.3, 3e5, 64)), np.log(kp)))
    a = (a_const * t_want ** 4 * kp_i).astype(np.float32).reshape(w.grid.shape)  # about those temperatures
    assert np.all(a > 0)
    got = tr.dust_temperature(torch.from_numpy(a).cuda()).double().cpu().numpy()
    ref = oracle.dust_temperature(a.astype(np.float64), None, w.nu, kappa)
    rel = np.abs(got / ref - 1)
    assert rel.max() < RTOL_T, (rel.max(), ref[np.argmax(rel)])
    tr.close()


def test_zero_source_gives_zero(torch):
    w = synth.disk2d(16, 8, 16)
    tr = _tracer(w)
    z = torch.zeros(w.grid.shape, dtype=torch.float32, device="cuda")
    assert torch.count_nonzero(tr.dust_temperature(z)) == 0
    tr.close()


def _gray_and_freq(w, torch):
    trf = _tracer(w)
    kp = trf.planck_mean_opacity(w.t_star)
    trg = _tracer(w, nu=np.array([5e14]), kappa=np.array([kp]))
    r, t = _fields(w, torch)
    _, af, _ = trf.irradiate(r, t)
    _, ag, _ = trg.irradiate(r, t)
    tf = trf.dust_temperature(af).double().cpu().numpy()
    tg = trf.dust_temperature(ag).double().cpu().numpy()
    trf.close()
    trg.close()
    return tf, tg


def test_gray_equals_frequency_dependent_when_thin(torch):
    """Gray irradiation with kappa_P(T*) (Eq. 19) absorbs sum_i kappa_i F_i in an
    optically thin medium, as the frequency-dependent one does: equal dust
    temperatures (tau550 = 1e-7: every bin's optical depth below 1e-4)."""
    w = synth.disk3d(48, 16, 4, n_nu=79, tau550=1e-7, seed=5)
    tf, tg = _gray_and_freq(w, torch)
    dust = w.tdust32() <= w.t_sub
    np.testing.assert_allclose(tf[dust], tg[dust], rtol=1e-4)


def test_gray_versus_frequency_dependent_thick(torch):
    """In the tau550 = 100 disk the gray opacity of the stellar spectrum stops the
    starlight earlier than the frequency-dependent treatment, whose long-wavelength
    bins reach deeper: the midplane interior is warmer with frequency dependence
    (the contrast of the paper's gray and frequency-dependent runs)."""
    w = synth.disk3d(64, 32, 4, n_nu=79, tau550=100.0, seed=5)
    tf, tg = _gray_and_freq(w, torch)
    mid = w.grid.ntheta // 2
    inner = slice(w.grid.nr // 4, 3 * w.grid.nr // 4)
    f, g = tf[:, mid - 1:mid + 1, inner], tg[:, mid - 1:mid + 1, inner]
    warmer = (f > 1.01 * g).mean()
    print(f"midplane interior: frequency-dependent warmer than gray in {100 * warmer:.0f} % of cells; "
          f"median T_freq {np.median(f):.1f} K, T_gray {np.median(g):.1f} K")
    assert warmer > 0.5
