"""rt_irradiate_static, the allocation-free entry point, against rt_irradiate.

It exists for callers that cannot allocate device memory when they need the
irradiation (a host code whose pool already holds the GPU memory, or a time
loop where cudaMalloc/cudaFree would synchronise the device). It keeps all its
scratch in one static device array that every call shares, so these checks call
it through the C ABI in a sequence meant to expose stale scratch: first on a
larger grid (other nr, other bin count, hotter star, tau550 = 100) whose density
holds a NaN, which must set the input-validity word and fail; then twice in a
row on a smaller grid, each result compared with the context-based entry point
on that grid, with the device's free memory unchanged across those two calls.
Every precision mode runs through it. The file name sorts last so that a run
stopping at the first failure has already run every other test; it also passes
on its own in a fresh process.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import synth
from tests import _parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _desc(lib_mod, grid, precision):
    P = ctypes.POINTER(ctypes.c_double)
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (grid.r_if, grid.theta_if, grid.phi_if)]
    d = lib_mod.RtGridDesc(grid.nr, grid.ntheta, grid.nphi, arrs[0].ctypes.data_as(P),
                           arrs[1].ctypes.data_as(P), arrs[2].ctypes.data_as(P), precision)
    return d, arrs


def _static_call(torch, lib_mod, w, rho, td, q, a, precision, t_star=None):
    """One call through the C ABI; returns (status, energy). q and a are
    pre-allocated so that nothing is allocated around the call."""
    d, keep = _desc(lib_mod, w.grid, precision)
    nu = np.ascontiguousarray(w.nu, dtype=np.float64)
    kap = np.ascontiguousarray(w.kappa, dtype=np.float64)
    P = ctypes.POINTER(ctypes.c_double)
    e = lib_mod.RtEnergy()
    st = lib_mod.lib.rt_irradiate_static(
        ctypes.byref(d), w.t_star if t_star is None else t_star, w.r_star, len(nu), nu.ctypes.data_as(P),
        kap.ctypes.data_as(P), w.t_sub, 0, rho.data_ptr(), td.data_ptr(), q.data_ptr(), a.data_ptr(),
        ctypes.byref(e), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, e


CASES = [("fp32_kahan", (256, 32, 16, 79)), ("fp32_kahan", (65, 9, 4, 17)),
         ("fp32_plain", (256, 32, 16, 79)), ("fp32_plain", (65, 9, 4, 17)),
         ("fp64", (65, 9, 4, 17))]


@pytest.mark.parametrize("precision,dims", CASES, ids=lambda x: x if isinstance(x, str) else "x".join(map(str, x)))
def test_static_matches_context_entry_point_twice(torch_cuda, precision, dims):
    torch = torch_cuda
    from paper_1001_3301_gb300 import Tracer, _lib
    code = {"fp32_kahan": _lib.RT_FP32_KAHAN, "fp32_plain": _lib.RT_FP32_PLAIN, "fp64": _lib.RT_FP64}[precision]
    nr, nth, nph, nnu = dims
    w = synth.disk3d(nr, nth, nph, n_nu=nnu, tau550=10.0, seed=nr)
    rho = torch.from_numpy(w.rho32()).cuda()
    td = torch.from_numpy(w.tdust32()).cuda()
    with Tracer.from_grid(w.grid, precision) as tr:
        tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
        tr.set_star(w.t_star, w.r_star)
        q_ref, a_ref, e_ref = tr.irradiate(rho, td, energy=True)
    orc = _parity.oracle_for(w)
    mq, _ = _parity.masks(w, orc)
    q_ref = q_ref.double().cpu().numpy()
    a_ref = a_ref.double().cpu().numpy()
    q = torch.empty_like(rho)
    a = torch.empty_like(rho)

    # a first call on this grid loads every kernel the measured calls use
    st, _ = _static_call(torch, _lib, w, rho, td, q, a, code)
    assert st == _lib.RT_OK, _lib.last_error(None)

    # a larger grid with another bin count, a hotter star, tau550 = 100 and one NaN
    # density: the call must report the invalid input and leave its tables behind
    wb = synth.disk3d(nr + 64, 24, 8, n_nu=nnu + 11 if nnu < 100 else nnu - 11, tau550=100.0, seed=5)
    rb = wb.rho32().copy()
    rb.reshape(-1)[rb.size // 3] = np.nan
    rho_b = torch.from_numpy(rb).cuda()
    td_b = torch.from_numpy(wb.tdust32()).cuda()
    qb = torch.empty_like(rho_b)
    ab = torch.empty_like(rho_b)
    st, _ = _static_call(torch, _lib, wb, rho_b, td_b, qb, ab, code, t_star=9000.0)
    assert st == _lib.RT_ERR_NONFINITE_INPUT, (st, _lib.last_error(None))
    del rho_b, td_b, qb, ab

    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):
        q.fill_(float("nan"))
        a.fill_(float("nan"))
        torch.cuda.synchronize()
        st, e = _static_call(torch, _lib, w, rho, td, q, a, code)
        assert st == _lib.RT_OK, (call, _lib.last_error(None))
        qh = q.double().cpu().numpy()
        ah = a.double().cpu().numpy()
        assert np.all(np.isfinite(qh)) and np.all(np.isfinite(ah)), call
        # the tolerance of the parity tests, relative to the context-based result
        assert np.max(np.abs(qh[mq] - q_ref[mq]) / q_ref[mq]) <= _parity.RTOL_Q, call
        assert np.max(np.abs(ah[mq] - a_ref[mq]) / np.abs(a_ref[mq])) <= _parity.RTOL_A, call
        assert np.max(np.abs(qh - q_ref)) <= _parity.RTOL_Q * q_ref.max(), call
        assert abs(e.e_abs - e_ref.e_abs) <= _parity.RTOL_ENERGY * e_ref.l_star, call
        assert abs(e.e_esc - e_ref.e_esc) <= _parity.RTOL_ENERGY * e_ref.l_star, call
        assert abs(e.rel_err) <= _parity.RTOL_ENERGY, call
        assert abs(e.l_star / e_ref.l_star - 1) <= 1e-12, call
    # nothing was allocated on the device by the two calls
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_rejects_grids_beyond_its_limits(torch_cuda):
    torch = torch_cuda
    from paper_1001_3301_gb300 import _lib
    g = synth.log_grid(1025, 2, 1)  # nr one above the limit of 1024
    w = synth.Workload("big", g, synth.nu_bins(4), synth.kappa_synth(synth.nu_bins(4)),
                       np.zeros(g.shape), np.full(g.shape, 50.0))
    x = torch.zeros(g.shape, device="cuda")
    d, keep = _desc(_lib, g, _lib.RT_FP32_KAHAN)
    nu = np.ascontiguousarray(w.nu)
    kap = np.ascontiguousarray(w.kappa)
    P = ctypes.POINTER(ctypes.c_double)
    st = _lib.lib.rt_irradiate_static(ctypes.byref(d), w.t_star, w.r_star, len(nu),
                                      nu.ctypes.data_as(P), kap.ctypes.data_as(P), w.t_sub, 0,
                                      x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), None, None)
    assert st == _lib.RT_ERR_INVALID_ARG
    assert "static scratch" in _lib.last_error(None)
