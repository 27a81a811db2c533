"""rt_irradiate_static, the allocation-free entry point, against rt_irradiate.

It exists for callers that cannot allocate device memory when they need the
irradiation (a host code whose pool already holds the GPU memory, or a time
loop where cudaMalloc/cudaFree would synchronise the device). It keeps all its
scratch in one static device array, so these checks call it through the C ABI
twice in a row (the second call reuses, and must not be disturbed by, what the
first left in the array) and compare both results with the context-based entry
point on the same inputs. The file name sorts last so that a run stopping at the
first failure has already run every other test; it also passes on its own in a
fresh process.
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


def _static_call(torch, lib_mod, w, rho, td, precision):
    q = torch.full_like(rho, float("nan"))
    a = torch.full_like(rho, float("nan"))
    d, keep = _desc(lib_mod, w.grid, precision)
    nu = np.ascontiguousarray(w.nu, dtype=np.float64)
    kap = np.ascontiguousarray(w.kappa, dtype=np.float64)
    P = ctypes.POINTER(ctypes.c_double)
    e = lib_mod.RtEnergy()
    st = lib_mod.lib.rt_irradiate_static(
        ctypes.byref(d), w.t_star, w.r_star, len(nu), nu.ctypes.data_as(P), kap.ctypes.data_as(P),
        w.t_sub, 0, rho.data_ptr(), td.data_ptr(), q.data_ptr(), a.data_ptr(), ctypes.byref(e),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == lib_mod.RT_OK, lib_mod.last_error(None)
    torch.cuda.synchronize()
    return q, a, e


@pytest.mark.parametrize("dims", [(256, 32, 16, 79), (65, 9, 4, 17)], ids=["ray-kernel", "tile-kernel"])
def test_static_matches_context_entry_point_twice(torch_cuda, dims):
    torch = torch_cuda
    from paper_1001_3301_gb300 import Tracer, _lib
    nr, nth, nph, nnu = dims
    w = synth.disk3d(nr, nth, nph, n_nu=nnu, tau550=10.0, seed=nr)
    rho = torch.from_numpy(w.rho32()).cuda()
    td = torch.from_numpy(w.tdust32()).cuda()
    with Tracer.from_grid(w.grid) as tr:
        tr.set_opacity_table(w.nu, w.kappa, w.t_sub)
        tr.set_star(w.t_star, w.r_star)
        q_ref, a_ref, e_ref = tr.irradiate(rho, td, energy=True)
    orc = _parity.oracle_for(w)
    mq, _ = _parity.masks(w, orc)
    q_ref = q_ref.double().cpu().numpy()
    a_ref = a_ref.double().cpu().numpy()
    for call in range(2):
        q, a, e = _static_call(torch, _lib, w, rho, td, _lib.RT_FP32_KAHAN)
        q = q.double().cpu().numpy()
        a = a.double().cpu().numpy()
        assert np.all(np.isfinite(q)) and np.all(np.isfinite(a)), call
        # the tolerance of the parity tests, relative to the context-based result
        assert np.max(np.abs(q[mq] - q_ref[mq]) / q_ref[mq]) <= _parity.RTOL_Q, call
        assert np.max(np.abs(a[mq] - a_ref[mq]) / np.abs(a_ref[mq])) <= _parity.RTOL_A, call
        assert np.max(np.abs(q - q_ref)) <= _parity.RTOL_Q * q_ref.max(), call
        assert abs(e.e_abs - e_ref.e_abs) <= _parity.RTOL_ENERGY * e_ref.l_star, call
        assert abs(e.e_esc - e_ref.e_esc) <= _parity.RTOL_ENERGY * e_ref.l_star, call
        assert abs(e.rel_err) <= _parity.RTOL_ENERGY, call


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
