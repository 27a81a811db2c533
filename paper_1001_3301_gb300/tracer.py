"""Python front end of the GB300 irradiation ray tracer.

A ``Tracer`` owns one library context (one grid). Device fields are torch CUDA
tensors; the work is enqueued on torch's current CUDA stream. PyTorch provides
device memory and streams only; the computation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _lib
from ._lib import (RT_SUR_NPARAMS, RtEnergy, RtFldStats, RtGridDesc, RtSurrogateStats, RtTrainCfg, RtTrainStats, check,
                   lib)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream_handle(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


class Energy:
    """Energy sums of one trace (erg/s): absorbed, escaped, emitted, and the
    relative mismatch (absorbed + escaped)/emitted - 1."""

    def __init__(self, e: RtEnergy):
        self.e_abs, self.e_esc, self.l_star, self.rel_err = e.e_abs, e.e_esc, e.l_star, e.rel_err

    def __repr__(self):
        return (f"Energy(e_abs={self.e_abs:.6e}, e_esc={self.e_esc:.6e}, "
                f"l_star={self.l_star:.6e}, rel_err={self.rel_err:.3e})")


class Tracer:
    """One spherical grid; see include/rt_irradiation.h for the semantics."""

    def __init__(self, r_if, theta_if, phi_if, precision: str | int = "fp32_kahan", stream=None):
        self.r_if, self.theta_if, self.phi_if = _f64(r_if), _f64(theta_if), _f64(phi_if)
        self.nr = len(self.r_if) - 1
        self.ntheta = len(self.theta_if) - 1
        self.nphi = len(self.phi_if) - 1
        self.shape = (self.nphi, self.ntheta, self.nr)
        self.precision = _lib.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        desc = RtGridDesc(self.nr, self.ntheta, self.nphi, _dptr(self.r_if), _dptr(self.theta_if),
                          _dptr(self.phi_if), self.precision)
        ctx = ctypes.c_void_p()
        check(lib.rt_create(ctypes.byref(desc), ctypes.c_void_p(_stream_handle(stream)),
                            ctypes.byref(ctx)), None)
        self._ctx = ctx
        self.n_nu = 0

    @classmethod
    def from_grid(cls, grid, precision="fp32_kahan", stream=None):
        return cls(grid.r_if, grid.theta_if, grid.phi_if, precision, stream)

    # -- configuration ---------------------------------------------------------
    def set_opacity_table(self, nu_mid, kappa, t_sub: float, kappa_bf16: bool = False):
        nu, kap = _f64(nu_mid), _f64(kappa)
        check(lib.rt_set_opacity_table(self._ctx, len(nu), _dptr(nu), _dptr(kap), float(t_sub),
                                       int(bool(kappa_bf16))), self._ctx)
        self.n_nu = len(nu)

    def set_opacity_table_t(self, nu_mid, t_grid, kappa_t, t_sub: float):
        """Temperature-dependent table: kappa_t [n_nu][n_t] on t_grid [n_t] (K)."""
        nu = _f64(nu_mid)
        tg = _f64(t_grid)
        kt = np.ascontiguousarray(kappa_t, dtype=np.float64)
        if kt.shape != (nu.size, tg.size):
            raise ValueError("kappa_t must be [n_nu][n_t]")
        check(lib.rt_set_opacity_table_t(self._ctx, nu.size, _dptr(nu), tg.size, _dptr(tg), _dptr(kt),
                                         float(t_sub)), self._ctx)
        self.n_nu = nu.size

    def set_star(self, t_star: float, r_star: float):
        check(lib.rt_set_star(self._ctx, float(t_star), float(r_star)), self._ctx)

    def set_stream(self, stream=None):
        check(lib.rt_set_stream(self._ctx, ctypes.c_void_p(_stream_handle(stream))), self._ctx)

    # -- tracing ---------------------------------------------------------------
    def _check_field(self, t, name):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and t.is_contiguous() and t.numel() == self.nr * self.ntheta * self.nphi):
            raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor of "
                             f"{self.shape} elements")

    def irradiate(self, rho, t_dust, q_abs=None, a_rad=None, energy: bool = False):
        """Trace every ray. Returns (q_abs, a_rad, Energy or None); outputs are
        allocated when not given."""
        import torch
        self._check_field(rho, "rho")
        self._check_field(t_dust, "t_dust")
        if q_abs is None:
            q_abs = torch.empty(self.shape, dtype=torch.float32, device=rho.device)
        if a_rad is None:
            a_rad = torch.empty(self.shape, dtype=torch.float32, device=rho.device)
        self._check_field(q_abs, "q_abs")
        self._check_field(a_rad, "a_rad")
        e = RtEnergy()
        check(lib.rt_irradiate(self._ctx, rho.data_ptr(), t_dust.data_ptr(), q_abs.data_ptr(),
                               a_rad.data_ptr(), ctypes.byref(e) if energy else None), self._ctx)
        return q_abs, a_rad, (Energy(e) if energy else None)

    def irradiate_host(self, rho, t_dust, q_abs, a_rad, energy: bool = False):
        """Host-buffer variant: rho, t_dust, q_abs, a_rad are C-contiguous float32
        numpy arrays or CPU torch tensors (page-locked for asynchronous copies)."""
        ptrs = []
        for x, name in ((rho, "rho"), (t_dust, "t_dust"), (q_abs, "q_abs"), (a_rad, "a_rad")):
            ptrs.append(_host_ptr(x, self.nr * self.ntheta * self.nphi, name))
        e = RtEnergy()
        check(lib.rt_irradiate_host(self._ctx, *ptrs, ctypes.byref(e) if energy else None), self._ctx)
        return Energy(e) if energy else None

    def irradiate_host_async(self, rho, t_dust, q_abs, a_rad):
        """Host-buffer variant that returns once the copies and the trace are enqueued;
        keep the buffers alive and untouched until host_wait()."""
        ptrs = []
        for x, name in ((rho, "rho"), (t_dust, "t_dust"), (q_abs, "q_abs"), (a_rad, "a_rad")):
            ptrs.append(_host_ptr(x, self.nr * self.ntheta * self.nphi, name))
        check(lib.rt_irradiate_host_async(self._ctx, *ptrs), self._ctx)

    def host_wait(self):
        """Wait for the last irradiate_host_async's outputs (raises on invalid input)."""
        check(lib.rt_host_wait(self._ctx), self._ctx)

    def energy_last(self) -> Energy:
        e = RtEnergy()
        check(lib.rt_energy_last(self._ctx, ctypes.byref(e)), self._ctx)
        return Energy(e)

    def lut_build(self, err_tol: float = 1e-3):
        """Build the lookup-table comparator of the per-bin sum (rt_lut_build)."""
        check(lib.rt_lut_build(self._ctx, float(err_tol)), self._ctx)

    def irradiate_lut(self, rho, t_dust, q_abs=None, a_rad=None, energy: bool = False, stats: bool = False):
        """Trace with the per-bin sum from the lookup table. Returns (q_abs, a_rad,
        Energy or None, warp-slots that fell back to the per-bin sum or None)."""
        import torch
        self._check_field(rho, "rho")
        self._check_field(t_dust, "t_dust")
        if q_abs is None:
            q_abs = torch.empty(self.shape, dtype=torch.float32, device=rho.device)
        if a_rad is None:
            a_rad = torch.empty(self.shape, dtype=torch.float32, device=rho.device)
        self._check_field(q_abs, "q_abs")
        self._check_field(a_rad, "a_rad")
        e = RtEnergy()
        fb = ctypes.c_uint()
        check(lib.rt_irradiate_lut(self._ctx, rho.data_ptr(), t_dust.data_ptr(), q_abs.data_ptr(), a_rad.data_ptr(),
                                   ctypes.byref(e) if energy else None, ctypes.byref(fb) if stats else None),
              self._ctx)
        return q_abs, a_rad, (Energy(e) if energy else None), (fb.value if stats else None)

    def table_kind(self) -> int:
        """RT_TABLE_NU, RT_TABLE_NU_T_SEPARABLE, RT_TABLE_NU_T_RANK2, RT_TABLE_NU_T_LOW_RANK or RT_TABLE_NU_T: how the table is traced."""
        k = ctypes.c_int()
        check(lib.rt_opacity_table_kind(self._ctx, ctypes.byref(k)), self._ctx)
        return k.value

    def energy_reduce(self):
        """Enqueue the FP64 energy reduction of the last trace (device only, no sync)."""
        check(lib.rt_energy_reduce(self._ctx), self._ctx)

    def bins(self) -> np.ndarray:
        out = np.empty(self.n_nu, dtype=np.float64)
        check(lib.rt_get_bins(self._ctx, _dptr(out)), self._ctx)
        return out

    # -- launch shape ----------------------------------------------------------
    def set_tuning(self, kind: int = 0, cells_per_lane: int = 0, warps: int = 0, min_blocks: int = 0):
        """Force (kernel kind, cells per lane, warps per CTA, min resident CTAs per SM);
        all zero restores the automatic choice."""
        check(lib.rt_set_tuning(self._ctx, int(kind), int(cells_per_lane), int(warps), int(min_blocks)),
              self._ctx)

    def tuning(self):
        """(kernel kind, cells per lane, warps per CTA, min resident CTAs per SM) in use."""
        v = [ctypes.c_int() for _ in range(4)]
        check(lib.rt_get_tuning(self._ctx, *[ctypes.byref(x) for x in v]), self._ctx)
        return tuple(x.value for x in v)

    def tunings(self):
        """Every compiled launch shape that applies to this grid and precision."""
        n = 64
        arrs = [(ctypes.c_int * n)() for _ in range(4)]
        m = lib.rt_list_tunings(self._ctx, *arrs, n)
        if m < 0:
            check(m, self._ctx)
        return [tuple(a[i] for a in arrs) for i in range(min(m, n))]

    def autotune(self, rho, t_dust, q_abs, a_rad, reps: int = 3):
        check(lib.rt_autotune(self._ctx, rho.data_ptr(), t_dust.data_ptr(), q_abs.data_ptr(),
                              a_rad.data_ptr(), int(reps)), self._ctx)
        return self.tuning()

    # -- Planck mean and dust temperature (Eq. 16) -------------------------------
    def planck_mean_opacity(self, t: float) -> float:
        """kappa_P(T) of the configured table (cm^2/g)."""
        k = ctypes.c_double()
        check(lib.rt_planck_mean_opacity(self._ctx, float(t), ctypes.byref(k)), self._ctx)
        return k.value

    def dust_temperature(self, a_rad, e_rad=None, t_dust=None):
        """Dust temperature from a T^4 = E_R + a_rad / kappa_P(T) (CUDA tensors)."""
        import torch
        self._check_field(a_rad, "a_rad")
        if e_rad is not None:
            self._check_field(e_rad, "e_rad")
        if t_dust is None:
            t_dust = torch.empty(self.shape, dtype=torch.float32, device=a_rad.device)
        self._check_field(t_dust, "t_dust")
        check(lib.rt_dust_temperature(self._ctx, a_rad.data_ptr(), None if e_rad is None else e_rad.data_ptr(),
                                      t_dust.data_ptr()), self._ctx)
        return t_dust

    # -- flux-limited diffusion (Eqs. 7-15) ----------------------------------------
    def rosseland_mean_opacity(self, t: float) -> float:
        """kappa_R(T) of the configured table (cm^2/g)."""
        k = ctypes.c_double()
        check(lib.rt_rosseland_mean_opacity(self._ctx, float(t), ctypes.byref(k)), self._ctx)
        return k.value

    def fld_step(self, rho, t_gas, q_abs, e_old, dt, c_v, t_bg, e_new=None, tol=1e-5, max_iter=20000):
        """One implicit flux-limited-diffusion step of E_R (CUDA tensors of this grid);
        returns (e_new, {"iterations", "passes", "rel_change", "levels"})."""
        import torch
        for f, name in ((rho, "rho"), (t_gas, "t_gas"), (q_abs, "q_abs"), (e_old, "e_old")):
            self._check_field(f, name)
        if e_new is None:
            e_new = torch.empty(self.shape, dtype=torch.float32, device=e_old.device)
        self._check_field(e_new, "e_new")
        st = RtFldStats()
        check(lib.rt_fld_step(self._ctx, rho.data_ptr(), t_gas.data_ptr(), q_abs.data_ptr(), e_old.data_ptr(),
                              e_new.data_ptr(), float(dt), float(c_v), float(t_bg), float(tol), int(max_iter),
                              ctypes.byref(st)), self._ctx)
        return e_new, {"iterations": st.iterations, "passes": st.passes, "rel_change": st.rel_change,
                       "levels": st.levels}

    # -- learned surrogate (rt_surrogate_*) -------------------------------------
    def surrogate_train(self, rho_list, t_list, n_samples=0, batch=0, steps=0, lr=0.0, seed=1):
        """Train the context's surrogate on the given fields (CUDA tensors of this
        grid); returns the training statistics as a dict."""
        for t in list(rho_list) + list(t_list):
            self._check_field(t, "training field")
        n = len(rho_list)
        if n != len(t_list) or n < 1:
            raise ValueError("rho_list and t_list must have the same non-zero length")
        rp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in rho_list])
        tp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in t_list])
        cfg = RtTrainCfg(int(n_samples), int(batch), int(steps), float(lr), int(seed))
        st = RtTrainStats()
        check(lib.rt_surrogate_train(self._ctx, ctypes.byref(cfg), rp, tp, n, ctypes.byref(st)), self._ctx)
        return {k: getattr(st, k) for k, _ in RtTrainStats._fields_}

    def irradiate_surrogate(self, rho, t_dust, q_abs=None, a_rad=None, err_tol=1e-3, validate=0, stats=True):
        """(q_abs, a_rad, stats dict or None) with the surrogate in place of the per-bin
        sum; validate: 0 trust-map gate, 1 judged by the exact tracer, 2 network only.
        stats=False leaves the call asynchronous."""
        import torch
        self._check_field(rho, "rho")
        self._check_field(t_dust, "t_dust")
        if q_abs is None:
            q_abs = torch.empty(self.shape, dtype=torch.float32, device=rho.device)
        if a_rad is None:
            a_rad = torch.empty(self.shape, dtype=torch.float32, device=rho.device)
        self._check_field(q_abs, "q_abs")
        self._check_field(a_rad, "a_rad")
        st = RtSurrogateStats()
        check(lib.rt_irradiate_surrogate(self._ctx, rho.data_ptr(), t_dust.data_ptr(), q_abs.data_ptr(),
                                         a_rad.data_ptr(), float(err_tol), int(validate),
                                         ctypes.byref(st) if stats else None), self._ctx)
        return q_abs, a_rad, ({k: getattr(st, k) for k, _ in RtSurrogateStats._fields_} if stats else None)

    def surrogate_set_params(self, params, mu, sigma):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != RT_SUR_NPARAMS:
            raise ValueError(f"expected {RT_SUR_NPARAMS} parameters")
        check(lib.rt_surrogate_set_params(self._ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          float(mu), float(sigma)), self._ctx)

    def surrogate_params(self):
        """(params [RT_SUR_NPARAMS] float32, mu, sigma)"""
        p = np.empty(RT_SUR_NPARAMS, dtype=np.float32)
        mu, sg = ctypes.c_double(), ctypes.c_double()
        check(lib.rt_surrogate_get_params(self._ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          ctypes.byref(mu), ctypes.byref(sg)), self._ctx)
        return p, mu.value, sg.value

    def surrogate_grad(self, x, t):
        """(loss, grad [RT_SUR_NPARAMS]) of mean((y - t)^2) by the training kernels."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        n = t.size
        if x.shape != (n, 8):
            raise ValueError("x must be [n][8]")
        g = np.empty(RT_SUR_NPARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        fp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        check(lib.rt_surrogate_grad(self._ctx, fp(x), fp(t), n, fp(g), ctypes.byref(loss)), self._ctx)
        return loss.value, g

    def surrogate_eval(self, x):
        """Standardised network outputs for feature rows x [n][8] (inference kernel)."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        n = x.shape[0]
        y = np.empty(n, dtype=np.float32)
        fp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        check(lib.rt_surrogate_eval(self._ctx, fp(x), n, fp(y)), self._ctx)
        return y

    def surrogate_loss_history(self):
        n = lib.rt_surrogate_loss_history(self._ctx, None, 0)
        if n < 0:
            check(n, self._ctx)
        out = np.empty(n, dtype=np.float32)
        lib.rt_surrogate_loss_history(self._ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n)
        return out

    def surrogate_trust_map(self, err_tol=1e-3):
        """(bits as a [64][64] bool array indexed [iu][iv], (u0, du, v0, dv))"""
        bits = (ctypes.c_uint * 128)()
        rng = (ctypes.c_float * 4)()
        check(lib.rt_surrogate_trust_map(self._ctx, float(err_tol), bits, rng), self._ctx)
        w = np.array(bits[:], dtype=np.uint32)
        b = np.array([(w[i >> 5] >> (i & 31)) & 1 for i in range(64 * 64)], dtype=bool).reshape(64, 64)
        return b, tuple(rng[:])

    def surrogate_save(self, path):
        check(lib.rt_surrogate_save(self._ctx, os.fsencode(path)), self._ctx)

    def surrogate_load(self, path):
        check(lib.rt_surrogate_load(self._ctx, os.fsencode(path)), self._ctx)

    # -- lifetime --------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            lib.rt_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _host_ptr(x, n, name):
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"] or x.size != n:
            raise ValueError(f"{name}: expected a C-contiguous float32 array of {n} elements")
        return x.ctypes.data
    import torch
    if isinstance(x, torch.Tensor):
        if x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous() or x.numel() != n:
            raise ValueError(f"{name}: expected a contiguous float32 CPU tensor of {n} elements")
        return x.data_ptr()
    raise TypeError(f"{name}: numpy array or CPU tensor expected")


def probe_ex2(x):
    """2^x on the device with the FP32 tracer's hardware exp2 (torch CUDA tensor in/out)."""
    import torch
    y = torch.empty_like(x)
    check(lib.rt_probe_ex2(x.data_ptr(), y.data_ptr(), x.numel(),
                           ctypes.c_void_p(_stream_handle())))
    return y


def probe_alu_rates():
    """(ex2 per SM per clock, FFMA per SM per clock, SM MHz) measured on the device."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(lib.rt_probe_alu_rates(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def probe_tanh(x, packed_bf16=False):
    """tanh(x) with the hardware approximation of the surrogate's activations."""
    import torch
    y = torch.empty_like(x)
    check(lib.rt_probe_tanh(x.data_ptr(), y.data_ptr(), x.numel(), int(bool(packed_bf16)),
                            ctypes.c_void_p(_stream_handle())))
    return y


def probe_umma(a_bits, b_bits):
    """D = A B^T (128 x 128) on the tcgen05 tensor core; a_bits, b_bits: int16 CUDA
    tensors [128][k] holding BF16 bit patterns."""
    import torch
    k = a_bits.shape[1]
    d = torch.empty((128, 128), dtype=torch.float32, device=a_bits.device)
    check(lib.rt_probe_umma(a_bits.data_ptr(), b_bits.data_ptr(), k, d.data_ptr(),
                            ctypes.c_void_p(_stream_handle())))
    return d


def probe_tensor_rates():
    """Per SM per clock: mma.sync MACs, tcgen05 MACs at N = 128 and 256, tanh.approx
    f32 and packed-bf16 instructions, rcp.approx f32 instructions."""
    v = [ctypes.c_double() for _ in range(6)]
    check(lib.rt_probe_tensor_rates(*[ctypes.byref(x) for x in v]))
    return dict(zip(("mma_sync_mac", "umma_n128_mac", "umma_n256_mac", "tanh_f32", "tanh_bf16x2", "rcp_f32"),
                    (x.value for x in v)))


class Batch:
    """Several configured tracers traced by one persistent launch replayed from a
    CUDA graph (include/rt_irradiation.h, rt_batch_*). The tracers must outlive
    the batch and keep their configuration."""

    def __init__(self, tracers, stream=None):
        n = len(tracers)
        arr = (ctypes.c_void_p * n)(*[t._ctx.value for t in tracers])
        b = ctypes.c_void_p()
        check(lib.rt_batch_create(arr, n, ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(b)), None)
        self._b = b
        self.tracers = list(tracers)
        self.n = n

    def _ptrs(self, tensors, name):
        if len(tensors) != self.n:
            raise ValueError(f"{name}: expected {self.n} tensors")
        for t, tr in zip(tensors, self.tracers):
            tr._check_field(t, name)
        return (ctypes.c_void_p * self.n)(*[t.data_ptr() for t in tensors])

    def _check(self, status):
        if status != _lib.RT_OK:
            raise _lib.RtError(status, lib.rt_batch_last_error(self._b).decode())

    def run(self, rho, t_dust, q_abs, a_rad):
        """Trace every grid: lists of device tensors, one per tracer."""
        self._check(lib.rt_batch_run(self._b, self._ptrs(rho, "rho"), self._ptrs(t_dust, "t_dust"),
                                     self._ptrs(q_abs, "q_abs"), self._ptrs(a_rad, "a_rad")))

    def energy(self):
        out = (RtEnergy * self.n)()
        self._check(lib.rt_batch_energy(self._b, out))
        return [Energy(e) for e in out]

    def autotune(self, rho, t_dust, q_abs, a_rad, reps: int = 3):
        self._check(lib.rt_batch_autotune(self._b, self._ptrs(rho, "rho"), self._ptrs(t_dust, "t_dust"),
                                          self._ptrs(q_abs, "q_abs"), self._ptrs(a_rad, "a_rad"), int(reps)))
        return self.tuning()

    def set_tuning(self, kind: int, cells_per_lane: int, warps: int, min_blocks: int = 0):
        """Select a compiled batch shape (kind 0 = tiles, 1 = warp per ray) and rebuild the graph."""
        self._check(lib.rt_batch_set_tuning(self._b, int(kind), int(cells_per_lane), int(warps), int(min_blocks)))
        return self.tuning()

    def tuning(self):
        v = [ctypes.c_int() for _ in range(4)]
        self._check(lib.rt_batch_get_tuning(self._b, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def close(self):
        if getattr(self, "_b", None):
            lib.rt_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
