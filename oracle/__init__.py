"""ctypes front end of the FP64 CPU oracle (``rt_oracle.c``).

TEST INFRASTRUCTURE: only the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package. The CUDA library and its Python
binding never import it.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "librt_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available); returns the .so path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    lib.rto_sigma_sb.restype = ctypes.c_double
    lib.rto_planck_H_small.restype = ctypes.c_double
    lib.rto_planck_H_small.argtypes = [ctypes.c_double]
    lib.rto_planck_G_large.restype = ctypes.c_double
    lib.rto_planck_G_large.argtypes = [ctypes.c_double]
    lib.rto_planck_band.restype = ctypes.c_double
    lib.rto_planck_band.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.rto_irradiate_tdep.restype = ctypes.c_int
    lib.rto_irradiate_tdep.argtypes = ([ctypes.c_int] * 3 + [_D] * 3 + [ctypes.c_double] * 2 +
                                       [ctypes.c_int, _D, ctypes.c_int, _D, _D, ctypes.c_double] + [_D] * 8 +
                                       [ctypes.c_int])
    lib.rto_rosseland_mean.restype = ctypes.c_double
    lib.rto_rosseland_mean.argtypes = [ctypes.c_double, ctypes.c_int, _D, _D]
    lib.rto_planck_mean.restype = ctypes.c_double
    lib.rto_planck_mean.argtypes = [ctypes.c_double, ctypes.c_int, _D, _D]
    lib.rto_dust_temperature.restype = ctypes.c_int
    lib.rto_dust_temperature.argtypes = [ctypes.c_longlong, _D, _D, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, _D, _D, _D, ctypes.c_int]
    lib.rto_planck_bins.restype = ctypes.c_int
    lib.rto_planck_bins.argtypes = [ctypes.c_double, ctypes.c_int, _D, _D]
    lib.rto_irradiate.restype = ctypes.c_int
    lib.rto_irradiate.argtypes = ([ctypes.c_int] * 3 + [_D] * 3 + [ctypes.c_double] * 2 +
                                  [ctypes.c_int, _D, _D, ctypes.c_double] + [_D] * 8 +
                                  [ctypes.c_int])
    lib.rto_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every oracle call through another build of ``rt_oracle.c``
    (the mutation tests load deliberately broken copies this way)."""
    global _lib
    saved = _load()
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def sigma_sb() -> float:
    return _load().rto_sigma_sb()


def planck_H(x: float) -> float:
    return _load().rto_planck_H_small(float(x))


def planck_G(x: float) -> float:
    return _load().rto_planck_G_large(float(x))


def planck_band(a: float, b: float) -> float:
    return _load().rto_planck_band(float(a), float(b))


def planck_bins(t_star: float, nu_mid) -> np.ndarray:
    """Per-bin stellar surface flux F_i (erg s^-1 cm^-2), Eq. 20."""
    nu = _f64(nu_mid)
    out = np.empty(len(nu), dtype=np.float64)
    if _load().rto_planck_bins(float(t_star), len(nu), _ptr(nu), _ptr(out)) != 0:
        raise ValueError("rto_planck_bins: bad argument")
    return out


def planck_mean(t: float, nu_mid, kappa) -> float:
    """kappa_P(T) of a bin table: sum kappa_i B_i(T) / sum B_i(T) (Eq. 16's mean)."""
    nu, k = _f64(nu_mid), _f64(kappa)
    v = _load().rto_planck_mean(float(t), len(nu), _ptr(nu), _ptr(k))
    if v < 0:
        raise ValueError("rto_planck_mean: bad argument")
    return v


def rosseland_mean(t: float, nu_mid, kappa) -> float:
    """kappa_R(T) of a bin table: sum W_i / sum (W_i / kappa_i), W_i = int dB/dT over bin i."""
    nu, k = _f64(nu_mid), _f64(kappa)
    v = _load().rto_rosseland_mean(float(t), len(nu), _ptr(nu), _ptr(k))
    if v < 0:
        raise ValueError("rto_rosseland_mean: bad argument")
    return v


def dust_temperature(a_rad, e_rad, nu_mid, kappa, t_lo=1.0, t_hi=1e5, nthreads=0) -> np.ndarray:
    """T per cell from a T^4 = E_R + a_rad / kappa_P(T) (Eq. 16, frequency-dependent
    fluxes), kappa_P held constant outside [t_lo, t_hi]; bisection in FP64."""
    ar = _f64(a_rad).ravel()
    er = None if e_rad is None else _f64(e_rad).ravel()
    nu, k = _f64(nu_mid), _f64(kappa)
    out = np.empty_like(ar)
    if _load().rto_dust_temperature(ar.size, _ptr(ar), _ptr(er), float(t_lo), float(t_hi), len(nu), _ptr(nu),
                                    _ptr(k), _ptr(out), int(nthreads or max_threads())) != 0:
        raise ValueError("rto_dust_temperature: bad argument")
    return out.reshape(np.shape(a_rad))


def max_threads() -> int:
    return _load().rto_max_threads()


class Result:
    """Oracle outputs; fields are float64 arrays in the [nphi][ntheta][nr] layout."""

    def __init__(self, q_abs, a_rad, p_abs, flux_if, p_esc, energy):
        self.q_abs = q_abs
        self.a_rad = a_rad
        self.p_abs = p_abs
        self.flux_if = flux_if
        self.p_esc = p_esc
        self.e_abs, self.e_esc, self.l_star, self.rel_err = (float(x) for x in energy)


def irradiate(r_if, theta_if, phi_if, t_star, r_star, nu_mid, kappa, t_sub, rho, tdust,
              want_flux: bool = False, nthreads: int = 1) -> Result:
    """Run the oracle on one grid. ``rho``/``tdust`` of shape [nphi][ntheta][nr]."""
    r_if, theta_if, phi_if = _f64(r_if), _f64(theta_if), _f64(phi_if)
    nu, kap = _f64(nu_mid), _f64(kappa)
    nr, nth, nph = len(r_if) - 1, len(theta_if) - 1, len(phi_if) - 1
    rho = _f64(rho).reshape(nph, nth, nr)
    tdust = _f64(tdust).reshape(nph, nth, nr)
    q = np.empty_like(rho)
    a = np.empty_like(rho)
    p = np.empty_like(rho)
    fl = np.empty((nph, nth, nr + 1)) if want_flux else None
    pe = np.empty((nph, nth))
    en = np.empty(4)
    rc = _load().rto_irradiate(nr, nth, nph, _ptr(r_if), _ptr(theta_if), _ptr(phi_if),
                               float(t_star), float(r_star), len(nu), _ptr(nu), _ptr(kap),
                               float(t_sub), _ptr(rho), _ptr(tdust), _ptr(q), _ptr(a), _ptr(p),
                               _ptr(fl), _ptr(pe), _ptr(en), int(nthreads))
    if rc != 0:
        raise ValueError("rto_irradiate: bad argument")
    return Result(q, a, p, fl, pe, en)


def irradiate_tdep(r_if, theta_if, phi_if, t_star, r_star, nu_mid, t_grid, kappa_t, t_sub, rho, tdust,
                   nthreads: int = 1) -> Result:
    """The oracle with temperature-dependent opacities kappa_t [n_nu][n_t] on t_grid."""
    r_if, theta_if, phi_if = _f64(r_if), _f64(theta_if), _f64(phi_if)
    nu, tg = _f64(nu_mid), _f64(t_grid)
    kt = np.ascontiguousarray(kappa_t, dtype=np.float64)
    assert kt.shape == (len(nu), len(tg))
    nr, nth, nph = len(r_if) - 1, len(theta_if) - 1, len(phi_if) - 1
    rho = _f64(rho).reshape(nph, nth, nr)
    tdust = _f64(tdust).reshape(nph, nth, nr)
    q = np.empty_like(rho)
    a = np.empty_like(rho)
    p = np.empty_like(rho)
    pe = np.empty((nph, nth))
    en = np.empty(4)
    rc = _load().rto_irradiate_tdep(nr, nth, nph, _ptr(r_if), _ptr(theta_if), _ptr(phi_if), float(t_star),
                                    float(r_star), len(nu), _ptr(nu), len(tg), _ptr(tg), _ptr(kt), float(t_sub),
                                    _ptr(rho), _ptr(tdust), _ptr(q), _ptr(a), _ptr(p), None, _ptr(pe), _ptr(en),
                                    int(nthreads))
    if rc != 0:
        raise ValueError("rto_irradiate_tdep: bad argument")
    return Result(q, a, p, None, pe, en)


def irradiate_workload(w, rho=None, tdust=None, kappa=None, want_flux=False, nthreads=1) -> Result:
    """Oracle on a ``synth.Workload``; by default on its FP32-rounded fields (what the
    GPU reads)."""
    g = w.grid
    return irradiate(g.r_if, g.theta_if, g.phi_if, w.t_star, w.r_star, w.nu,
                     w.kappa if kappa is None else kappa, w.t_sub,
                     w.rho32().astype(np.float64) if rho is None else rho,
                     w.tdust32().astype(np.float64) if tdust is None else tdust,
                     want_flux=want_flux, nthreads=nthreads)
