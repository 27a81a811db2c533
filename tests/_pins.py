"""Independent references that pin the oracle: numerical quadrature (scipy),
textbook constants and the paper's printed numbers. Nothing here calls the
oracle's own Planck series or ray loop."""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import integrate

# CODATA 2018 (exact SI definitions and the printed derived constants), cgs
C = 2.99792458e10
H = 6.62607015e-27
K_B = 1.380649e-16
SIGMA_PRINTED = 5.670374419e-5       # erg cm^-2 s^-1 K^-4 (CODATA 2018, rounded)
A_RAD_PRINTED = 7.565733250e-15      # erg cm^-3 K^-4   (radiation density constant)


def pi_bnu(nu, t):
    """pi B_nu(T): surface flux density of a black body, erg s^-1 cm^-2 Hz^-1."""
    x = H * nu / (K_B * t)
    if x > 700.0:
        return 0.0
    return math.pi * 2.0 * H * nu ** 3 / (C * C) / math.expm1(x)


def bin_flux_quad(t, lo, hi):
    """int_lo^hi pi B_nu dnu by adaptive quadrature in ln(nu)."""
    lo = max(lo, 1.0)
    hi = min(hi, 1e3 * K_B * t / H)
    if hi <= lo:
        return 0.0
    f = lambda u: pi_bnu(math.exp(u), t) * math.exp(u)
    a, b = math.log(lo), math.log(hi)
    # split at the peak region so quad sees the structure
    knots = [a] + [u for u in np.linspace(a, b, 9)[1:-1]] + [b]
    total = 0.0
    for u0, u1 in zip(knots[:-1], knots[1:]):
        with warnings.catch_warnings():
            # quad reports "bad integrand behaviour" where the Wien tail underflows
            warnings.simplefilter("ignore", integrate.IntegrationWarning)
            val, _ = integrate.quad(f, u0, u1, epsabs=0.0, epsrel=1e-13, limit=400)
        total += val
    return total


def bin_edges(nu_mid):
    nu = np.asarray(nu_mid, dtype=np.float64)
    lo = np.concatenate([[0.0], 0.5 * (nu[:-1] + nu[1:])])
    hi = np.concatenate([0.5 * (nu[:-1] + nu[1:]), [np.inf]])
    return lo, hi


def bin_fluxes_quad(t, nu_mid):
    lo, hi = bin_edges(nu_mid)
    return np.array([bin_flux_quad(t, a, b) for a, b in zip(lo, hi)])


def solid_angles(theta_if, phi_if):
    """dOmega per ray in the [nphi][ntheta] layout."""
    dcos = np.cos(theta_if[:-1]) - np.cos(theta_if[1:])
    dphi = np.diff(phi_if)
    return dphi[:, None] * dcos[None, :]


def shell_volumes(r_if):
    """(r+^3 - r-^3)/3 per radial cell (multiply by dOmega for the cell volume)."""
    return (r_if[1:] ** 3 - r_if[:-1] ** 3) / 3.0


def brute_force_cells(r_if, theta_if, phi_if, t_star, r_star, nu_mid, kappa, t_sub,
                      rho, tdust, f_bin=None):
    """Absorbed power P and force numerator per cell by quadrature of Eq. 27/28:
    P = dOmega int kappa rho F(r) r^2 dr, F(r) = sum_i F_i (R*/r)^2 exp(-tau_i(r)),
    tau_i(r) the integral of the piecewise-constant kappa rho from r_min (Eq. 19).
    Returns (P, A) with A = dOmega int kappa F(r) r^2 dr (so a_rad = A/(V c))."""
    nr = len(r_if) - 1
    nth, nph = len(theta_if) - 1, len(phi_if) - 1
    if f_bin is None:
        f_bin = bin_fluxes_quad(t_star, nu_mid)
    dom = solid_angles(theta_if, phi_if)
    P = np.zeros((nph, nth, nr))
    A = np.zeros((nph, nth, nr))
    for ip in range(nph):
        for it in range(nth):
            for i, (fi, ki) in enumerate(zip(f_bin, kappa)):
                tau_left = 0.0
                for k in range(nr):
                    kap = ki if tdust[ip, it, k] <= t_sub else 0.0
                    kr = kap * rho[ip, it, k]
                    r0, r1 = r_if[k], r_if[k + 1]
                    # r^2 F(r) = F_i R*^2 exp(-(tau_left + kr (r - r0)))
                    g = lambda r: math.exp(-(tau_left + kr * (r - r0)))
                    val, _ = integrate.quad(g, r0, r1, epsabs=0.0, epsrel=1e-13, limit=200)
                    P[ip, it, k] += dom[ip, it] * fi * r_star ** 2 * kr * val
                    A[ip, it, k] += dom[ip, it] * fi * r_star ** 2 * kap * val
                    tau_left += kr * (r1 - r0)
    return P, A
