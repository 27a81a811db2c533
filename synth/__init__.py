"""Seeded synthetic workloads for the stellar-irradiation ray tracer.

This module builds *inputs only*: spherical grids, the flared-disk density of the
irradiated-disk benchmark (Sect. 3.1.1), dust temperatures and a synthetic
frequency-dependent opacity table. It contains none of the ray tracer's
arithmetic; both the FP64 CPU oracle and the CUDA library consume the arrays it
returns, unchanged.

Every random draw comes from a counter-based generator (SplitMix64's output
mixer applied to a per-cell counter), so any host regenerates any cell of any
workload from (seed, stream, cell index) alone, in any order.

Units are cgs throughout (cm, g, s, K, Hz), as in the paper.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

AU_CM = 1.495978707e13          # IAU 2012 astronomical unit
R_SUN_CM = 6.957e10             # IAU 2015 nominal solar radius
M_SUN_G = 1.98841e33            # solar mass (CODATA/IAU G*M / G)
C_CM_S = 2.99792458e10          # speed of light (exact)

# Benchmark star and disk (Sect. 3.1.1)
T_STAR_K = 5800.0
R_STAR_CM = R_SUN_CM
R_MIN_AU, R_MAX_AU = 1.0, 1000.0
R_D_AU = R_MAX_AU / 2.0          # r_d = r_max / 2
Z_D_AU = R_MAX_AU / 8.0          # z_d = r_max / 8
DENSITY_FLOOR_REL = 1e-100       # lowest density relative to the highest one
NU_550NM_HZ = C_CM_S / 550e-7    # visual reference frequency
T_SUB_K = 1500.0                 # dust sublimation temperature used by the workloads

# frequency grid: log-spaced mid-frequencies with inclusive end points
NU_LO_HZ, NU_HI_HZ = 1e11, 1e16


# ----------------------------------------------------------------------------
# counter-based random numbers
# ----------------------------------------------------------------------------
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_STREAM = np.uint64(0xD1B54A32D192ED03)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (Steele, Lea & Flood 2014)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


def hash_u01(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in (0, 1] from (seed, stream, counter); any order, any host."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = (np.uint64(seed) * _GOLDEN + np.uint64(stream) * _STREAM) & _M64
        z = _mix64(idx * _GOLDEN + base)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def hash_normal(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Standard normal deviates via Box-Muller on two hashed uniforms."""
    u1 = hash_u01(seed, 2 * stream, idx)
    u2 = hash_u01(seed, 2 * stream + 1, idx)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# grids
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Grid:
    """Spherical grid given by its cell interfaces (cm, rad)."""
    r_if: np.ndarray      # [nr+1], increasing, r_if[0] > 0
    theta_if: np.ndarray  # [ntheta+1] in [0, pi]
    phi_if: np.ndarray    # [nphi+1]; nphi == 1 spans 2 pi (axisymmetric)

    @property
    def nr(self) -> int:
        return len(self.r_if) - 1

    @property
    def ntheta(self) -> int:
        return len(self.theta_if) - 1

    @property
    def nphi(self) -> int:
        return len(self.phi_if) - 1

    @property
    def shape(self) -> tuple:
        """Field layout [nphi][ntheta][nr], r fastest."""
        return (self.nphi, self.ntheta, self.nr)

    @property
    def ncells(self) -> int:
        return self.nr * self.ntheta * self.nphi

    def centres(self):
        """Cell-centre coordinates (r_c, theta_c) as arithmetic midpoints."""
        r_c = 0.5 * (self.r_if[:-1] + self.r_if[1:])
        th_c = 0.5 * (self.theta_if[:-1] + self.theta_if[1:])
        return r_c, th_c


def log_grid(nr: int, ntheta: int, nphi: int,
             r_min_au: float = R_MIN_AU, r_max_au: float = R_MAX_AU) -> Grid:
    """Log-spaced radial interfaces, uniform full-sphere theta and phi."""
    r_if = np.geomspace(r_min_au * AU_CM, r_max_au * AU_CM, nr + 1)
    theta_if = np.linspace(0.0, math.pi, ntheta + 1)
    phi_if = np.linspace(0.0, 2.0 * math.pi, nphi + 1)
    return Grid(r_if, theta_if, phi_if)


def stretched_grid(nr: int, ntheta: int, nphi: int, stretch: float = 1.1,
                   r_min_au: float = R_MIN_AU, r_max_au: float = R_MAX_AU) -> Grid:
    """Radial cells growing by a constant factor (the paper's 10 % stretch)."""
    w = stretch ** np.arange(nr)
    edges = np.concatenate([[0.0], np.cumsum(w)]) / np.sum(w)
    r_if = r_min_au * AU_CM + edges * (r_max_au - r_min_au) * AU_CM
    theta_if = np.linspace(0.0, math.pi, ntheta + 1)
    phi_if = np.linspace(0.0, 2.0 * math.pi, nphi + 1)
    return Grid(r_if, theta_if, phi_if)


# ----------------------------------------------------------------------------
# opacity table
# ----------------------------------------------------------------------------
def nu_bins(n_nu: int) -> np.ndarray:
    """Log-spaced mid-frequencies 1e11..1e16 Hz, end points included."""
    if n_nu == 1:
        return np.array([NU_550NM_HZ])
    i = np.arange(n_nu, dtype=np.float64)
    return NU_LO_HZ * (NU_HI_HZ / NU_LO_HZ) ** (i / (n_nu - 1))


_BUMPS = ((C_CM_S / 9.7e-4, 50.0), (C_CM_S / 18e-4, 25.0))  # (centre Hz, cm^2/g)
_BUMP_SIGMA_DEX = 0.05


def kappa_synth(nu: np.ndarray) -> np.ndarray:
    """Synthetic dust opacity (cm^2/g): a nu^1.5 power law plus two Gaussian
    bumps in log10(nu) at 9.7 and 18 micron (silicate-like features)."""
    nu = np.asarray(nu, dtype=np.float64)
    k = 1e3 * (nu / 1e15) ** 1.5
    lg = np.log10(nu)
    for centre, amp in _BUMPS:
        k = k + amp * np.exp(-0.5 * ((lg - math.log10(centre)) / _BUMP_SIGMA_DEX) ** 2)
    return k


# ----------------------------------------------------------------------------
# density (Sect. 3.1.1)
# ----------------------------------------------------------------------------
# temperature-dependent variant: ice mantles evaporating near 150 K remove 30 % of
# the opacity (a smooth logistic step of width 15 K), on a log-spaced T grid
T_GRID_LO_K, T_GRID_HI_K = 10.0, 1500.0


def t_grid(n_t: int = 24) -> np.ndarray:
    return np.geomspace(T_GRID_LO_K, T_GRID_HI_K, n_t)


def kappa_synth_t(nu: np.ndarray, tg: np.ndarray) -> np.ndarray:
    """kappa(nu, T) [n_nu][n_t] = kappa_synth(nu) (1 - 0.3 / (1 + e^{-(T - 150 K) / 15 K}))."""
    s = 1.0 - 0.3 / (1.0 + np.exp(-(np.asarray(tg, dtype=np.float64) - 150.0) / 15.0))
    return np.outer(kappa_synth(nu), s)


# a second species with its own spectral shape: water-ice bands at 3.1 and 45 micron
# (Gaussians in log10 nu, 0.08 dex wide, 40 and 20 cm^2/g) present below ~150 K
_ICE_BANDS = ((C_CM_S / 3.1e-4, 40.0), (C_CM_S / 45e-4, 20.0))


def kappa_synth_t2(nu: np.ndarray, tg: np.ndarray) -> np.ndarray:
    """A kappa(nu, T) [n_nu][n_t] that does not separate into kappa(nu) b(T): the
    table of kappa_synth_t plus ice bands whose carrier evaporates near 150 K (the
    same logistic step), two spectral shapes with different temperature factors."""
    nu = np.asarray(nu, dtype=np.float64)
    step = 1.0 / (1.0 + np.exp(-(np.asarray(tg, dtype=np.float64) - 150.0) / 15.0))
    lg = np.log10(nu)
    ice = np.zeros_like(nu)
    for centre, amp in _ICE_BANDS:
        ice = ice + amp * np.exp(-0.5 * ((lg - math.log10(centre)) / 0.08) ** 2)
    return kappa_synth_t(nu, tg) + np.outer(ice, 1.0 - step)


# a third species: CO2-ice bands at 4.27 and 15.2 micron (0.06 dex wide, 25 and 12
# cm^2/g) whose carrier evaporates near 70 K
_CO2_BANDS = ((C_CM_S / 4.27e-4, 25.0), (C_CM_S / 15.2e-4, 12.0))


def kappa_synth_t3(nu: np.ndarray, tg: np.ndarray) -> np.ndarray:
    """A kappa(nu, T) [n_nu][n_t] of rank three: the table of kappa_synth_t2 plus
    CO2-ice bands present below ~70 K (logistic step, 8 K wide)."""
    nu = np.asarray(nu, dtype=np.float64)
    step = 1.0 / (1.0 + np.exp(-(np.asarray(tg, dtype=np.float64) - 70.0) / 8.0))
    lg = np.log10(nu)
    co2 = np.zeros_like(nu)
    for centre, amp in _CO2_BANDS:
        co2 = co2 + amp * np.exp(-0.5 * ((lg - math.log10(centre)) / 0.06) ** 2)
    return kappa_synth_t2(nu, tg) + np.outer(co2, 1.0 - step)


# a fourth species: CO-ice band at 4.67 micron (0.05 dex wide, 30 cm^2/g) whose carrier
# evaporates near 25 K
_CO_BANDS = ((C_CM_S / 4.67e-4, 30.0),)


def kappa_synth_t4(nu: np.ndarray, tg: np.ndarray) -> np.ndarray:
    """A kappa(nu, T) [n_nu][n_t] of rank four: the table of kappa_synth_t3 plus a
    CO-ice band present below ~25 K (logistic step, 3 K wide)."""
    nu = np.asarray(nu, dtype=np.float64)
    step = 1.0 / (1.0 + np.exp(-(np.asarray(tg, dtype=np.float64) - 25.0) / 3.0))
    lg = np.log10(nu)
    co = np.zeros_like(nu)
    for centre, amp in _CO_BANDS:
        co = co + amp * np.exp(-0.5 * ((lg - math.log10(centre)) / 0.05) ** 2)
    return kappa_synth_t3(nu, tg) + np.outer(co, 1.0 - step)


def kappa_synth_t_full(nu: np.ndarray, tg: np.ndarray, seed: int = 0) -> np.ndarray:
    """A kappa(nu, T) [n_nu][n_t] with no low-rank structure: kappa_synth(nu) times an
    independent factor in [0.5, 1.5) per entry (full rank)."""
    rng = np.random.default_rng(seed)
    return kappa_synth(np.asarray(nu, dtype=np.float64))[:, None] * (0.5 + rng.random((len(nu), len(tg))))


def rho0_for_tau550(tau550: float, kappa550: float | None = None) -> float:
    """Midplane normalisation: tau550 = int_{r_min}^{r_max} rho0 (r_d/r) kappa dr
    along z = 0, i.e. rho0 = tau550 / (kappa550 r_d ln(r_max/r_min))."""
    if kappa550 is None:
        kappa550 = float(kappa_synth(np.array([NU_550NM_HZ]))[0])
    return tau550 / (kappa550 * R_D_AU * AU_CM * math.log(R_MAX_AU / R_MIN_AU))


def disk_density(r_cyl: np.ndarray, z: np.ndarray, rho0: float) -> np.ndarray:
    """rho = rho0 f1 f2 with f1 = r_d/r, f2 = exp(-pi/4 (z/h)^2), h = z_d (r/r_d)^1.125."""
    rd = R_D_AU * AU_CM
    zd = Z_D_AU * AU_CM
    h = zd * (r_cyl / rd) ** 1.125
    with np.errstate(divide="ignore", over="ignore", under="ignore", invalid="ignore"):
        return rho0 * (rd / r_cyl) * np.exp(-0.25 * math.pi * (z / h) ** 2)


def density(grid: Grid, tau550: float, envelope: bool = False,
            perturb_sigma: float = 0.0, seed: int = 0,
            kappa550: float | None = None) -> np.ndarray:
    """Cell-centre density [nphi][ntheta][nr] (float64).

    Disk term normalised to the midplane tau550, optional envelope
    1e-3 rho0 (r/r_d)^-1.5, optional i.i.d. lognormal perturbation
    exp(perturb_sigma * g), then the 1e-100 floor relative to the maximum.
    """
    rho0 = rho0_for_tau550(tau550, kappa550)
    r_c, th_c = grid.centres()
    R, TH = np.meshgrid(r_c, th_c)                    # [ntheta][nr]
    r_cyl = R * np.sin(TH)
    z = R * np.cos(TH)
    base = np.where(r_cyl > 0, disk_density(np.maximum(r_cyl, 1e-300), z, rho0), 0.0)
    if envelope:
        base = base + 1e-3 * rho0 * (R / (R_D_AU * AU_CM)) ** -1.5
    out = np.empty(grid.shape, dtype=np.float64)
    plane = grid.ntheta * grid.nr
    for p in range(grid.nphi):
        if perturb_sigma > 0.0:
            idx = np.arange(p * plane, (p + 1) * plane, dtype=np.uint64)
            g = hash_normal(seed, 1, idx).reshape(grid.ntheta, grid.nr)
            out[p] = base * np.exp(perturb_sigma * g)
        else:
            out[p] = base
    floor = DENSITY_FLOOR_REL * out.max()
    np.maximum(out, floor, out=out)
    return out


def tdust_uniform(grid: Grid, t: float) -> np.ndarray:
    return np.full(grid.shape, t, dtype=np.float64)


def tdust_random(grid: Grid, t_lo: float, t_hi: float, seed: int) -> np.ndarray:
    """i.i.d. uniform dust temperatures in [t_lo, t_hi] (K)."""
    idx = np.arange(grid.ncells, dtype=np.uint64)
    u = hash_u01(seed, 7, idx)
    return (t_lo + (t_hi - t_lo) * u).reshape(grid.shape)


def fld_fields(grid: Grid, seed: int = 1, t_in: float = 300.0, e_in: float = 1e-5, q_in: float = 1e-12):
    """Old state of a radiation-diffusion step on ``grid`` [nphi][ntheta][nr] (float64):
    gas temperature t_in (r/r_in)^-1/2 x lognormal(0.1), clipped to 10..1500 K;
    radiation energy density e_in (r/r_in)^-2 x lognormal(0.3) (erg cm^-3);
    source q_in (r/r_in)^-5/2 x U(0, 1) (erg s^-1 cm^-3)."""
    r_c, _ = grid.centres()
    x = np.broadcast_to(r_c / grid.r_if[0], grid.shape)
    idx = np.arange(grid.ncells, dtype=np.uint64)
    g1 = hash_normal(seed, 30, idx).reshape(grid.shape)
    g2 = hash_normal(seed, 31, idx).reshape(grid.shape)
    u = hash_u01(seed, 32, idx).reshape(grid.shape)
    t = np.clip(t_in * x ** -0.5 * np.exp(0.1 * g1), 10.0, 1500.0)
    e = e_in * x ** -2.0 * np.exp(0.3 * g2)
    q = q_in * x ** -2.5 * u
    return t, e, q


def gas_mass(grid: Grid, rho: np.ndarray) -> float:
    """Total mass (g) of a cell-centred density field on a spherical grid."""
    dv_r = (grid.r_if[1:] ** 3 - grid.r_if[:-1] ** 3) / 3.0
    dcos = np.cos(grid.theta_if[:-1]) - np.cos(grid.theta_if[1:])
    dphi = np.diff(grid.phi_if)
    vol = dphi[:, None, None] * dcos[None, :, None] * dv_r[None, None, :]
    return float(np.sum(rho * vol))


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    nu: np.ndarray
    kappa: np.ndarray
    rho: np.ndarray          # float64
    tdust: np.ndarray        # float64
    t_star: float = T_STAR_K
    r_star: float = R_STAR_CM
    t_sub: float = T_SUB_K
    tau550: float = 1.0

    def rho32(self) -> np.ndarray:
        return self.rho.astype(np.float32)

    def tdust32(self) -> np.ndarray:
        return self.tdust.astype(np.float32)


def disk2d(nr=64, ntheta=32, n_nu=32, tau550=1.0) -> Workload:
    """2-D axisymmetric disk, no envelope, no perturbation, uniform 50 K dust."""
    g = log_grid(nr, ntheta, 1)
    nu = nu_bins(n_nu)
    return Workload(f"disk2d_{nr}x{ntheta}x1_nu{n_nu}_tau{tau550:g}", g, nu, kappa_synth(nu),
                    density(g, tau550), tdust_uniform(g, 50.0), tau550=tau550)


def disk3d(nr=256, ntheta=128, nphi=256, n_nu=79, tau550=1.0, seed=1) -> Workload:
    """3-D disk plus envelope, +-20 % lognormal perturbation, dust 20-1600 K."""
    g = log_grid(nr, ntheta, nphi)
    nu = nu_bins(n_nu)
    rho = density(g, tau550, envelope=True, perturb_sigma=math.log(1.2), seed=seed)
    td = tdust_random(g, 20.0, 1600.0, seed)
    return Workload(f"disk3d_{nr}x{ntheta}x{nphi}_nu{n_nu}_tau{tau550:g}_s{seed}", g, nu,
                    kappa_synth(nu), rho, td, tau550=tau550)


def batch_specs(n_grids=96, seed=3):
    """Shapes and optical depths of the uneven multi-grid batch: Nr in 64..512,
    Ntheta in 32..256, Nphi in {1, 64, 128}, Nnu in {32, 79, 128},
    tau550 log-uniform in 0.1..100."""
    idx = np.arange(n_grids, dtype=np.uint64)
    u = [hash_u01(seed, 20 + s, idx) for s in range(5)]
    nr = 64 + np.minimum((u[0] * 449).astype(int), 448)
    nth = 32 + np.minimum((u[1] * 225).astype(int), 224)
    nph = np.array([1, 64, 128])[np.minimum((u[2] * 3).astype(int), 2)]
    nnu = np.array([32, 79, 128])[np.minimum((u[3] * 3).astype(int), 2)]
    tau = 10.0 ** (-1.0 + 3.0 * u[4])
    return [dict(nr=int(a), ntheta=int(b), nphi=int(c), n_nu=int(d), tau550=float(t),
                 seed=int(seed * 1000 + i))
            for i, (a, b, c, d, t) in enumerate(zip(nr, nth, nph, nnu, tau))]
