"""FP64 reference of one implicit flux-limited-diffusion step (Sect. 2.1, Eqs. 7-15,
with the irradiation source of Eq. 15).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only tests and the benchmark's
CPU legs use it; the CUDA library never does.

The step, backward Euler in E = E_R with the coefficients frozen at the old state:
    (E' - E) / dt = f_c (div(D grad E') + q_abs)                       (Eqs. 8, 15)
    f_c = 1 / (c_V rho / (4 a T^3) + 1)                                 (Eq. 9)
    D = lambda c / (kappa_R rho), lambda = (2 + R) / (6 + 3 R + R^2),
    R = |grad E| / (kappa_R rho E)                                      (Eqs. 10-13)
with q_abs = -div F_* the absorbed stellar power (Eq. 15) and Q+ = 0 (no gas
motion). With s = kappa_R rho and g = |grad E| / E, D = c (2 s + g) / (6 s^2 + 3 s g
+ g^2), the same expression without the division by s (finite as s -> 0).

Finite volumes on the spherical grid: cell volume V = dOmega (r+^3 - r-^3) / 3; a
face carries w = D_f A / d (harmonic mean of the two cells' D, area A, distance d
between the cell centres), so the step is the symmetric positive definite system
    (V / (dt f_c)) E'_c + sum_faces w (E'_c - E'_nb) = (V / (dt f_c)) E_c + V q_abs,c.
Boundaries: no flux through the inner radius and through theta faces at the poles
(zero area) or at the ends of a partial theta range; E = a T_bg^4 beyond the outer
radius, at half a cell; periodic in phi when nphi > 1. Gradients for R are central
differences (one-sided at the radial and theta ends, periodic in phi).
The sparse system is solved directly (scipy.sparse.linalg.spsolve).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import rosseland_mean, sigma_sb

C = 2.99792458e10
T_LO, T_HI = 1.0, 1e5   # temperature range over which kappa_R(T) is evaluated (clamped outside)


def radiation_constant() -> float:
    return 4.0 * sigma_sb() / C


def limiter(R):
    """Levermore-Pomraning flux limiter (Eq. 12)."""
    R = np.asarray(R, dtype=np.float64)
    return (2.0 + R) / (6.0 + 3.0 * R + R * R)


def diffusion_coefficient(s, g):
    """D = lambda c / s with R = g / s (Eqs. 11-13), written as c (2 s + g) / (6 s^2 + 3 s g + g^2);
    0 where s = g = 0 (no matter and no gradient: the limiter leaves D undefined)."""
    s = np.asarray(s, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    num = 2.0 * s + g
    den = 6.0 * s * s + 3.0 * s * g + g * g
    return np.where(num > 0.0, C * num / np.where(num > 0.0, den, 1.0), 0.0)


class Geometry:
    def __init__(self, r_if, th_if, ph_if):
        self.r_if, self.th_if, self.ph_if = (np.asarray(a, dtype=np.float64) for a in (r_if, th_if, ph_if))
        self.nr, self.nth, self.nph = len(self.r_if) - 1, len(self.th_if) - 1, len(self.ph_if) - 1
        self.rc = 0.5 * (self.r_if[:-1] + self.r_if[1:])
        self.thc = 0.5 * (self.th_if[:-1] + self.th_if[1:])
        self.phc = 0.5 * (self.ph_if[:-1] + self.ph_if[1:])
        dcos = np.cos(self.th_if[:-1]) - np.cos(self.th_if[1:])
        dph = np.diff(self.ph_if)
        self.dom = dph[:, None] * dcos[None, :]                       # [nph][nth]
        d3 = (self.r_if[1:] ** 3 - self.r_if[:-1] ** 3) / 3.0
        self.vol = self.dom[:, :, None] * d3[None, None, :]             # [nph][nth][nr]
        self.dr2 = 0.5 * (self.r_if[1:] ** 2 - self.r_if[:-1] ** 2)     # int r dr over a cell


def gradient_norm(geo: Geometry, e):
    """|grad E| per cell by central differences (one-sided at the r and theta ends,
    periodic in phi)."""
    e = np.asarray(e, dtype=np.float64)
    rc, thc, phc = geo.rc, geo.thc, geo.phc
    gr = np.zeros_like(e)
    if geo.nr > 1:
        gr[..., 1:-1] = (e[..., 2:] - e[..., :-2]) / (rc[2:] - rc[:-2])
        gr[..., 0] = (e[..., 1] - e[..., 0]) / (rc[1] - rc[0])
        gr[..., -1] = (e[..., -1] - e[..., -2]) / (rc[-1] - rc[-2])
    gt = np.zeros_like(e)
    if geo.nth > 1:
        rr = rc[None, None, :]
        gt[:, 1:-1, :] = (e[:, 2:, :] - e[:, :-2, :]) / (rr * (thc[2:] - thc[:-2])[None, :, None])
        gt[:, 0, :] = (e[:, 1, :] - e[:, 0, :]) / (rr[:, 0, :] * (thc[1] - thc[0]))
        gt[:, -1, :] = (e[:, -1, :] - e[:, -2, :]) / (rr[:, 0, :] * (thc[-1] - thc[-2]))
    gp = np.zeros_like(e)
    if geo.nph > 1:
        up = np.roll(e, -1, axis=0)
        dn = np.roll(e, 1, axis=0)
        dphi = (np.roll(phc, -1) - np.roll(phc, 1)) % (2.0 * np.pi)
        dphi = np.where(dphi == 0.0, 2.0 * np.pi, dphi)
        scale = rc[None, None, :] * np.sin(thc)[None, :, None] * dphi[:, None, None]
        gp = (up - dn) / scale
    return np.sqrt(gr * gr + gt * gt + gp * gp)


def cell_coefficients(geo, rho, t, e, kappa_r, c_v):
    """D and f_c per cell (Eqs. 9, 11-13) from the old state."""
    a = radiation_constant()
    s = np.asarray(kappa_r, dtype=np.float64) * np.asarray(rho, dtype=np.float64)
    g = gradient_norm(geo, e) / np.asarray(e, dtype=np.float64)
    d = diffusion_coefficient(s, g)
    t = np.asarray(t, dtype=np.float64)
    fc = 1.0 / (c_v * np.asarray(rho, dtype=np.float64) / (4.0 * a * t ** 3) + 1.0)
    return d, fc


def assemble(geo, d, fc, dt, t_bg):
    """Diagonal, face list (index pairs, weights) and the constant terms of the system."""
    a = radiation_constant()
    shape = geo.vol.shape
    idx = np.arange(geo.vol.size).reshape(shape)
    rows, cols, ws = [], [], []

    def faces(ia, ib, da, db, area, dist):
        pos = (da > 0.0) & (db > 0.0)
        df = np.where(pos, 2.0 * da * db / np.where(pos, da + db, 1.0), 0.0)
        rows.append(ia.ravel())
        cols.append(ib.ravel())
        ws.append((df * area / dist).ravel())

    # radial faces between k and k+1
    if geo.nr > 1:
        area = geo.dom[:, :, None] * (geo.r_if[1:-1] ** 2)[None, None, :]
        dist = np.broadcast_to((geo.rc[1:] - geo.rc[:-1])[None, None, :], area.shape)
        faces(idx[..., :-1], idx[..., 1:], d[..., :-1], d[..., 1:], area, dist)
    # theta faces between j and j+1
    if geo.nth > 1:
        dph = np.diff(geo.ph_if)
        area = dph[:, None, None] * np.sin(geo.th_if[1:-1])[None, :, None] * geo.dr2[None, None, :]
        dist = geo.rc[None, None, :] * (geo.thc[1:] - geo.thc[:-1])[None, :, None]
        dist = np.broadcast_to(dist, area.shape)
        faces(idx[:, :-1, :], idx[:, 1:, :], d[:, :-1, :], d[:, 1:, :], area, dist)
    # phi faces between l and l+1 (periodic)
    if geo.nph > 1:
        dth = np.diff(geo.th_if)
        area = np.broadcast_to(dth[None, :, None] * geo.dr2[None, None, :], shape)
        dphc = (np.roll(geo.phc, -1) - geo.phc) % (2.0 * np.pi)
        dist = geo.rc[None, None, :] * np.sin(geo.thc)[None, :, None] * dphc[:, None, None]
        faces(idx, np.roll(idx, -1, axis=0), d, np.roll(d, -1, axis=0), area, dist)
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    ws = np.concatenate(ws) if ws else np.zeros(0)
    diag = (geo.vol / (dt * fc)).ravel().copy()
    np.add.at(diag, rows, ws)
    np.add.at(diag, cols, ws)
    # outer radial boundary: E = a T_bg^4 half a cell beyond the last centre
    w_out = d[..., -1] * geo.dom * geo.r_if[-1] ** 2 / (geo.r_if[-1] - geo.rc[-1])
    diag[idx[..., -1].ravel()] += w_out.ravel()
    bnd = np.zeros(geo.vol.size)
    bnd[idx[..., -1].ravel()] = (w_out * a * t_bg ** 4).ravel()
    return diag, rows, cols, ws, bnd


def fld_step(r_if, th_if, ph_if, rho, t, q_abs, e_old, dt, c_v, t_bg, nu_mid, kappa, kappa_r=None):
    """E_R after one implicit step; kappa_r per cell (default: the table's Rosseland
    mean at each cell's temperature, clamped to T_LO .. T_HI)."""
    geo = Geometry(r_if, th_if, ph_if)
    rho = np.asarray(rho, dtype=np.float64).reshape(geo.vol.shape)
    t = np.asarray(t, dtype=np.float64).reshape(geo.vol.shape)
    e_old = np.asarray(e_old, dtype=np.float64).reshape(geo.vol.shape)
    q = np.asarray(q_abs, dtype=np.float64).reshape(geo.vol.shape)
    if kappa_r is None:
        # kappa_R at T clamped to 1 K .. 1e5 K, the range of the library's table
        uniq, inv = np.unique(np.clip(t, T_LO, T_HI), return_inverse=True)
        kr_u = np.array([rosseland_mean(float(tt), nu_mid, kappa) for tt in uniq])
        kappa_r = kr_u[inv].reshape(t.shape)
    d, fc = cell_coefficients(geo, rho, t, e_old, kappa_r, c_v)
    diag, rows, cols, ws, bnd = assemble(geo, d, fc, dt, t_bg)
    n = geo.vol.size
    A = sp.coo_matrix((np.concatenate([diag, -ws, -ws]),
                       (np.concatenate([np.arange(n), rows, cols]), np.concatenate([np.arange(n), cols, rows]))),
                      shape=(n, n)).tocsr()
    b = (geo.vol / (dt * fc)).ravel() * e_old.ravel() + (geo.vol * q).ravel() + bnd
    return spla.spsolve(A.tocsc(), b).reshape(geo.vol.shape)


def _grad_at(geo, e, l, j, k):
    """|grad E| at one cell, by the same differences as gradient_norm."""
    gr = gt = gp = 0.0
    if geo.nr > 1:
        ka, kb = max(k - 1, 0), min(k + 1, geo.nr - 1)
        gr = (e[l, j, kb] - e[l, j, ka]) / (geo.rc[kb] - geo.rc[ka])
    if geo.nth > 1:
        ja, jb = max(j - 1, 0), min(j + 1, geo.nth - 1)
        gt = (e[l, jb, k] - e[l, ja, k]) / (geo.rc[k] * (geo.thc[jb] - geo.thc[ja]))
    if geo.nph > 1:
        la, lb = (l - 1) % geo.nph, (l + 1) % geo.nph
        dphi = (geo.phc[lb] - geo.phc[la]) % (2.0 * np.pi)
        if dphi == 0.0:
            dphi = 2.0 * np.pi
        gp = (e[lb, j, k] - e[la, j, k]) / (geo.rc[k] * np.sin(geo.thc[j]) * dphi)
    return float(np.sqrt(gr * gr + gt * gt + gp * gp))


def row_residuals(r_if, th_if, ph_if, rho, t, q_abs, e_old, e_new, dt, c_v, t_bg, kappa_r_of_t, cells):
    """For each (l, j, k) in ``cells``: the residual of that cell's row of the implicit
    system (the equation ``assemble`` writes, rebuilt for the one cell from its own
    and its neighbours' coefficients) at ``e_new``, divided by the sum of the
    magnitudes of the row's terms. kappa_r_of_t: T -> kappa_R. For checking a
    solution at sizes where the whole system is too large to solve here."""
    geo = Geometry(r_if, th_if, ph_if)
    shp = geo.vol.shape
    rho, t, q, e0, e1 = (np.asarray(a, dtype=np.float64).reshape(shp) for a in (rho, t, q_abs, e_old, e_new))
    a = radiation_constant()
    dph = np.diff(geo.ph_if)
    dth = np.diff(geo.th_if)
    memo = {}

    def d_at(l, j, k):
        key = (l, j, k)
        if key not in memo:
            s = kappa_r_of_t(float(t[l, j, k])) * rho[l, j, k]
            g = _grad_at(geo, e0, l, j, k) / e0[l, j, k]
            memo[key] = float(diffusion_coefficient(s, g))
        return memo[key]

    def harm(x, y):
        return 2.0 * x * y / (x + y) if x > 0.0 and y > 0.0 else 0.0

    out = []
    for (l, j, k) in cells:
        dc = d_at(l, j, k)
        fc = 1.0 / (c_v * rho[l, j, k] / (4.0 * a * t[l, j, k] ** 3) + 1.0)
        store = geo.vol[l, j, k] / (dt * fc)
        terms = [store * e1[l, j, k], -store * e0[l, j, k], -geo.vol[l, j, k] * q[l, j, k]]
        nbs = []
        dom = geo.dom[l, j]
        for kk in (k - 1, k + 1):
            if 0 <= kk < geo.nr:
                rf = geo.r_if[max(k, kk)]
                nbs.append(((l, j, kk), dom * rf * rf / abs(geo.rc[kk] - geo.rc[k])))
        if k == geo.nr - 1:
            w_out = dc * dom * geo.r_if[-1] ** 2 / (geo.r_if[-1] - geo.rc[k])
            terms += [w_out * e1[l, j, k], -w_out * a * t_bg ** 4]
        for jj in (j - 1, j + 1):
            if 0 <= jj < geo.nth:
                tf = geo.th_if[max(j, jj)]
                nbs.append(((l, jj, k), dph[l] * np.sin(tf) * geo.dr2[k] / (geo.rc[k] * abs(geo.thc[jj] - geo.thc[j]))))
        if geo.nph > 1:
            for step in (-1, 1):
                ll = (l + step) % geo.nph
                lo = l if step == 1 else ll     # the face lies between lo and lo + 1
                dphc = (geo.phc[(lo + 1) % geo.nph] - geo.phc[lo]) % (2.0 * np.pi)
                nbs.append(((ll, j, k), dth[j] * geo.dr2[k] / (geo.rc[k] * np.sin(geo.thc[j]) * dphc)))
        for nb, geom in nbs:
            wf = harm(dc, d_at(*nb)) * geom
            terms += [wf * e1[l, j, k], -wf * e1[nb]]
        terms = np.array(terms)
        out.append(abs(terms.sum()) / max(np.abs(terms).sum(), 1e-300))
    return np.array(out)
