"""The algebra behind the tracer's series for bins optically thin along a whole ray
(FP64, on the CPU): for Phi(u) = sum_i w_i e^{-kappa_i u},

    Phi(N) - Phi(N + dN) = dN s sum_{k>=1} C_k h_{k-1}(s (N + dN), s N),
    C_k = (-1)^{k+1} / k! sum_i w_i (kappa_i / s)^k,  h_{k-1}(a, c) = sum_{j<k} a^j c^{k-1-j},

evaluated as the divided difference of P(u) = sum_k C_k u^k by the paired Horner
recurrence, and Phi(N) = S_0 - P(s N). These are checked against the direct sums of
exponentials (Eqs. 17, 31-32 per bin) where every kappa_i (N + dN) <= 1, with the
truncation the tracer uses (10 terms). The per-lane form of the same series (the row
shifted to a lane's first column, merged with the bins thin within the lane's
cells) is checked against the same direct sums."""
from __future__ import annotations

import math

import numpy as np
import pytest

K_TERMS = 10
X_MAX = 1.0


def _coefficients(kappa, w):
    s = kappa.max()
    c = [0.0] + [(1 if k % 2 else -1) * np.sum(w * (kappa / s) ** k) / math.factorial(k) for k in range(1, K_TERMS + 1)]
    return s, c, float(np.sum(w))


def _divided_difference(c, a, b):
    """(P(a) - P(b)) / (a - b) for P(u) = sum_{k=1..K} c_k u^k, without forming a - b."""
    dd = np.full_like(a, c[K_TERMS])
    pb = dd * b + c[K_TERMS - 1]
    for k in range(K_TERMS - 2, 0, -1):
        dd = dd * a + pb
        pb = pb * b + c[k]
    return dd * a + pb


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_absorbed_part_matches_the_bin_sum(seed):
    rng = np.random.default_rng(seed)
    kappa = 10.0 ** rng.uniform(-3, 1, 40)
    w = 10.0 ** rng.uniform(-6, 0, 40)
    n_tot = X_MAX / kappa.max()
    n = rng.uniform(0, 1, 2000) * n_tot
    dn = rng.uniform(0, 1, 2000) * (n_tot - n)
    dn[:10] = 1e-12 * n_tot          # cells far thinner than their column: no cancellation
    exact = np.sum(w[None, :] * np.exp(-kappa[None, :] * n[:, None]) * -np.expm1(-kappa[None, :] * dn[:, None]), axis=1)
    s, c, _ = _coefficients(kappa, w)
    series = dn * s * _divided_difference(c, s * (n + dn), s * n)
    np.testing.assert_allclose(series, exact, rtol=math.exp(X_MAX) * X_MAX ** K_TERMS / math.factorial(K_TERMS))


def test_divided_difference_is_the_homogeneous_sum():
    """The recurrence equals sum_k C_k h_{k-1}(a, c), h written out term by term."""
    rng = np.random.default_rng(5)
    c = [0.0] + list(rng.normal(size=K_TERMS))
    a, b = rng.uniform(0, X_MAX, 50), rng.uniform(0, X_MAX, 50)
    direct = sum(c[k] * sum(a ** j * b ** (k - 1 - j) for j in range(k)) for k in range(1, K_TERMS + 1))
    np.testing.assert_allclose(_divided_difference(c, a, b), direct, rtol=1e-13)
    # and the secant form where a and b are far apart
    p = lambda u: sum(c[k] * u ** k for k in range(1, K_TERMS + 1))
    far = np.abs(a - b) > 0.1
    np.testing.assert_allclose(_divided_difference(c, a, b)[far], ((p(a) - p(b)) / (a - b))[far], rtol=1e-12)


def test_escaping_part_matches_the_bin_sum():
    rng = np.random.default_rng(7)
    kappa = 10.0 ** rng.uniform(-2, 2, 60)
    w = 10.0 ** rng.uniform(-4, 0, 60)
    s, c, s0 = _coefficients(kappa, w)
    n = np.linspace(0.0, X_MAX / s, 101)
    exact = np.sum(w[None, :] * np.exp(-kappa[None, :] * n[:, None]), axis=1)
    u = s * n
    p = sum(c[k] * u ** k for k in range(1, K_TERMS + 1))
    # first omitted term C_{K+1} u^{K+1} <= S_0 X^{K+1} / (K+1)!, against Phi >= S_0 e^{-X}
    np.testing.assert_allclose(s0 - p, exact, rtol=math.exp(X_MAX) * X_MAX ** (K_TERMS + 1) / math.factorial(K_TERMS + 1))


def test_truncation_bound():
    """At the edge of the thin region (every kappa_i (N + dN) = X_MAX) the first omitted
    term bounds the error: x^K / K! relative to the leading term."""
    kappa = np.array([1.0])
    w = np.array([1.0])
    s, c, _ = _coefficients(kappa, w)
    n, dn = np.array([X_MAX / 2]), np.array([X_MAX / 2])
    exact = np.exp(-X_MAX / 2) * -np.expm1(-X_MAX / 2)
    series = dn * s * _divided_difference(c, s * (n + dn), s * n)
    assert abs(series[0] / exact - 1) < X_MAX ** K_TERMS / math.factorial(K_TERMS)


def _lane_series(kappa, w, bt, bt2, n0, u, dn, n_max):
    """The tracer's per-lane form (rt_ray.cuh, lane_coefficients and lane_series) in
    FP64: the row of the bins i < bt (thin along the whole ray) shifted to the lane's
    column n0 by synthetic division and rescaled to v = s2 u, plus the bins
    bt <= i < bt2 (thin within the lane's cells) expanded about n0; then the divided
    difference between v = s2 (u + dn) and v = s2 u."""
    K = K_TERMS
    f = np.zeros(K + 1)
    s2 = kappa[bt2 - 1]
    if bt > 0:
        s = kappa[bt - 1]
        c = [0.0] + [(1 if k % 2 else -1) * np.sum(w[:bt] * (kappa[:bt] / s) ** k) / math.factorial(k)
                     for k in range(1, K + 1)]
        x0 = s * n0
        for i in range(K):
            for j in range(K - 1, max(i, 1) - 1, -1):
                c[j] = x0 * c[j + 1] + c[j]
        if bt2 == bt:
            s2 = s
        for k in range(1, K + 1):
            f[k] = c[k] * (s / s2) ** k
    if bt2 > bt:
        g = w[bt:bt2] * np.exp(-kappa[bt:bt2] * n0)
        for k in range(1, K + 1):
            f[k] += (1 if k % 2 else -1) / math.factorial(k) * np.sum(g * (kappa[bt:bt2] / s2) ** k)
    return dn * s2 * _divided_difference(f, s2 * (u + dn), s2 * u)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_lane_series_matches_the_bin_sum(seed):
    """Cells of one lane (16 of them) behind a column n0: the bins with kappa_i n_max <=
    X_MAX (n_max the largest total column of the warp's rays) and those with kappa_i
    times the lane's own column <= X_MAX, summed by the per-lane series, against the
    per-bin sums of exponentials."""
    rng = np.random.default_rng(seed)
    kappa = np.sort(10.0 ** rng.uniform(-3, 4, 60))
    w = 10.0 ** rng.uniform(-8, 0, 60)
    for trial in range(50):
        dn = 10.0 ** rng.uniform(-7, -1, 16) * rng.uniform(0, 1, 16)
        u = np.concatenate([[0.0], np.cumsum(dn)[:-1]])
        n0 = 10.0 ** rng.uniform(-4, 0.5) * rng.uniform(0, 1)
        n_max = (n0 + dn.sum()) * 10.0 ** rng.uniform(0, 1)   # the warp's longest ray holds the lane's cells
        bt = int(np.searchsorted(kappa, X_MAX / n_max, side="right"))
        bt2 = max(bt, int(np.searchsorted(kappa, X_MAX / dn.sum(), side="right")))
        if bt2 == 0:
            continue
        exact = np.array([np.sum(w[:bt2] * np.exp(-kappa[:bt2] * (n0 + u[j])) * -np.expm1(-kappa[:bt2] * dn[j]))
                          for j in range(16)])
        series = _lane_series(kappa, w, bt, bt2, n0, u, dn, n_max)
        m = exact > 0
        # the first omitted term is below X^K / K! of the leading one, and the value
        # below the leading term by at most e^{-X}
        np.testing.assert_allclose(series[m], exact[m], rtol=math.exp(X_MAX) * X_MAX ** K_TERMS / math.factorial(K_TERMS))


def test_mixed_class_fraction_bound():
    """The absorbed fraction of the mixed class (rt_device.cuh): the smaller of the
    5-term series of 1 - e^{-x} and 1 - e^{-x} (1 + d) + 2^-22, with |d| up to the
    hardware exp2 error 2^-22.7 (either sign), stays within 1.6e-6 of 1 - e^{-x} for
    every x, and is the series itself below x = 1/8; the series is an upper bound."""
    x = np.geomspace(1e-9, 90.0, 200001)
    om = -np.expm1(-x)
    t5 = x - x ** 2 / 2 + x ** 3 / 6 - x ** 4 / 24 + x ** 5 / 120
    assert np.all(t5 >= om * (1 - 1e-15))
    for d in (-2.0 ** -22.7, 0.0, 2.0 ** -22.7):
        big = 1.0 - np.exp(-x) * (1 + d) + 2.0 ** -22
        v = np.minimum(t5, big)
        assert np.max(np.abs(v / om - 1)) < 1.6e-6
        small = x < 0.125
        assert np.all(v[small] == t5[small])
