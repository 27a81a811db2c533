"""The algebra behind the tracer's series for bins optically thin along a whole ray
(FP64, on the CPU): for Phi(u) = sum_i w_i e^{-kappa_i u},

    Phi(N) - Phi(N + dN) = dN s sum_{k>=1} C_k h_{k-1}(s (N + dN), s N),
    C_k = (-1)^{k+1} / k! sum_i w_i (kappa_i / s)^k,  h_{k-1}(a, c) = sum_{j<k} a^j c^{k-1-j},

evaluated as the divided difference of P(u) = sum_k C_k u^k by the paired Horner
recurrence, and Phi(N) = S_0 - P(s N). These are checked against the direct sums of
exponentials (Eqs. 17, 31-32 per bin) where every kappa_i (N + dN) <= 1/2, with the
truncation the tracer uses (8 terms)."""
from __future__ import annotations

import math

import numpy as np
import pytest

K_TERMS = 8
X_MAX = 0.5


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
    np.testing.assert_allclose(series, exact, rtol=2e-7)


def test_divided_difference_is_the_homogeneous_sum():
    """The recurrence equals sum_k C_k h_{k-1}(a, c), h written out term by term."""
    rng = np.random.default_rng(5)
    c = [0.0] + list(rng.normal(size=K_TERMS))
    a, b = rng.uniform(0, 0.5, 50), rng.uniform(0, 0.5, 50)
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
    np.testing.assert_allclose(s0 - p, exact, rtol=2e-8)


def test_truncation_bound():
    """At the edge of the thin region (every kappa_i (N + dN) = 1/2) the first omitted term
    bounds the error: x^K / K! relative to the leading term."""
    kappa = np.array([1.0])
    w = np.array([1.0])
    s, c, _ = _coefficients(kappa, w)
    n, dn = np.array([0.25]), np.array([0.25])
    exact = np.exp(-0.25) * -np.expm1(-0.25)
    series = dn * s * _divided_difference(c, s * (n + dn), s * n)
    assert abs(series[0] / exact - 1) < X_MAX ** K_TERMS / math.factorial(K_TERMS)
