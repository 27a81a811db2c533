// The Planck band integral in x = h nu / (k T), shared by the set-up of the stellar
// bin fluxes (Eq. 20) and the Planck-mean opacity table of the temperature update.
#pragma once

#include <math.h>

namespace rt {
namespace {

// t^3 / (e^t - 1), the Planck integrand in x = h nu / (k T)
__device__ double planck_x(double t) { return t * t * t / expm1(t); }

// 8-point Gauss-Legendre rule on [a, b] (nodes and weights of the Legendre
// polynomial P_8, Abramowitz & Stegun Table 25.4).
__device__ double gauss_legendre8(double a, double b)
{
    const double xs[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267,
                          0.9602898564975363};
    const double ws[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745,
                          0.1012285362903763};
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double s = 0.0;
    for (int i = 0; i < 4; ++i) s += ws[i] * (planck_x(c - h * xs[i]) + planck_x(c + h * xs[i]));
    return s * h;
}

// int_a^b t^3/(e^t-1) dt by composite Gauss-Legendre on panels no wider than one
// unit of x, the panels spread over the 32 lanes of a warp. The integrand is
// analytic with its nearest poles at +-2 pi i, so each panel converges far below
// double rounding. The upper edge is cut at a + 60 (an infinite one included):
// beyond it the integrand is below e^-60 of its value at a. Bands starting above
// x = 700 (t^3 e^-t below 1e-295) are zero. Result valid in every lane.
__device__ double planck_band_warp(double a, double b, int lane)
{
    if (a > 700.0) return 0.0;
    b = fmin(b, a + 60.0);
    double s = 0.0;
    if (b > a) {
        const int n = (int)ceil(b - a);
        const double h = (b - a) / n;
        for (int p = lane; p < n; p += 32) s += gauss_legendre8(a + p * h, a + (p + 1) * h);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Rosseland weight of the band [a, b]: int t^4 e^t / (e^t - 1)^2 dt, by parts
// a^4/(e^a - 1) - b^4/(e^b - 1) + 4 int_a^b t^3/(e^t - 1) dt (result in every lane).
__device__ double rosseland_band_warp(double a, double b, int lane)
{
    if (a > 700.0) return 0.0;
    const double ea = a > 0.0 ? a * a * a * a / expm1(a) : 0.0;
    const double eb = (isinf(b) || b > 700.0) ? 0.0 : b * b * b * b / expm1(b);
    return ea - eb + 4.0 * planck_band_warp(a, b, lane);
}

// kappa of bin row `row` at temperature t: linear between the bracketing points of
// t_grid, the end values beyond (n_t <= 1: the one value)
__device__ double kappa_at(const double *row, int n_t, const double *t_grid, double t)
{
    if (n_t <= 1 || t <= t_grid[0]) return row[0];
    if (t >= t_grid[n_t - 1]) return row[n_t - 1];
    int j = 0;
    while (!(t < t_grid[j + 1])) ++j;
    return row[j] + (row[j + 1] - row[j]) * ((t - t_grid[j]) / (t_grid[j + 1] - t_grid[j]));
}

}  // namespace
}  // namespace rt
