// Lookup-table comparator for the per-bin sum of the tracer (Sect. 2.3, Eqs. 17,
// 28-32, 36): a non-learned stand-in beside the learned surrogate.
//
// With kappa depending on the frequency only, the power a cell absorbs over all bins
// is a function of two numbers, its column N_in in front of it and its own column dN:
//   acc(N_in, dN) = sum_i w_i e^{-kappa_i N_in} (1 - e^{-kappa_i dN}),  w_i = F_i / F_max.
// The table holds log2 G with G = acc / (kappa_ref dN) (finite as dN -> 0, where it
// is sum_i w_i kappa_i e^{-kappa_i N_in} / kappa_ref) on a uniform grid of
// s = log2(kappa_ref N_in + 2^-20) and d = log2(kappa_ref dN + 2^-30), steps of 1/32;
// the tracer interpolates it bilinearly (rt_ray.cuh). Along a ray N_in changes from
// cell to cell and dN slowly, so s is the fast index, and every entry holds the pair
// (node (s_i, d_j), node (s_{i+1}, d_j)): one 8-byte read per row of the square. Every
// grid square is checked in FP64 at its centre and at the midpoints of its four edges:
// where the bilinear value is off by more than half the tolerance the square is
// flagged (the lowest mantissa bit of the first value of its lower-left entry), and a
// warp-slot that meets a flagged square takes the per-bin sum. kappa_ref is the
// flux-weighted mean opacity sum_i w_i kappa_i / sum w_i.
#include <math.h>

#include "rt_internal.cuh"

namespace rt {
namespace {

// FP64 G at the grid point (s, d) from the tracer's own (FP32) bin table
__device__ double lut_g(const NuEntry *nu, int na, double kref, double s, double d)
{
    const double n = (exp2(s) - 0x1p-20) / kref;
    const double dn = (exp2(d) - 0x1p-30) / kref;
    double acc = 0.0;
    for (int i = 0; i < na; ++i) {
        const double k = -(double)nu[i].nk * kLn2;
        const double w = exp2((double)nu[i].lf);
        const double g = w * exp(-k * fmax(n, 0.0));
        acc += dn > 0.0 ? g * -expm1(-k * dn) : g * k;
    }
    return dn > 0.0 ? acc / (kref * dn) : acc / kref;
}

// raw[j][i] = log2 G(s_i, d_j)
__global__ void k_lut_nodes(const NuEntry *nu, const DevScalars *sc, double kref, float *raw)
{
    const int na = sc->n_active;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)kLutNs * kLutNd;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / kLutNs), i = (int)(t % kLutNs);
        const double g = lut_g(nu, na, kref, kLutS0 + i / (double)kLutInvH, kLutD0 + j / (double)kLutInvH);
        raw[t] = (float)log2(g);
    }
}

// tab[j][i] = (raw[j][i] with the flag of square (i, j) in its lowest bit, raw[j][i + 1])
__global__ void k_lut_flags(const NuEntry *nu, const DevScalars *sc, double kref, const float *raw, float2 *tab,
                            double tol)
{
    const int na = sc->n_active;
    const double h = 1.0 / kLutInvH;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)kLutNs * kLutNd;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / kLutNs), i = (int)(t % kLutNs);
        unsigned bits = __float_as_uint(raw[t]) & ~1u;
        const float next = i + 1 < kLutNs ? raw[t + 1] : raw[t];
        if (i < kLutNs - 1 && j < kLutNd - 1) {
            // v_ab: node (s_{i+a}, d_{j+b})
            const double v00 = raw[t], v10 = raw[t + 1], v01 = raw[t + kLutNs], v11 = raw[t + kLutNs + 1];
            bool bad = !(isfinite(v00) && isfinite(v01) && isfinite(v10) && isfinite(v11));
            const double pts[5][2] = {{0.5, 0.5}, {0.5, 0.0}, {0.0, 0.5}, {1.0, 0.5}, {0.5, 1.0}};
            for (int k = 0; k < 5 && !bad; ++k) {
                const double ts = pts[k][0], td = pts[k][1];
                const double v0 = v00 + td * (v01 - v00), v1 = v10 + td * (v11 - v10);
                const double bil = v0 + ts * (v1 - v0);
                const double g = lut_g(nu, na, kref, kLutS0 + (i + ts) * h, kLutD0 + (j + td) * h);
                bad = !(g > 0.0) || fabs(exp2(bil - log2(g)) - 1.0) > 0.5 * tol;
            }
            if (bad) bits |= 1u;
        }
        tab[t] = make_float2(__uint_as_float(bits), next);
    }
}

}  // namespace

cudaError_t launch_build_lut(const NuEntry *nu, const DevScalars *sc, double kref, float *raw, float2 *tab, double tol,
                             cudaStream_t st)
{
    const int blocks = (int)(((long long)kLutNs * kLutNd + 255) / 256);
    k_lut_nodes<<<blocks, 256, 0, st>>>(nu, sc, kref, raw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_lut_flags<<<blocks, 256, 0, st>>>(nu, sc, kref, raw, tab, tol);
    return cudaGetLastError();
}

}  // namespace rt
