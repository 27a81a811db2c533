// Set-up kernels: per-bin stellar fluxes (Eq. 20), geometry tables, and the FP64
// energy reduction. All run once per configuration change (or once per energy
// request) and are tiny next to the tracer.
#include <cuda_bf16.h>
#include <math.h>

#include "rt_internal.cuh"
#include "rt_planck.cuh"

namespace rt {
namespace {

// One warp per bin (the block has RT_MAX_NU / 4 warps, each doing four bins),
// then thread 0 compacts the bins with kappa > 0 into the tracer's table.
__global__ void k_setup_bins(int n_nu, const double *nu_mid, const double *kappa, double t_star,
                             double r_star, int kappa_bf16, double *f_bin, NuEntry *nu,
                             float *kap, double2 *nu64, DevScalars *sc, int *order_out)
{
    __shared__ double s_f[RT_MAX_NU];
    __shared__ double s_k[RT_MAX_NU];
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x >> 5; i < n_nu; i += blockDim.x >> 5) {
        // Eq. 20 with B_nu the specific intensity: F_i = pi int B_nu dnu over the bin
        // = 2 pi (k T)^4 / (h^3 c^2) int_{x_lo}^{x_hi} t^3/(e^t-1) dt.
        const double lo = (i == 0) ? 0.0 : 0.5 * (nu_mid[i - 1] + nu_mid[i]);
        const double hi = (i == n_nu - 1) ? INFINITY : 0.5 * (nu_mid[i] + nu_mid[i + 1]);
        const double kt_h = kKB * t_star / kH;
        const double pref = 2.0 * kPi * pow(kKB * t_star, 4) / (kH * kH * kH * kC * kC);
        const double f = pref * planck_band_warp(lo / kt_h, hi / kt_h, lane);
        double k = kappa[i];
        if (kappa_bf16) k = (double)__bfloat162float(__float2bfloat16_rn((float)k));
        if (lane == 0) {
            s_f[i] = f;
            s_k[i] = k;
            f_bin[i] = f;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double fmax = 0.0, ftr = 0.0;
    for (int b = 0; b < n_nu; ++b) fmax = fmax > s_f[b] ? fmax : s_f[b];
    // bins with kappa > 0, sorted by kappa ascending (insertion sort, <= 128 bins);
    // the tracer classifies contiguous ranges of this order per warp
    int order[RT_MAX_NU];
    int na = 0;
    for (int b = 0; b < n_nu; ++b) {
        if (s_k[b] > 0.0) {
            int pos = na++;
            while (pos > 0 && s_k[order[pos - 1]] > s_k[b]) {
                order[pos] = order[pos - 1];
                --pos;
            }
            order[pos] = b;
        } else {
            ftr += s_f[b];
        }
    }
    for (int a = 0; a < na; ++a) {
        const int b = order[a];
        if (order_out) order_out[a] = b;
        nu[a].nk = (float)(-s_k[b] * kLog2e);
        nu[a].lf = (float)log2(s_f[b] / fmax);
        kap[a] = (float)s_k[b];
        nu64[a] = make_double2(s_k[b], s_f[b] / fmax);
    }
    int pad = ((na + kNuPad - 1) / kNuPad) * kNuPad;
    if (pad < kNuPad) pad = kNuPad;
    for (int b = na; b < pad; ++b) {
        nu[b].nk = -1.0f;
        nu[b].lf = -INFINITY;
        kap[b] = 0.0f;
        nu64[b] = make_double2(1.0, 0.0);
    }
    sc->f_max = fmax;
    sc->f_transparent = ftr;
    sc->r2 = r_star * r_star;
    sc->n_active = na;
    sc->nnu_pad = pad;
}

// Series rows of the bins thin along whole rays (layout at kThinTerms in
// rt_internal.cuh), one block of one warp per row b = 0..RT_MAX_NU: s_b = kappa_{b-1},
// C_k(b) = (-1)^{k+1} / k! sum_{i<b} w_i (kappa_i / s_b)^k and S_0(b) = sum_{i<b} w_i,
// in FP64 from the FP32 table the tracer uses (kappa_i = -nk_i ln 2, w_i = 2^lf_i).
__global__ void k_thin_table(const NuEntry *nu, const DevScalars *sc, float *thin)
{
    const int b = blockIdx.x, lane = threadIdx.x;
    const int na = sc->n_active;
    float *row = thin + (size_t)b * kThinStride;
    if (b == 0 || b > na) {
        if (lane < kThinStride) row[lane] = 0.0f;
        return;
    }
    const double s = -(double)nu[b - 1].nk * kLn2;
    double m[kThinTerms + 1];
#pragma unroll
    for (int k = 0; k <= kThinTerms; ++k) m[k] = 0.0;
    for (int i = lane; i < b; i += 32) {
        const double r = -(double)nu[i].nk * kLn2 / s;
        double p = exp2((double)nu[i].lf);
        m[0] += p;
#pragma unroll
        for (int k = 1; k <= kThinTerms; ++k) {
            p *= r;
            m[k] += p;
        }
    }
#pragma unroll
    for (int k = 0; k <= kThinTerms; ++k)
        for (int o = 16; o > 0; o >>= 1) m[k] += __shfl_xor_sync(0xffffffffu, m[k], o);
    if (lane == 0) {
        row[0] = (float)s;
        double fact = 1.0;
#pragma unroll
        for (int k = 1; k <= kThinTerms; ++k) {
            fact *= k;
            row[k] = (float)(((k & 1) ? m[k] : -m[k]) / fact);
        }
        row[kThinTerms + 1] = (float)m[0];
        for (int k = kThinTerms + 2; k < kThinStride; ++k) row[k] = 0.0f;
    }
}

// Per-radius and per-ray tables. Gq = 3 R*^2 F_max / (r+^3 - r-^3) turns the
// per-ray sum of F_i/F_max e^-tau (1-e^-dtau) into power per volume; Ga0 = Gq dr / c
// is the rho -> 0 force factor.
__global__ void k_setup_geometry(int nr, int ntheta, int nphi, const double *r_if,
                                 const double *theta_if, const double *phi_if, float4 *rtab,
                                 RadRow64 *rtab64, double *domega, float *domega32,
                                 const DevScalars *sc)
{
    const long long nrays = (long long)ntheta * nphi;
    const long long n = nrays > nr ? nrays : nr;
    const double gscale = 3.0 * sc->r2 * sc->f_max;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < nr) {
            const double r0 = r_if[t], r1 = r_if[t + 1];
            const double dr = r1 - r0;
            const double d3 = dr * (r1 * r1 + r1 * r0 + r0 * r0);  // r1^3 - r0^3
            const double gq = gscale / d3;
            const double ga0 = gq * dr / kC;
            rtab[t] = make_float4((float)dr, (float)gq, (float)ga0, 0.0f);
            rtab64[t] = RadRow64{dr, gq, ga0, 0.0};
        }
        if (t < nrays) {
            const int it = (int)(t % ntheta);
            const int ip = (int)(t / ntheta);
            const double dom = (cos(theta_if[it]) - cos(theta_if[it + 1])) * (phi_if[ip + 1] - phi_if[ip]);
            domega[t] = dom;
            domega32[t] = (float)dom;
        }
    }
}

__device__ double block_sum(double v, double *s_red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s_red[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? s_red[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;  // valid in thread 0
}

__global__ void k_sum_domega(long long nrays, const double *domega, double t_star,
                             DevScalars *sc)
{
    __shared__ double s_red[32];
    double v = 0.0;
    for (long long j = threadIdx.x; j < nrays; j += blockDim.x) v += domega[j];
    v = block_sum(v, s_red);
    if (threadIdx.x == 0) {
        const double sigma = 2.0 * pow(kPi, 5) * pow(kKB, 4) / (15.0 * kH * kH * kH * kC * kC);
        sc->sum_domega = v;
        sc->l_grid = sc->r2 * sigma * pow(t_star, 4) * v;
    }
}

__global__ void k_energy_reduce(const double2 *partials, long long ntiles, const DevScalars *sc,
                                rt_energy *out)
{
    __shared__ double s_red[32];
    double sa = 0.0, se = 0.0;
    for (long long t = threadIdx.x; t < ntiles; t += blockDim.x) {
        sa += partials[t].x;
        se += partials[t].y;
    }
    sa = block_sum(sa, s_red);
    se = block_sum(se, s_red);
    if (threadIdx.x == 0) {
        const double scale = sc->r2 * sc->f_max;
        rt_energy e;
        e.e_abs = scale * sa;
        e.e_esc = scale * se + sc->r2 * sc->f_transparent * sc->sum_domega;
        e.l_star = sc->l_grid;
        e.rel_err = (e.e_abs + e.e_esc) / e.l_star - 1.0;
        *out = e;
    }
}

}  // namespace

cudaError_t launch_setup_bins(int n_nu, const double *nu_mid_dev, const double *kappa_dev,
                              double t_star, double r_star, int kappa_bf16, double *f_bin_dev,
                              NuEntry *nu_dev, float *kap_dev, double2 *nu64_dev,
                              DevScalars *sc_dev, cudaStream_t stream, int *order_dev)
{
    k_setup_bins<<<1, 32 * (RT_MAX_NU / 4), 0, stream>>>(n_nu, nu_mid_dev, kappa_dev, t_star, r_star,
                                              kappa_bf16, f_bin_dev, nu_dev, kap_dev, nu64_dev,
                                              sc_dev, order_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static_assert(kThinStride >= kThinTerms + 2, "a row holds s, C_1..C_K and S_0");
    k_thin_table<<<RT_MAX_NU + 1, 32, 0, stream>>>(nu_dev, sc_dev, kap_dev + kKapTable);
    return cudaGetLastError();
}

cudaError_t launch_setup_geometry(int nr, int ntheta, int nphi, const double *r_if_dev,
                                  const double *theta_if_dev, const double *phi_if_dev,
                                  double t_star, float4 *rtab, RadRow64 *rtab64, double *domega,
                                  float *domega32, DevScalars *sc_dev, cudaStream_t stream)
{
    const long long nrays = (long long)ntheta * nphi;
    const long long n = nrays > nr ? nrays : nr;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_setup_geometry<<<blocks, 256, 0, stream>>>(nr, ntheta, nphi, r_if_dev, theta_if_dev,
                                                 phi_if_dev, rtab, rtab64, domega, domega32, sc_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_domega<<<1, 1024, 0, stream>>>(nrays, domega, t_star, sc_dev);
    return cudaGetLastError();
}

cudaError_t launch_energy_reduce(const double2 *partials, long long ntiles,
                                 const DevScalars *sc_dev, rt_energy *out_dev, cudaStream_t stream)
{
    k_energy_reduce<<<1, 1024, 0, stream>>>(partials, ntiles, sc_dev, out_dev);
    return cudaGetLastError();
}

}  // namespace rt
