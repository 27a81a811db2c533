// Dust temperature from the irradiation (Sect. 2.2, Eq. 16, in the frequency-
// dependent form of Sect. 2.3): with the stellar fluxes of every bin,
//     a T^4 = E_R + sum_i kappa_i |F_i| / (c kappa_P(T)),
// and over a cell sum_i kappa_i F_i = q_abs / rho = c a_rad, so
//     a T^4 = E_R + a_rad / kappa_P(T)
// per cell, from the tracer's radial acceleration (finite also where rho = 0).
// kappa_P(T) = sum_i kappa_i B_i(T) / sum_i B_i(T) is the Planck mean of the bin
// table, B_i(T) the Planck integral over bin i (the bins of Eq. 20 at T).
//
// The mean is tabulated once per table on 1024 points of ln T in [0, ln 1e5]
// (FP64 quadrature, stored as ln kappa_P) and read with cubic Hermite interpolation
// (Catmull-Rom tangents); outside the range it is held constant. Each cell solves
// 4 y + ln a = ln(E_R + a_rad e^{-L(y)}), y = ln T, L = ln kappa_P, by Newton's
// method in FP32 (the derivative 4 + w L'(y), 0 <= w <= 1, is positive wherever
// the mean grows slower than T^4). Where E_R = 0 the equation is
// 4 y + L(y) = ln a_rad - ln a: a cell reads y from the tabulated inverse of the left
// side (built once per table) and polishes it with a Newton step.
#include <math.h>

#include <string>
#include <vector>

#include "rt_internal.cuh"
#include "rt_planck.cuh"

namespace rt {

constexpr int kTempNodes = 1024;
constexpr double kTempLnLo = 0.0;                    // ln 1 K
constexpr double kTempLnHi = 11.512925464970229;     // ln 1e5 K

namespace {

// Planck mean of the table at temperature exp(y[n]); one warp per node, the bins'
// band integrals in FP64. kp_out[n] = kappa_P (double) and lkp[n] = ln kappa_P.
__global__ void k_planck_mean(int n_nodes, const double *t_nodes, int n_nu, const double *nu_mid,
                              const double *kappa, int n_t, const double *t_grid, double *kp_out, float *lkp)
{
    const int lane = threadIdx.x & 31;
    const int node = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (node >= n_nodes) return;
    const double t = t_nodes[node];
    const double kt_h = kKB * t / kH;
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n_nu; ++i) {
        const double lo = (i == 0) ? 0.0 : 0.5 * (nu_mid[i - 1] + nu_mid[i]);
        const double hi = (i == n_nu - 1) ? INFINITY : 0.5 * (nu_mid[i] + nu_mid[i + 1]);
        const double b = planck_band_warp(lo / kt_h, hi / kt_h, lane);
        num += kappa_at(kappa + (size_t)i * n_t, n_t, t_grid, t) * b;
        den += b;
    }
    if (lane == 0) {
        const double kp = den > 0.0 ? num / den : 0.0;
        if (kp_out) kp_out[node] = kp;
        if (lkp) lkp[node] = (float)log(kp > 1e-300 ? kp : 1e-300);
    }
}

// The inverse of X(y) = 4 y + L(y) (y = ln T, L = ln kappa_P by the interpolation the
// cells use, held constant outside the table) on kTempNodes uniform points of X between
// X(y_lo) and X(y_hi): with E_R = 0, Eq. 16 reads X(y) = ln a_rad - ln a, so a cell's ln T
// is this table at its X, polished by a Newton step. One CTA; bisection in FP64.
// inv[n] = y, inv[n + 0..1] after the table: X(y_lo), X(y_hi).
__device__ double interp_d(const float *s, double y, double y0, double inv_dy)
{
    double u = (y - y0) * inv_dy;
    if (!(u > 0.0)) return s[0];
    if (u >= (double)(kTempNodes - 1)) return s[kTempNodes - 1];
    const int k = min((int)u, kTempNodes - 2);
    const double t = u - (double)k;
    const double p0 = s[k], p1 = s[k + 1];
    const double m0 = 0.5 * (p1 - s[k > 0 ? k - 1 : 0]) * (k > 0 ? 1.0 : 2.0);
    const double m1 = 0.5 * (s[k + 2 < kTempNodes ? k + 2 : kTempNodes - 1] - p0) * (k + 2 < kTempNodes ? 1.0 : 2.0);
    const double t2 = t * t, t3 = t2 * t;
    return (2.0 * t3 - 3.0 * t2 + 1.0) * p0 + (t3 - 2.0 * t2 + t) * m0 + (-2.0 * t3 + 3.0 * t2) * p1 + (t3 - t2) * m1;
}

__global__ void __launch_bounds__(1024) k_inverse_table(const float *lkp, float *inv, double y0, double y1)
{
    __shared__ float s[kTempNodes];
    for (int i = threadIdx.x; i < kTempNodes; i += blockDim.x) s[i] = lkp[i];
    __syncthreads();
    const double inv_dy = (kTempNodes - 1) / (y1 - y0);
    const double x_lo = 4.0 * y0 + s[0], x_hi = 4.0 * y1 + s[kTempNodes - 1];
    for (int i = threadIdx.x; i < kTempNodes; i += blockDim.x) {
        const double x = x_lo + (x_hi - x_lo) * i / (kTempNodes - 1);
        double lo = y0, hi = y1;
        for (int it = 0; it < 64; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (4.0 * mid + interp_d(s, mid, y0, inv_dy) < x) lo = mid;
            else hi = mid;
        }
        inv[i] = (float)(0.5 * (lo + hi));
    }
    if (threadIdx.x == 0) {
        inv[kTempNodes] = (float)x_lo;
        inv[kTempNodes + 1] = (float)x_hi;
    }
}

struct TempArgs {
    const float *a_rad;
    const float *e_rad;   // may be null (E_R = 0)
    float *t_out;
    const float *lkp;     // [kTempNodes] ln kappa_P on the uniform ln T grid
    const float *inv;     // [kTempNodes + 2] ln T on the uniform grid of 4 ln T + ln kappa_P
    long long n;
    float y0, inv_dy;     // grid origin and 1 / spacing
    float ln_a;           // ln of the radiation constant a = 4 sigma / c
};

// ln kappa_P(e^y) and its derivative by cubic Hermite interpolation
__device__ __forceinline__ void interp(const float *s, float y, float y0, float inv_dy, float &L, float &dL)
{
    float u = (y - y0) * inv_dy;
    if (!(u > 0.0f)) {  // below the table (or NaN): constant
        L = s[0];
        dL = 0.0f;
        return;
    }
    if (u >= (float)(kTempNodes - 1)) {
        L = s[kTempNodes - 1];
        dL = 0.0f;
        return;
    }
    const int k = min((int)u, kTempNodes - 2);
    const float t = u - (float)k;
    const float p0 = s[k], p1 = s[k + 1];
    const float m0 = 0.5f * (p1 - s[k > 0 ? k - 1 : 0]) * (k > 0 ? 1.0f : 2.0f);
    const float m1 = 0.5f * (s[k + 2 < kTempNodes ? k + 2 : kTempNodes - 1] - p0) * (k + 2 < kTempNodes ? 1.0f : 2.0f);
    const float t2 = t * t, t3 = t2 * t;
    L = (2.0f * t3 - 3.0f * t2 + 1.0f) * p0 + (t3 - 2.0f * t2 + t) * m0 + (-2.0f * t3 + 3.0f * t2) * p1 +
        (t3 - t2) * m1;
    dL = ((6.0f * t2 - 6.0f * t) * p0 + (3.0f * t2 - 4.0f * t + 1.0f) * m0 + (-6.0f * t2 + 6.0f * t) * p1 +
          (3.0f * t2 - 2.0f * t) * m1) *
         inv_dy;
}

__global__ void __launch_bounds__(256) k_dust_temperature(const TempArgs p)
{
    __shared__ float s[kTempNodes], s_inv[kTempNodes + 2];
    for (int i = threadIdx.x; i < kTempNodes; i += blockDim.x) s[i] = p.lkp[i];
    for (int i = threadIdx.x; i < kTempNodes + 2; i += blockDim.x) s_inv[i] = p.inv[i];
    __syncthreads();
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < p.n;
         c += (long long)gridDim.x * blockDim.x) {
        const float ar = fmaxf(p.a_rad[c], 0.0f);
        const float er = p.e_rad ? fmaxf(p.e_rad[c], 0.0f) : 0.0f;
        if (!(ar > 0.0f) && !(er > 0.0f)) {
            p.t_out[c] = 0.0f;
            continue;
        }
        float L, dL, y;
        if (!(er > 0.0f)) {
            // X(y) = 4 y + L(y) = ln a_rad - ln a: the inverse table, then Newton steps
            // until one is below 2e-6 (quadratic convergence: one step from the table)
            const float x = logf(ar) - p.ln_a;
            const float x_lo = s_inv[kTempNodes], x_hi = s_inv[kTempNodes + 1];
            if (x <= x_lo) {
                y = 0.25f * (x - s[0]);
            } else if (x >= x_hi) {
                y = 0.25f * (x - s[kTempNodes - 1]);
            } else {
                float yi, dyi;
                interp(s_inv, x, x_lo, (float)(kTempNodes - 1) / (x_hi - x_lo), yi, dyi);
                y = yi;
            }
            for (int it = 0; it < 24; ++it) {
                interp(s, y, p.y0, p.inv_dy, L, dL);
                float dy = -__fdividef(4.0f * y + L - x, fmaxf(4.0f + dL, 0.5f));  // the step, not the root: fast divide
                dy = fminf(fmaxf(dy, -2.0f), 2.0f);
                y += dy;
                if (fabsf(dy) < 2e-6f) break;
            }
        } else {
            // Newton on F(y) = 4 y + ln a - ln(E_R + a_rad e^{-L}) from 300 K's opacity;
            // it converges quadratically: once a step is below 1e-5 the next one reaches
            // the FP32 resolution of ln T, so one more step ends the solve
            interp(s, 5.7037825f, p.y0, p.inv_dy, L, dL);
            y = 0.25f * (logf(er + ar * expf(-L)) - p.ln_a);
            bool close = false;
            for (int it = 0; it < 24; ++it) {
                interp(s, y, p.y0, p.inv_dy, L, dL);
                const float src = ar * expf(-L);
                const float rhs = er + src;
                const float f = 4.0f * y + p.ln_a - logf(rhs);
                const float fp = 4.0f + dL * __fdividef(src, rhs);
                float dy = -__fdividef(f, fmaxf(fp, 0.5f));
                dy = fminf(fmaxf(dy, -2.0f), 2.0f);
                y += dy;
                if (close) break;
                close = fabsf(dy) < 1e-5f;
            }
        }
        p.t_out[c] = expf(y);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host: the table belongs to the context (built on first use, per table)
// ---------------------------------------------------------------------------
namespace {

int planck_means(const CtxInfo &in, const std::vector<double> &t_nodes, double *kp_host, float *lkp_dev,
                 cudaStream_t st, std::string &err)
{
    const int n = (int)t_nodes.size();
    // the table's opacities: one value per bin, or rows on a temperature grid
    const int n_t = in.n_t > 0 ? in.n_t : 1;
    const double *kap_h = in.n_t > 0 ? in.kappa_t_h : in.kappa_h;
    double *tn = nullptr, *nu = nullptr, *ka = nullptr, *kp = nullptr, *tg = nullptr;
    bool ok = cudaMalloc(&tn, sizeof(double) * n) == cudaSuccess &&
              cudaMalloc(&nu, sizeof(double) * in.n_nu) == cudaSuccess &&
              cudaMalloc(&ka, sizeof(double) * in.n_nu * n_t) == cudaSuccess &&
              cudaMalloc(&tg, sizeof(double) * n_t) == cudaSuccess &&
              cudaMalloc(&kp, sizeof(double) * n) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(tn, t_nodes.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(nu, in.nu_h, sizeof(double) * in.n_nu, cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(ka, kap_h, sizeof(double) * in.n_nu * n_t, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok && in.n_t > 0)
        ok = cudaMemcpyAsync(tg, in.t_grid_h, sizeof(double) * n_t, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok) {
        k_planck_mean<<<(n + 7) / 8, 256, 0, st>>>(n, tn, in.n_nu, nu, ka, n_t, tg, kp, lkp_dev);
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (ok && kp_host) ok = cudaMemcpyAsync(kp_host, kp, sizeof(double) * n, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) err = std::string("Planck-mean kernel: ") + cudaGetErrorString(cudaGetLastError());
    cudaFree(tn);
    cudaFree(nu);
    cudaFree(ka);
    cudaFree(tg);
    cudaFree(kp);
    return ok ? RT_OK : RT_ERR_CUDA;
}

}  // namespace
}  // namespace rt

using namespace rt;

extern "C" {

int rt_planck_mean_opacity(rt_ctx *ctx, double t, double *kappa_p)
{
    if (!ctx || !kappa_p) return RT_ERR_INVALID_ARG;
    CtxInfo in;
    ctx_info(ctx, &in);
    if (!in.configured) return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "call rt_set_star and rt_set_opacity_table first");
    if (!(t > 0.0) || !isfinite(t)) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "t must be finite and > 0");
    if (cudaSetDevice(in.dev) != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, "cudaSetDevice");
    std::string err;
    const int rc = planck_means(in, std::vector<double>{t}, kappa_p, nullptr, in.stream, err);
    return rc == RT_OK ? RT_OK : ctx_fail(ctx, rc, err);
}

int rt_dust_temperature(rt_ctx *ctx, const float *a_rad, const float *e_rad, float *t_dust)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    CtxInfo in;
    ctx_info(ctx, &in);
    if (!in.configured) return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "call rt_set_star and rt_set_opacity_table first");
    if (!a_rad || !t_dust) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "a_rad and t_dust must be non-NULL");
    if (cudaSetDevice(in.dev) != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, "cudaSetDevice");
    float *&lkp = ctx_temp_table(ctx);
    unsigned long long &fp = ctx_temp_fingerprint(ctx);
    if (!lkp || fp != in.table_fingerprint) {
        if (!lkp && cudaMalloc(&lkp, sizeof(float) * (2 * kTempNodes + 2)) != cudaSuccess) {
            lkp = nullptr;
            cudaGetLastError();
            return ctx_fail(ctx, RT_ERR_NO_MEMORY, "Planck-mean table");
        }
        std::vector<double> tn(kTempNodes);
        for (int i = 0; i < kTempNodes; ++i)
            tn[i] = exp(kTempLnLo + (kTempLnHi - kTempLnLo) * i / (kTempNodes - 1));
        std::string err;
        const int rc = planck_means(in, tn, nullptr, lkp, in.stream, err);
        if (rc != RT_OK) return ctx_fail(ctx, rc, err);
        k_inverse_table<<<1, 1024, 0, in.stream>>>(lkp, lkp + kTempNodes, kTempLnLo, kTempLnHi);
        if (cudaGetLastError() != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, "inverse temperature table");
        fp = in.table_fingerprint;
    }
    const double sigma = 2.0 * pow(kPi, 5) * pow(kKB, 4) / (15.0 * kH * kH * kH * kC * kC);
    TempArgs p;
    p.a_rad = a_rad;
    p.e_rad = e_rad;
    p.t_out = t_dust;
    p.lkp = lkp;
    p.inv = lkp + kTempNodes;
    p.n = in.ncells;
    p.y0 = (float)kTempLnLo;
    p.inv_dy = (float)((kTempNodes - 1) / (kTempLnHi - kTempLnLo));
    p.ln_a = (float)log(4.0 * sigma / kC);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, in.dev);
    long long blocks = (in.ncells + 255) / 256;
    if (blocks > 8LL * nsm) blocks = 8LL * nsm;
    if (blocks < 1) blocks = 1;
    k_dust_temperature<<<(unsigned)blocks, 256, 0, in.stream>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, std::string("temperature kernel: ") + cudaGetErrorString(e));
    return RT_OK;
}

}  // extern "C"
