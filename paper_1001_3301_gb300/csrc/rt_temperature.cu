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
// 4 y + L(y) = ln a_rad - ln a: a cell reads T itself from the tabulated inverse of the
// left side (built once per table, each interval checked against the FP64 root) and
// takes Newton steps only in the intervals where that check failed.
#include <math.h>

#include <string>
#include <vector>

#include "rt_internal.cuh"
#include "rt_planck.cuh"

namespace rt {

constexpr int kTempNodes = 1024;
// The inverse table of T (E_R = 0) sits on the grid v = lg2 a_rad with spacing 2^-e:
// node i at v = (v_org + i) 2^-e, v_org an integer, at most kTempInvNodes nodes.
constexpr int kTempInvNodes = 2048;
// the context's table buffer: lkp [kTempNodes]; 8 constants (X(y_lo), X(y_hi), 2^e,
// v_org, the node count of the inverse table); then (16-byte aligned) the cubic
// coefficients of lkp [kTempNodes - 1] and of the inverse table [kTempInvNodes - 1],
// float4 each
constexpr int kTempConsts = kTempNodes;
constexpr int kTempCoefLkp = kTempConsts + 8;
constexpr int kTempCoefInv = kTempCoefLkp + 4 * (kTempNodes - 1);
constexpr int kTempTableFloats = kTempCoefInv + 4 * (kTempInvNodes - 1);
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

// ln kappa_P by the interpolation the cells use (cubic Hermite with Catmull-Rom
// tangents on the node table s, constant outside it), and its derivative, in FP64
__device__ double interp_d(const float *s, double y, double y0, double inv_dy, double *deriv = nullptr)
{
    double u = (y - y0) * inv_dy;
    if (!(u > 0.0) || u >= (double)(kTempNodes - 1)) {
        if (deriv) *deriv = 0.0;
        return !(u > 0.0) ? s[0] : s[kTempNodes - 1];
    }
    const int k = min((int)u, kTempNodes - 2);
    const double t = u - (double)k;
    const double p0 = s[k], p1 = s[k + 1];
    const double m0 = 0.5 * (p1 - s[k > 0 ? k - 1 : 0]) * (k > 0 ? 1.0 : 2.0);
    const double m1 = 0.5 * (s[k + 2 < kTempNodes ? k + 2 : kTempNodes - 1] - p0) * (k + 2 < kTempNodes ? 1.0 : 2.0);
    const double t2 = t * t, t3 = t2 * t;
    if (deriv)
        *deriv = ((6.0 * t2 - 6.0 * t) * p0 + (3.0 * t2 - 4.0 * t + 1.0) * m0 + (-6.0 * t2 + 6.0 * t) * p1 +
                  (3.0 * t2 - 2.0 * t) * m1) * inv_dy;
    return (2.0 * t3 - 3.0 * t2 + 1.0) * p0 + (t3 - 2.0 * t2 + t) * m0 + (-2.0 * t3 + 3.0 * t2) * p1 + (t3 - t2) * m1;
}

// the root y of 4 y + L(y) = x (bisection in [y0, y1], FP64); outside the table L is
// constant and the root is (x - L_end) / 4
__device__ double inverse_root(const float *s, double x, double y0, double y1, double inv_dy)
{
    const double x_lo = 4.0 * y0 + s[0], x_hi = 4.0 * y1 + s[kTempNodes - 1];
    if (x <= x_lo) return 0.25 * (x - s[0]);
    if (x >= x_hi) return 0.25 * (x - s[kTempNodes - 1]);
    double lo = y0, hi = y1;
    for (int it = 0; it < 64; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (4.0 * mid + interp_d(s, mid, y0, inv_dy) < x) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// The inverse of X(y) = 4 y + L(y) (y = ln T): with E_R = 0, Eq. 16 reads
// X(y) = ln a_rad - ln a. The nodes are uniform in v = lg2 a_rad (spacing 2^-e, node i
// at v = (v_org + i) 2^-e, X = v ln 2 - ln a), so a cell finds its interval and its
// offset t in it from lg2 a_rad with exact arithmetic. Per interval the cubic Hermite
// of T = e^y in t in [0, 1] with the exact slopes dT/dX = T / (4 + L'(y)), as
// coefficients (c0, c1, c2, c3) like k_hermite_coeffs. Each interval is checked at 8
// points against the FP64 root, evaluated the way a cell does (FP32 FMAs); where the
// cubic is off by more than 4e-7 of T the lowest bit of c3 is set, and the cells
// there polish ln T with Newton steps. One CTA.
__global__ void __launch_bounds__(1024) k_inverse_table(const float *lkp, float *consts, float4 *c, double y0,
                                                        double y1, double ln_a, int e, int v_org, int n_inv)
{
    __shared__ float s[kTempNodes];
    __shared__ double s_y[kTempInvNodes], s_m[kTempInvNodes];
    for (int i = threadIdx.x; i < kTempNodes; i += blockDim.x) s[i] = lkp[i];
    __syncthreads();
    const double inv_dy = (kTempNodes - 1) / (y1 - y0);
    const double hv = ldexp(1.0, -e), hx = hv * kLn2;
    auto node_x = [&](double i) { return (v_org + i) * hv * kLn2 - ln_a; };
    for (int i = threadIdx.x; i < n_inv; i += blockDim.x) {
        const double y = inverse_root(s, node_x(i), y0, y1, inv_dy);
        double dl = 0.0;
        interp_d(s, y, y0, inv_dy, &dl);
        s_y[i] = y;
        s_m[i] = hx * exp(y) / fmax(4.0 + dl, 0.5);  // dT/dt
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_inv - 1; k += blockDim.x) {
        const double p0 = exp(s_y[k]), p1 = exp(s_y[k + 1]), m0 = s_m[k], m1 = s_m[k + 1];
        const float c0 = (float)p0, c1 = (float)m0, c2 = (float)(3.0 * (p1 - p0) - 2.0 * m0 - m1);
        const float c3 = __uint_as_float(__float_as_uint((float)(2.0 * (p0 - p1) + m0 + m1)) & ~1u);
        bool bad = false;
        for (int j = 0; j < 8; ++j) {
            const float t = (j + 0.5f) * 0.125f;
            const float tc = fmaf(fmaf(fmaf(c3, t, c2), t, c1), t, c0);
            const double te = exp(inverse_root(s, node_x(k + (double)t), y0, y1, inv_dy));
            bad |= !(fabs((double)tc / te - 1.0) <= 4e-7);
        }
        c[k] = make_float4(c0, c1, c2, __uint_as_float(__float_as_uint(c3) | (bad ? 1u : 0u)));
    }
    if (threadIdx.x == 0) {
        consts[0] = (float)(4.0 * y0 + s[0]);
        consts[1] = (float)(4.0 * y1 + s[kTempNodes - 1]);
        consts[2] = (float)ldexp(1.0, e);
        consts[3] = (float)v_org;
        consts[4] = (float)n_inv;
    }
}

// Per-interval cubic coefficients of a node table (the cubic Hermite interpolation of
// interp_d, with the same tangents): on interval k, t in [0, 1],
//   f = c0 + t (c1 + t (c2 + t c3)),  c0 = p0, c1 = m0, c2 = 3 (p1 - p0) - 2 m0 - m1,
//   c3 = 2 (p0 - p1) + m0 + m1,
// so a cell evaluates one interval with one 16-byte load and three FMAs.
__global__ void k_hermite_coeffs(const float *s, float4 *c)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kTempNodes - 1; k += gridDim.x * blockDim.x) {
        const double p0 = s[k], p1 = s[k + 1];
        const double m0 = 0.5 * (p1 - s[k > 0 ? k - 1 : 0]) * (k > 0 ? 1.0 : 2.0);
        const double m1 = 0.5 * (s[k + 2 < kTempNodes ? k + 2 : kTempNodes - 1] - p0) * (k + 2 < kTempNodes ? 1.0 : 2.0);
        c[k] = make_float4((float)p0, (float)m0, (float)(3.0 * (p1 - p0) - 2.0 * m0 - m1),
                           (float)(2.0 * (p0 - p1) + m0 + m1));
    }
}

struct TempArgs {
    const float *a_rad;
    const float *e_rad;   // may be null (E_R = 0)
    float *t_out;
    const float *lkp;     // [kTempNodes] ln kappa_P on the uniform ln T grid
    const float *consts;  // X(y_lo), X(y_hi), 2^e, v_org, node count of the inverse table
    const float4 *c_lkp;  // [kTempNodes - 1] cubic coefficients of lkp per interval
    const float4 *c_inv;  // [n_inv - 1] cubic coefficients of T on the v = lg2 a_rad grid
    int vec;              // a_rad, e_rad (if any) and t_out are 16-byte aligned
    long long n;
    float y0, inv_dy;     // grid origin and 1 / spacing
    float ln_a;           // ln of the radiation constant a = 4 sigma / c
};

// ln kappa_P(e^y) and its derivative from the per-interval coefficients; lo, hi: the
// node values held outside the table.
__device__ __forceinline__ void interp_c(const float4 *c, float lo, float hi, float y, float y0, float inv_dy,
                                         float &L, float &dL)
{
    const float u = (y - y0) * inv_dy;
    if (!(u > 0.0f)) {  // below the table (or NaN): constant
        L = lo;
        dL = 0.0f;
        return;
    }
    if (u >= (float)(kTempNodes - 1)) {
        L = hi;
        dL = 0.0f;
        return;
    }
    const int k = min((int)u, kTempNodes - 2);
    const float t = u - (float)k;
    const float4 q = __ldg(c + k);
    L = fmaf(fmaf(fmaf(q.w, t, q.z), t, q.y), t, q.x);
    dL = fmaf(fmaf(3.0f * q.w, t, 2.0f * q.z), t, q.y) * inv_dy;
}

// e^y for |y| up to ~88 from the hardware 2^x: y log2(e) is formed as hi + lo with an
// FMA (Dekker's product, log2(e) split into two floats), so the rounding of the
// product does not grow with |y|; e^y = 2^hi (1 + lo ln 2) to about 2^-22.
__device__ __forceinline__ float exp_ex2(float y)
{
    constexpr float kL2eHi = 1.44269502162933349609375f;  // log2(e) rounded to float
    constexpr float kL2eLo = 1.92596298909109e-8f;        // log2(e) - kL2eHi
    const float hi = y * kL2eHi;
    const float lo = fmaf(y, kL2eHi, -hi) + y * kL2eLo;
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(hi));
    return fmaf(r, lo * 0.69314718055994530942f, r);
}

// the hardware log2 (absolute error ~2^-22)
__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ln x for x > 0 from the hardware log2
__device__ __forceinline__ float log_lg2(float x) { return lg2_approx(x) * 0.69314718055994530942f; }

// The table ends and the inverse table's grid, read once per thread.
struct TempConsts {
    float l_lo, l_hi, v_scale, v_org, u_max;
    int k_max;
};

// T of one cell (Eq. 16): a T^4 = E_R + a_rad / kappa_P(T); 0 where both sources vanish.
// ER: an E_R field is given (without one, E_R = 0 and every cell takes the table)
template <bool ER>
__device__ __forceinline__ float cell_temperature(const TempArgs &p, const TempConsts &k, float ar, float er)
{
    ar = fmaxf(ar, 0.0f);
    if constexpr (ER) er = fmaxf(er, 0.0f);
    if (!(ar > 0.0f) && (!ER || !(er > 0.0f))) return 0.0f;
    float L, dL, y;
    if (!ER || !(er > 0.0f)) {
        // X(y) = 4 y + L(y) = ln a_rad - ln a: T from the inverse table at v = lg2 a_rad.
        // The interval index from u = v 2^e - v_org, the offset in it from one FMA with
        // the exact integer v_org + k (so t keeps the full precision of v).
        const float lg = lg2_approx(ar);
        const float u = fmaf(lg, k.v_scale, -k.v_org);
        if (u > 0.0f && u < k.u_max) {
            const int kk = min((int)u, k.k_max);
            const float t = fmaf(lg, k.v_scale, -(k.v_org + (float)kk));
            const float4 q = __ldg(p.c_inv + kk);
            const float tc = fmaf(fmaf(fmaf(q.w, t, q.z), t, q.y), t, q.x);
            if (!(__float_as_uint(q.w) & 1u)) return tc;
            // an interval whose cubic failed its check: Newton steps on ln T from it,
            // until one is below 2e-6 (quadratic convergence: the root to FP32)
            const float x = fmaf(lg, 0.69314718055994530942f, -p.ln_a);
            y = log_lg2(tc);
            for (int it = 0; it < 24; ++it) {
                interp_c(p.c_lkp, k.l_lo, k.l_hi, y, p.y0, p.inv_dy, L, dL);
                float dy = -__fdividef(4.0f * y + L - x, fmaxf(4.0f + dL, 0.5f));  // the step, not the root
                dy = fminf(fmaxf(dy, -2.0f), 2.0f);
                y += dy;
                if (fabsf(dy) < 2e-6f) break;
            }
            return exp_ex2(y);
        }
        // beyond the table kappa_P is held constant: the root in closed form
        const float x = fmaf(lg, 0.69314718055994530942f, -p.ln_a);
        return exp_ex2(0.25f * (x - (u > 0.0f ? k.l_hi : k.l_lo)));
    }
    // Newton on F(y) = 4 y + ln a - ln(E_R + a_rad e^{-L}) from 300 K's opacity; it
    // converges quadratically: once a step is below 1e-5 the next one reaches the FP32
    // resolution of ln T, so one more step ends the solve
    interp_c(p.c_lkp, k.l_lo, k.l_hi, 5.7037825f, p.y0, p.inv_dy, L, dL);
    y = 0.25f * (logf(er + ar * expf(-L)) - p.ln_a);
    bool close = false;
    for (int it = 0; it < 24; ++it) {
        interp_c(p.c_lkp, k.l_lo, k.l_hi, y, p.y0, p.inv_dy, L, dL);
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
    return expf(y);
}

// Four cells per thread and iteration, moved as 16-byte vectors where the fields allow
// (p.vec): one load in flight per thread would leave HBM latency-bound. ER: p.e_rad is
// given (a separate instance, so the common E_R = 0 call carries none of its tests).
template <bool ER>
__global__ void __launch_bounds__(256) k_dust_temperature(const TempArgs p)
{
    TempConsts k;
    k.l_lo = __ldg(p.lkp);
    k.l_hi = __ldg(p.lkp + kTempNodes - 1);
    k.v_scale = __ldg(p.consts + 2);
    k.v_org = __ldg(p.consts + 3);
    k.k_max = (int)__ldg(p.consts + 4) - 2;
    k.u_max = (float)(k.k_max + 1);
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = p.vec ? p.n / 4 : 0;
    // D quads in flight per thread: slot d holds the inputs of quad v + d stride, and is
    // refilled with quad v + (d + D) stride before quad v + d stride is solved (one with
    // an E_R field: its Newton solve needs the registers)
    constexpr int D = ER ? 1 : 2;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 an[D], en[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const long long v = tid + d * stride;
        an[d] = v < n4 ? __ldg(reinterpret_cast<const float4 *>(p.a_rad) + v) : zero4;
        en[d] = (ER && v < n4) ? __ldg(reinterpret_cast<const float4 *>(p.e_rad) + v) : zero4;
    }
    for (long long v0 = tid; v0 < n4; v0 += D * stride) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const long long v = v0 + d * stride;
            if (v >= n4) break;
            const float4 a4 = an[d], e4 = en[d];
            const long long vn = v + D * stride;
            if (vn < n4) {
                an[d] = __ldg(reinterpret_cast<const float4 *>(p.a_rad) + vn);
                if constexpr (ER) en[d] = __ldg(reinterpret_cast<const float4 *>(p.e_rad) + vn);
            }
            float4 t4;
            t4.x = cell_temperature<ER>(p, k, a4.x, e4.x);
            t4.y = cell_temperature<ER>(p, k, a4.y, e4.y);
            t4.z = cell_temperature<ER>(p, k, a4.z, e4.z);
            t4.w = cell_temperature<ER>(p, k, a4.w, e4.w);
            reinterpret_cast<float4 *>(p.t_out)[v] = t4;
        }
    }
    for (long long c = 4 * n4 + tid; c < p.n; c += stride)
        p.t_out[c] = cell_temperature<ER>(p, k, p.a_rad[c], ER ? p.e_rad[c] : 0.0f);
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
    const double sigma = 2.0 * pow(kPi, 5) * pow(kKB, 4) / (15.0 * kH * kH * kH * kC * kC);
    const double ln_a = log(4.0 * sigma / kC);
    float *&lkp = ctx_temp_table(ctx);
    unsigned long long &fp = ctx_temp_fingerprint(ctx);
    if (!lkp || fp != in.table_fingerprint) {
        if (!lkp && cudaMalloc(&lkp, sizeof(float) * kTempTableFloats) != cudaSuccess) {
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
        // the inverse table's grid in v = lg2 a_rad: the finest spacing 2^-e whose nodes
        // (whole steps from v_org) cover X(y_lo)..X(y_hi) within kTempInvNodes
        float ends[2];
        if (cudaMemcpyAsync(&ends[0], lkp, sizeof(float), cudaMemcpyDeviceToHost, in.stream) != cudaSuccess ||
            cudaMemcpyAsync(&ends[1], lkp + kTempNodes - 1, sizeof(float), cudaMemcpyDeviceToHost, in.stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(in.stream) != cudaSuccess)
            return ctx_fail(ctx, RT_ERR_CUDA, "Planck-mean table ends");
        const double v_lo = (4.0 * kTempLnLo + ends[0] + ln_a) / kLn2, v_hi = (4.0 * kTempLnHi + ends[1] + ln_a) / kLn2;
        int e = 6, v_org = 0, n_inv = 0;
        for (; e >= 0; --e) {
            v_org = (int)floor(ldexp(v_lo, e));
            n_inv = (int)ceil(ldexp(v_hi, e)) - v_org + 1;
            if (n_inv <= kTempInvNodes) break;
        }
        if (e < 0 || n_inv < 2) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "Planck mean outside the tabulated range");
        k_inverse_table<<<1, 1024, 0, in.stream>>>(lkp, lkp + kTempConsts, reinterpret_cast<float4 *>(lkp + kTempCoefInv),
                                                   kTempLnLo, kTempLnHi, ln_a, e, v_org, n_inv);
        k_hermite_coeffs<<<4, 256, 0, in.stream>>>(lkp, reinterpret_cast<float4 *>(lkp + kTempCoefLkp));
        if (cudaGetLastError() != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, "inverse temperature table");
        fp = in.table_fingerprint;
    }
    TempArgs p;
    p.a_rad = a_rad;
    p.e_rad = e_rad;
    p.t_out = t_dust;
    p.lkp = lkp;
    p.consts = lkp + kTempConsts;
    p.c_lkp = reinterpret_cast<const float4 *>(lkp + kTempCoefLkp);
    p.c_inv = reinterpret_cast<const float4 *>(lkp + kTempCoefInv);
    p.vec = ((reinterpret_cast<size_t>(a_rad) | reinterpret_cast<size_t>(e_rad) | reinterpret_cast<size_t>(t_dust)) % 16) == 0;
    p.n = in.ncells;
    p.y0 = (float)kTempLnLo;
    p.inv_dy = (float)((kTempNodes - 1) / (kTempLnHi - kTempLnLo));
    p.ln_a = (float)ln_a;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, in.dev);
    long long blocks = (in.ncells / 4 + 255) / 256;
    if (blocks > 8LL * nsm) blocks = 8LL * nsm;
    if (blocks < 1) blocks = 1;
    if (e_rad) k_dust_temperature<true><<<(unsigned)blocks, 256, 0, in.stream>>>(p);
    else k_dust_temperature<false><<<(unsigned)blocks, 256, 0, in.stream>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, std::string("temperature kernel: ") + cudaGetErrorString(e));
    return RT_OK;
}

}  // extern "C"
