// One implicit flux-limited-diffusion step of the radiation energy density E = E_R
// (Sect. 2.1, Eqs. 7-15) with the absorbed stellar power as source (Eq. 15):
//     (E' - E) / dt = f_c (div(D grad E') + q_abs),   f_c = 1 / (c_V rho / (4 a T^3) + 1),
//     D = lambda c / (kappa_R rho),  lambda = (2 + R) / (6 + 3 R + R^2),  R = |grad E| / (kappa_R rho E),
// coefficients frozen at the old state and written D = c (2 s + g) / (6 s^2 + 3 s g + g^2)
// with s = kappa_R rho, g = |grad E| / E (finite as s -> 0; D = 0 where s = g = 0).
//
// Finite volumes on the spherical grid: a face carries the harmonic mean of its two
// cells' D times area over centre distance; no flux through the inner radius or the
// theta ends; E = a T_bg^4 half a cell beyond the outer radius; periodic in phi
// (nphi > 1). Lengths are in units of the outer radius L (r^3 in cm overflows FP32)
// and the system is divided by c L^2, so with tau = c dt / L
//     (V'/(tau f_c)) (E'_c - E_c) + sum_faces F_f A'/d' (E'_c - E'_nb) = V' q_c L / c,
// F = (2 s' + g') / (6 s'^2 + 3 s' g' + g'^2), s' = kappa_R rho L, g' = L |grad E| / E.
//
// The matrix is symmetric positive definite. It is applied matrix-free and solved
// by Jacobi-preconditioned conjugate gradients inside mixed-precision iterative
// refinement (FP32 vectors, FP64 reductions, every scalar of the iteration kept on
// the device), from E_old, until the last refinement changed no cell by more than
// tol relative.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "rt_internal.cuh"
#include "rt_planck.cuh"

namespace rt {

constexpr int kRossNodes = 1024;
constexpr double kRossLnLo = 0.0, kRossLnHi = 11.512925464970229;  // ln 1 K .. ln 1e5 K

struct FldState {
    long long cap = 0;
    float *buf = nullptr;  // F, tc, b0, w[3], s, 1/dg, b, d, r, p, q, z: 15 n floats, then BF16
                           // copies of s, w[3], 1/dg (5 n halves) for the finest V-cycle
    float *mg_buf = nullptr;              // coarse levels: s, w[3], 1/dg, b, x each
    std::vector<int> mg_dims;             // (nr, ntheta, nphi) of every level, finest first
    double *part = nullptr, *scal = nullptr;
    unsigned *bad = nullptr, *count = nullptr;
    int part_cap = 0;
    float *geo = nullptr;  // axis tables
    float *lkr = nullptr;  // ln kappa_R on the ln T nodes
    unsigned long long lkr_fp = 0;
    bool lkr_valid = false;
    // the solve runs on a private stream (after the context's stream), so that its
    // inner-iteration bursts can be captured and replayed as a CUDA graph
    cudaStream_t gs = nullptr;
    cudaEvent_t ev_in = nullptr;
    cudaGraphExec_t burst = nullptr;
    const void *burst_x = nullptr, *burst_buf = nullptr;  // what the captured launches point at
    bool no_graph = false;
};

namespace {

// Rosseland mean of the table at t_nodes[n] (FP64, one warp per node):
// 1/kappa_R = sum_i w_i / kappa_i / sum_i w_i with w_i the band integral of dB/dT.
// A bin with kappa = 0 and nonzero weight makes the mean 0.
__global__ void k_rosseland(int n_nodes, const double *t_nodes, int n_nu, const double *nu_mid, const double *kappa,
                            int n_t, const double *t_grid, double *kr_out, float *lkr)
{
    const int lane = threadIdx.x & 31;
    const int node = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (node >= n_nodes) return;
    const double t = t_nodes[node];
    const double kt_h = kKB * t / kH;
    double num = 0.0, den = 0.0;
    bool gap = false;
    for (int i = 0; i < n_nu; ++i) {
        const double lo = (i == 0) ? 0.0 : 0.5 * (nu_mid[i - 1] + nu_mid[i]);
        const double hi = (i == n_nu - 1) ? INFINITY : 0.5 * (nu_mid[i] + nu_mid[i + 1]);
        const double w = rosseland_band_warp(lo / kt_h, hi / kt_h, lane);
        const double k = kappa_at(kappa + (size_t)i * n_t, n_t, t_grid, t);
        den += w;
        if (k > 0.0) num += w / k;
        else if (w > 0.0) gap = true;
    }
    if (lane == 0) {
        const double kr = (gap || !(num > 0.0)) ? 0.0 : den / num;
        if (kr_out) kr_out[node] = kr;
        if (lkr) lkr[node] = (float)log(kr > 1e-300 ? kr : 1e-300);
    }
}

struct FldGeo {
    const float *rif;       // [nr+1] r / L
    const float *rc;        // [nr]   centre radii
    const float *drc;       // [nr]   rc[k+1] - rc[k] (last entry unused)
    const float *d3;        // [nr]   (r+^3 - r-^3) / 3
    const float *dr2;       // [nr]   (r+^2 - r-^2) / 2
    const float *sin_thif;  // [nth+1]
    const float *dthc;      // [nth]  thc[j+1] - thc[j] (last entry unused)
    const float *sin_thc;   // [nth]
    const float *dcos;      // [nth]  cos th- - cos th+
    const float *dth;       // [nth]  th+ - th-
    const float *dph;       // [nph]  phi+ - phi-
    const float *dphc;      // [nph]  phi centre l to centre l+1, wrapped
    int nr, nth, nph;
    FastDiv div_nr, div_nth;
};

// (k, j, l) of flat cell c of the [nphi][ntheta][nr] layout (c < 2^31)
__device__ __forceinline__ void cell_ijk(unsigned c, int nr, int nth, const FastDiv &dr, const FastDiv &dt, int &k,
                                         int &j, int &l)
{
    const unsigned rest = dr.div(c);
    k = (int)(c - rest * (unsigned)nr);
    l = (int)dt.div(rest);
    j = (int)(rest - (unsigned)l * (unsigned)nth);
}

__device__ __forceinline__ float lnk_interp(const float *s, float y, float y0, float inv_dy)
{
    const float u = (y - y0) * inv_dy;
    if (!(u > 0.0f)) return s[0];
    if (u >= (float)(kRossNodes - 1)) return s[kRossNodes - 1];
    const int k = min((int)u, kRossNodes - 2);
    const float t = u - (float)k;
    const float p0 = s[k], p1 = s[k + 1];
    const float m0 = k > 0 ? 0.5f * (p1 - s[k - 1]) : p1 - p0;
    const float m1 = k + 2 < kRossNodes ? 0.5f * (s[k + 2] - p0) : p1 - p0;
    const float t2 = t * t, t3 = t2 * t;
    return (2.0f * t3 - 3.0f * t2 + 1.0f) * p0 + (t3 - 2.0f * t2 + t) * m0 + (-2.0f * t3 + 3.0f * t2) * p1 +
           (t3 - t2) * m1;
}

struct FldCellArgs {
    FldGeo g;
    const float *rho, *t, *q, *e;
    const float *lkr;
    float y0, inv_dy;   // ln T nodes
    float L;            // outer radius, cm
    float c_v, four_a;  // specific heat, 4 a
    float inv_tau;      // L / (c dt)
    float q_scale;      // L / c
    float *F, *tc, *b0;
    unsigned *bad;
    long long n;
};

// per cell: the face factor F, the storage term V'/(tau f_c) and the old-state
// right-hand side; flags invalid input (rho < 0, T <= 0, E_old < 0, q < 0, NaN/Inf)
__global__ void __launch_bounds__(256) k_fld_cell(const FldCellArgs p)
{
    __shared__ float s_l[kRossNodes];
    for (int i = threadIdx.x; i < kRossNodes; i += blockDim.x) s_l[i] = p.lkr[i];
    __syncthreads();
    const FldGeo &g = p.g;
    const long long plane = (long long)g.nr * g.nth;
    bool bad = false;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < p.n;
         c += (long long)gridDim.x * blockDim.x) {
        int k, j, l;
        cell_ijk((unsigned)c, g.nr, g.nth, g.div_nr, g.div_nth, k, j, l);
        const float rho = p.rho[c], t = p.t[c], e = p.e[c], q = p.q[c];
        if (!(rho >= 0.0f && rho < INFINITY && t > 0.0f && t < INFINITY && e >= 0.0f && e < INFINITY &&
              q >= 0.0f && q < INFINITY)) {
            bad = true;
            p.F[c] = 0.0f;
            p.tc[c] = 1.0f;
            p.b0[c] = 0.0f;
            continue;
        }
        const float kr = expf(lnk_interp(s_l, logf(t), p.y0, p.inv_dy));
        const float s = (kr * rho) * p.L;
        // |grad E| / E in units of 1/L: central differences, one-sided at the r and
        // theta ends, periodic in phi (relative to this cell's E)
        const float inv_e = e > 0.0f ? 1.0f / e : 0.0f;
        float gr = 0.0f, gt = 0.0f, gp = 0.0f;
        if (g.nr > 1) {
            const int ka = k > 0 ? k - 1 : k, kb = k < g.nr - 1 ? k + 1 : k;
            float d = 0.0f;
            for (int i = ka; i < kb; ++i) d += g.drc[i];
            gr = (p.e[c + (kb - k)] - p.e[c + (ka - k)]) * inv_e / d;
        }
        if (g.nth > 1) {
            const int ja = j > 0 ? j - 1 : j, jb = j < g.nth - 1 ? j + 1 : j;
            float d = 0.0f;
            for (int i = ja; i < jb; ++i) d += g.dthc[i];
            gt = (p.e[c + (long long)(jb - j) * g.nr] - p.e[c + (long long)(ja - j) * g.nr]) * inv_e /
                 (g.rc[k] * d);
        }
        if (g.nph > 1) {
            const int la = (l + g.nph - 1) % g.nph, lb = (l + 1) % g.nph;
            const float dphi = g.nph == 2 ? 6.283185307179586f : g.dphc[la] + g.dphc[l];
            gp = (p.e[c + (long long)(lb - l) * plane] - p.e[c + (long long)(la - l) * plane]) * inv_e /
                 (g.rc[k] * g.sin_thc[j] * dphi);
        }
        const float gg = sqrtf(gr * gr + gt * gt + gp * gp);
        const float num = 2.0f * s + gg;
        p.F[c] = num > 0.0f ? num / (6.0f * s * s + 3.0f * s * gg + gg * gg) : 0.0f;
        const float t3 = t * t * t;
        const float fc = 1.0f / (p.c_v * rho / (p.four_a * t3) + 1.0f);
        const float vol = g.dcos[j] * g.dph[l] * g.d3[k];
        const float tc = vol * p.inv_tau / fc;
        p.tc[c] = tc;
        p.b0[c] = tc * e + vol * q * p.q_scale;
    }
    if (bad) atomicOr(p.bad, 1u);
}

struct FldFaceArgs {
    FldGeo g;
    const float *F, *tc, *b0;
    float e_bg;               // a T_bg^4
    float *w, *s, *idg, *b;   // w [3][n]: to the k+1, j+1 and l+1 neighbours
    unsigned short *hs, *hw, *hidg;  // BF16 copies of s, w, 1/dg (the finest V-cycle's operator)
    long long n;
};

__device__ __forceinline__ float harm(float a, float b)
{
    return (a > 0.0f && b > 0.0f) ? 2.0f * a * b / (a + b) : 0.0f;
}

// face weights to the + neighbours; s = storage + outer-boundary weight; the
// inverse of the Jacobi diagonal s + all six face weights; the right-hand side
__global__ void __launch_bounds__(256) k_fld_faces(const FldFaceArgs p)
{
    const FldGeo &g = p.g;
    const long long plane = (long long)g.nr * g.nth, n = p.n;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        int k, j, l;
        cell_ijk((unsigned)c, g.nr, g.nth, g.div_nr, g.div_nth, k, j, l);
        const float Fc = p.F[c];
        const float dom = g.dcos[j] * g.dph[l];
        float sc = p.tc[c], rhs = p.b0[c], faces = 0.0f;
        float wr = 0.0f, wt = 0.0f, wp = 0.0f;
        if (k + 1 < g.nr) {
            wr = harm(Fc, p.F[c + 1]) * dom * (g.rif[k + 1] * g.rif[k + 1]) / g.drc[k];
            faces += wr;
        } else {  // outer boundary: E_bg half a cell beyond the last centre
            const float wo = Fc * dom * (g.rif[g.nr] * g.rif[g.nr]) / (g.rif[g.nr] - g.rc[k]);
            sc += wo;
            rhs += wo * p.e_bg;
        }
        if (k > 0) faces += harm(Fc, p.F[c - 1]) * dom * (g.rif[k] * g.rif[k]) / g.drc[k - 1];
        if (j + 1 < g.nth) {
            wt = harm(Fc, p.F[c + g.nr]) * g.dph[l] * g.sin_thif[j + 1] * g.dr2[k] / (g.rc[k] * g.dthc[j]);
            faces += wt;
        }
        if (j > 0)
            faces += harm(Fc, p.F[c - g.nr]) * g.dph[l] * g.sin_thif[j] * g.dr2[k] / (g.rc[k] * g.dthc[j - 1]);
        if (g.nph > 1) {
            const int lb = (l + 1) % g.nph, la = (l + g.nph - 1) % g.nph;
            const float area = g.dth[j] * g.dr2[k] / (g.rc[k] * g.sin_thc[j]);
            wp = harm(Fc, p.F[c + (long long)(lb - l) * plane]) * area / g.dphc[l];
            faces += wp;
            faces += harm(Fc, p.F[c + (long long)(la - l) * plane]) * area / g.dphc[la];
        }
        const float idg = 1.0f / (sc + faces);
        p.w[c] = wr;
        p.w[n + c] = wt;
        p.w[2 * n + c] = wp;
        p.s[c] = sc;
        p.idg[c] = idg;
        p.b[c] = rhs;
        p.hw[c] = __bfloat16_as_ushort(__float2bfloat16_rn(wr));
        p.hw[n + c] = __bfloat16_as_ushort(__float2bfloat16_rn(wt));
        p.hw[2 * n + c] = __bfloat16_as_ushort(__float2bfloat16_rn(wp));
        p.hs[c] = __bfloat16_as_ushort(__float2bfloat16_rn(sc));
        p.hidg[c] = __bfloat16_as_ushort(__float2bfloat16_rn(idg));
    }
}

// --- the solve -----------------------------------------------------------------
// A v = s v + sum_faces w (v_c - v_nb) is applied in this flux form: the storage
// and boundary term s is stored apart from the face weights, so nothing small is
// left as the difference of large rounded numbers (a diagonal holding s + sum w
// would bury s under the rounding of the face weights wherever diffusion dominates).
// Mixed-precision iterative refinement: each pass computes the true residual
// r = b - A x, solves A d = r by preconditioned CG from d = 0 until the
// preconditioned residual norm fell by the inner drop, and adds d to x. FP32
// recurrences lose the true residual after a few hundred iterations; the restart
// from the true residual recovers it, and the passes end when max |d| / |x| < tol.
// The drops were measured per step on the 256x128x256 disk: with multigrid, loose
// inner solves and more passes are cheapest (0.2: 65.8 ms, 12 passes; 1e-2: 77.9
// ms, 6 passes); for Jacobi, 1e-2 took the fewest iterations in an FP32 emulation.
constexpr double kInnerDrop = 1e-2;    // Jacobi-preconditioned inner solves
constexpr double kInnerDropMg = 2e-1;  // multigrid-preconditioned inner solves

// device scalars of the solve
enum : int {
    kRz = 0,     // r.z of the current inner iterate
    kRz0,        // r.z at the start of the inner solve
    kAlpha,
    kBeta,
    kDone,       // 1 once the inner solve converged (the remaining launches return at once)
    kIters,      // inner iterations taken in total
    kCorr,       // max |d| / |x| of the last pass (infinite: x not finite)
    kNScal
};

struct CgArgs {
    int nr, nth, nph;
    FastDiv div_nr, div_nth;
    long long n;
    const float *w, *s, *idg, *b;
    float *x, *d, *r, *p, *q;
    double *part;     // [grid]
    double *scal;     // kNScal
    unsigned *count;  // blocks finished (last-block reductions)
};

__device__ __forceinline__ float apply_flux(const CgArgs &a, const float *v, unsigned c)
{
    int k, j, l;
    cell_ijk(c, a.nr, a.nth, a.div_nr, a.div_nth, k, j, l);
    const unsigned n = (unsigned)a.n, plane = (unsigned)a.nr * (unsigned)a.nth;
    const float vc = v[c];
    float acc = a.s[c] * vc;
    if (k + 1 < a.nr) acc = fmaf(a.w[c], vc - v[c + 1], acc);
    if (k > 0) acc = fmaf(a.w[c - 1], vc - v[c - 1], acc);
    if (j + 1 < a.nth) acc = fmaf(a.w[n + c], vc - v[c + a.nr], acc);
    if (j > 0) acc = fmaf(a.w[n + c - a.nr], vc - v[c - a.nr], acc);
    if (a.nph > 1) {
        const unsigned cb = l + 1 < a.nph ? c + plane : c - (unsigned)l * plane;
        const unsigned ca = l > 0 ? c - plane : c + (unsigned)(a.nph - 1) * plane;
        acc = fmaf(a.w[2 * n + c], vc - v[cb], acc);
        acc = fmaf(a.w[2 * n + ca], vc - v[ca], acc);
    }
    return acc;
}

// block reduction (sum, or max for MAX) into thread 0
template <bool MAX>
__device__ double block_reduce(double v)
{
    __shared__ double s_w[32];
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = MAX ? fmax(v, u) : v + u;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = MAX ? fmax(t, s_w[i]) : t + s_w[i];
    return t;
}

// Writes this block's partial; the block that finishes last reduces all partials in
// a fixed order (deterministic) and returns true in its thread 0 with the total.
template <bool MAX>
__device__ bool grid_reduce(const CgArgs &a, double v, double *out)
{
    __shared__ bool s_last;
    const double t = block_reduce<MAX>(v);
    if (threadIdx.x == 0) {
        a.part[blockIdx.x] = t;
        __threadfence();
        s_last = atomicAdd(a.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    double u = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        const double pi = __ldcg(a.part + i);
        u = MAX ? fmax(u, pi) : u + pi;
    }
    const double tot = block_reduce<MAX>(u);
    if (threadIdx.x == 0) {
        *out = tot;
        *a.count = 0u;
    }
    return threadIdx.x == 0;
}

// Per-thread sums in compensated FP32 (TwoSum; GB300's FP64 rate is a small
// fraction of its FP32 rate), handed to the FP64 block and grid reductions once.
struct KSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v)
    {
        const float t = s + v;
        const float bp = t - s;
        c += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

#define FLD_CELLS(c)                                                                          \
    for (unsigned c = blockIdx.x * blockDim.x + threadIdx.x; c < (unsigned)a.n; c += gridDim.x * blockDim.x)

// r = b - A x, d = 0, p = z = r / dg; rz0 = r.z; restarts the inner solve
__global__ void __launch_bounds__(256) k_cg_residual(const CgArgs a)
{
    KSum rz;
    FLD_CELLS(c)
    {
        const float rc = a.b[c] - apply_flux(a, a.x, c);
        const float zc = rc * a.idg[c];
        a.r[c] = rc;
        a.d[c] = 0.0f;
        a.p[c] = zc;
        rz.add(rc * zc);
    }
    double tot;
    if (grid_reduce<false>(a, rz.value(), &tot)) {
        a.scal[kRz] = tot;
        a.scal[kRz0] = tot;
        a.scal[kDone] = tot > 0.0 ? 0.0 : 1.0;
    }
}

// q = A p; alpha = rz / p.q
__global__ void __launch_bounds__(256) k_cg_apply(const CgArgs a)
{
    if (a.scal[kDone] != 0.0) return;
    KSum pq;
    FLD_CELLS(c)
    {
        const float qc = apply_flux(a, a.p, c);
        a.q[c] = qc;
        pq.add(a.p[c] * qc);
    }
    double tot;
    if (grid_reduce<false>(a, pq.value(), &tot)) {
        a.scal[kAlpha] = tot > 0.0 ? a.scal[kRz] / tot : 0.0;
        if (!(tot > 0.0)) a.scal[kDone] = 1.0;
    }
}

// d += alpha p, r -= alpha q; beta = rz_new / rz; done once rz_new <= drop^2 rz0
__global__ void __launch_bounds__(256) k_cg_update(const CgArgs a)
{
    if (a.scal[kDone] != 0.0) return;
    const float alpha = (float)a.scal[kAlpha];
    KSum rz;
    FLD_CELLS(c)
    {
        a.d[c] = fmaf(alpha, a.p[c], a.d[c]);
        const float rc = fmaf(-alpha, a.q[c], a.r[c]);
        a.r[c] = rc;
        rz.add(rc * (rc * a.idg[c]));
    }
    double tot;
    if (grid_reduce<false>(a, rz.value(), &tot)) {
        a.scal[kBeta] = a.scal[kRz] > 0.0 ? tot / a.scal[kRz] : 0.0;
        a.scal[kRz] = tot;
        a.scal[kIters] += 1.0;
        if (!(tot > kInnerDrop * kInnerDrop * a.scal[kRz0])) a.scal[kDone] = 1.0;
    }
}

// p = r / dg + beta p
__global__ void __launch_bounds__(256) k_cg_direction(const CgArgs a)
{
    if (a.scal[kDone] != 0.0) return;
    const float beta = (float)a.scal[kBeta];
    FLD_CELLS(c) a.p[c] = fmaf(beta, a.p[c], a.r[c] * a.idg[c]);
}

// x += d; kCorr = max |d| / |x|, capped at 1e30 (infinite if an x is not finite)
__global__ void __launch_bounds__(256) k_cg_accumulate(const CgArgs a)
{
    float m = 0.0f;
    FLD_CELLS(c)
    {
        const float dc = a.d[c];
        const float xc = a.x[c] + dc;
        a.x[c] = xc;
        if (!isfinite(xc)) m = INFINITY;
        else if (dc != 0.0f) m = fmaxf(m, fminf(fabsf(dc) / fmaxf(fabsf(xc), 1e-37f), 1e30f));
    }
    double tot;
    if (grid_reduce<true>(a, (double)m, &tot)) a.scal[kCorr] = tot;
}

// --- the same kernels on four consecutive cells per thread (nr % 4 == 0: the four
// cells share (j, l), every array offset is a multiple of 16 bytes) -----------------
#define FLD_QUADS(c)                                                                          \
    for (unsigned c = 4u * (blockIdx.x * blockDim.x + threadIdx.x); c < (unsigned)a.n;         \
         c += 4u * gridDim.x * blockDim.x)

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// A v on cells c .. c+3 of one ray
__device__ __forceinline__ float4 apply_flux4(const CgArgs &a, const float *v, unsigned c)
{
    int k, j, l;
    cell_ijk(c, a.nr, a.nth, a.div_nr, a.div_nth, k, j, l);
    const unsigned n = (unsigned)a.n, plane = (unsigned)a.nr * (unsigned)a.nth;
    const float4 vc = ld4(v + c), s = ld4(a.s + c), wr = ld4(a.w + c);
    float4 acc = make_float4(s.x * vc.x, s.y * vc.y, s.z * vc.z, s.w * vc.w);
    // radial faces: inside the quad, and to c-1 / c+4
    acc.x = fmaf(wr.x, vc.x - vc.y, acc.x);
    acc.y = fmaf(wr.y, vc.y - vc.z, acc.y);
    acc.z = fmaf(wr.z, vc.z - vc.w, acc.z);
    acc.y = fmaf(wr.x, vc.y - vc.x, acc.y);
    acc.z = fmaf(wr.y, vc.z - vc.y, acc.z);
    acc.w = fmaf(wr.z, vc.w - vc.z, acc.w);
    if (k + 4 < a.nr) acc.w = fmaf(wr.w, vc.w - v[c + 4], acc.w);
    if (k > 0) acc.x = fmaf(a.w[c - 1], vc.x - v[c - 1], acc.x);
    auto face4 = [&](float4 w, float4 u) {
        acc.x = fmaf(w.x, vc.x - u.x, acc.x);
        acc.y = fmaf(w.y, vc.y - u.y, acc.y);
        acc.z = fmaf(w.z, vc.z - u.z, acc.z);
        acc.w = fmaf(w.w, vc.w - u.w, acc.w);
    };
    if (j + 1 < a.nth) face4(ld4(a.w + n + c), ld4(v + c + a.nr));
    if (j > 0) face4(ld4(a.w + n + c - a.nr), ld4(v + c - a.nr));
    if (a.nph > 1) {
        const unsigned cb = l + 1 < a.nph ? c + plane : c - (unsigned)l * plane;
        const unsigned ca = l > 0 ? c - plane : c + (unsigned)(a.nph - 1) * plane;
        face4(ld4(a.w + 2 * n + c), ld4(v + cb));
        face4(ld4(a.w + 2 * n + ca), ld4(v + ca));
    }
    return acc;
}

__global__ void __launch_bounds__(256) k_cg_residual4(const CgArgs a)
{
    KSum rz;
    FLD_QUADS(c)
    {
        const float4 ax = apply_flux4(a, a.x, c), b = ld4(a.b + c), idg = ld4(a.idg + c);
        const float4 r = make_float4(b.x - ax.x, b.y - ax.y, b.z - ax.z, b.w - ax.w);
        const float4 z = make_float4(r.x * idg.x, r.y * idg.y, r.z * idg.z, r.w * idg.w);
        st4(a.r + c, r);
        st4(a.d + c, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
        st4(a.p + c, z);
        rz.add(r.x * z.x);
        rz.add(r.y * z.y);
        rz.add(r.z * z.z);
        rz.add(r.w * z.w);
    }
    double tot;
    if (grid_reduce<false>(a, rz.value(), &tot)) {
        a.scal[kRz] = tot;
        a.scal[kRz0] = tot;
        a.scal[kDone] = tot > 0.0 ? 0.0 : 1.0;
    }
}

__global__ void __launch_bounds__(256) k_cg_apply4(const CgArgs a)
{
    if (a.scal[kDone] != 0.0) return;
    KSum pq;
    FLD_QUADS(c)
    {
        const float4 q = apply_flux4(a, a.p, c), p = ld4(a.p + c);
        st4(a.q + c, q);
        pq.add(p.x * q.x);
        pq.add(p.y * q.y);
        pq.add(p.z * q.z);
        pq.add(p.w * q.w);
    }
    double tot;
    if (grid_reduce<false>(a, pq.value(), &tot)) {
        a.scal[kAlpha] = tot > 0.0 ? a.scal[kRz] / tot : 0.0;
        if (!(tot > 0.0)) a.scal[kDone] = 1.0;
    }
}

__global__ void __launch_bounds__(256) k_cg_update4(const CgArgs a)
{
    if (a.scal[kDone] != 0.0) return;
    const float alpha = (float)a.scal[kAlpha];
    KSum rz;
    FLD_QUADS(c)
    {
        const float4 p = ld4(a.p + c), q = ld4(a.q + c), idg = ld4(a.idg + c);
        float4 d = ld4(a.d + c), r = ld4(a.r + c);
        d = make_float4(fmaf(alpha, p.x, d.x), fmaf(alpha, p.y, d.y), fmaf(alpha, p.z, d.z), fmaf(alpha, p.w, d.w));
        r = make_float4(fmaf(-alpha, q.x, r.x), fmaf(-alpha, q.y, r.y), fmaf(-alpha, q.z, r.z),
                        fmaf(-alpha, q.w, r.w));
        st4(a.d + c, d);
        st4(a.r + c, r);
        rz.add(r.x * (r.x * idg.x));
        rz.add(r.y * (r.y * idg.y));
        rz.add(r.z * (r.z * idg.z));
        rz.add(r.w * (r.w * idg.w));
    }
    double tot;
    if (grid_reduce<false>(a, rz.value(), &tot)) {
        a.scal[kBeta] = a.scal[kRz] > 0.0 ? tot / a.scal[kRz] : 0.0;
        a.scal[kRz] = tot;
        a.scal[kIters] += 1.0;
        if (!(tot > kInnerDrop * kInnerDrop * a.scal[kRz0])) a.scal[kDone] = 1.0;
    }
}

__global__ void __launch_bounds__(256) k_cg_direction4(const CgArgs a)
{
    if (a.scal[kDone] != 0.0) return;
    const float beta = (float)a.scal[kBeta];
    FLD_QUADS(c)
    {
        const float4 r = ld4(a.r + c), idg = ld4(a.idg + c), p = ld4(a.p + c);
        st4(a.p + c, make_float4(fmaf(beta, p.x, r.x * idg.x), fmaf(beta, p.y, r.y * idg.y),
                                 fmaf(beta, p.z, r.z * idg.z), fmaf(beta, p.w, r.w * idg.w)));
    }
}

#undef FLD_QUADS
// --- aggregation multigrid preconditioner ---------------------------------------
// Levels coarsen by 2 in every direction longer than one cell. The coarse operator
// is the Galerkin product with piecewise-constant prolongation: the storage terms
// of an aggregate add up, and a coarse face carries the sum of the fine faces that
// cross from one aggregate into the next (faces inside an aggregate drop out), so
// every level keeps the flux form. One V-cycle per CG iteration: a damped Jacobi
// step from zero, the restricted residual, the coarser levels, the prolonged
// correction and one more Jacobi step (symmetric, so CG keeps its guarantees);
// 16 Jacobi sweeps on the coarsest level (<= 1024 cells, one CTA). The fine-level
// intermediates are formed on the fly at the stencil's points, never stored.
constexpr float kMgOmega = 0.8f;
constexpr int kMgCoarseSweeps = 16;
constexpr unsigned kMgCoarsest = 512;  // coarsen while a level has more cells

struct MgLevel {
    int nr, nth, nph;
    FastDiv dnr, dnth;
    unsigned n;
    float *s, *w, *idg;  // operator in flux form, w [3][n]
    float *b, *x;        // right-hand side and result of the level
};

// BF16 copies of the finest level's operator. The V-cycle is a preconditioner: it
// needs a symmetric positive definite approximation of A, not A itself (CG applies
// the FP32 operator), so the finest level's restriction and prolongation read these
// (BF16 keeps FP32's exponent range; s, w and 1/dg move 10 bytes per cell, not 20).
struct HalfOp {
    const unsigned short *s, *w, *idg;
};

struct MgPair {
    MgLevel f, c;    // fine and coarse level
    int sr, st, sp;  // log2 of the aggregation factors (0 or 1)
    CgArgs cg;       // scalars and reduction scratch (the finest pair's up kernel)
    HalfOp h;        // the finest level's BF16 operator (finest pair, four-cell kernels)
};

template <class V>
__device__ __forceinline__ float apply_lv(const MgLevel &L, const V &v, unsigned c, int k, int j, int l, float vc)
{
    const unsigned n = L.n, plane = (unsigned)L.nr * (unsigned)L.nth;
    float acc = L.s[c] * vc;
    if (k + 1 < L.nr) acc = fmaf(L.w[c], vc - v(c + 1), acc);
    if (k > 0) acc = fmaf(L.w[c - 1], vc - v(c - 1), acc);
    if (j + 1 < L.nth) acc = fmaf(L.w[n + c], vc - v(c + L.nr), acc);
    if (j > 0) acc = fmaf(L.w[n + c - L.nr], vc - v(c - L.nr), acc);
    if (L.nph > 1) {
        const unsigned cb = l + 1 < L.nph ? c + plane : c - (unsigned)l * plane;
        const unsigned ca = l > 0 ? c - plane : c + (unsigned)(L.nph - 1) * plane;
        acc = fmaf(L.w[2 * n + c], vc - v(cb), acc);
        acc = fmaf(L.w[2 * n + ca], vc - v(ca), acc);
    }
    return acc;
}

#define MG_LOOP(i, N) for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < (N); i += gridDim.x * blockDim.x)

// coarse storage terms and face weights of an aggregate
__global__ void __launch_bounds__(256) k_mg_coarsen(const MgPair P)
{
    const MgLevel &F = P.f, &C = P.c;
    MG_LOOP(cc, C.n)
    {
        int K, J, L;
        cell_ijk(cc, C.nr, C.nth, C.dnr, C.dnth, K, J, L);
        float sum = 0.0f, wr = 0.0f, wt = 0.0f, wp = 0.0f;
#pragma unroll
        for (int dl = 0; dl < 2; ++dl)
#pragma unroll
            for (int dj = 0; dj < 2; ++dj)
#pragma unroll
                for (int dk = 0; dk < 2; ++dk) {
                    const int l = (L << P.sp) + dl, j = (J << P.st) + dj, k = (K << P.sr) + dk;
                    if (!((dl <= P.sp && l < F.nph) && (dj <= P.st && j < F.nth) && (dk <= P.sr && k < F.nr)))
                        continue;
                    const unsigned c = ((unsigned)l * F.nth + j) * F.nr + k;
                    sum += F.s[c];
                    if (k + 1 < F.nr && ((k + 1) >> P.sr) != (k >> P.sr)) wr += F.w[c];
                    if (j + 1 < F.nth && ((j + 1) >> P.st) != (j >> P.st)) wt += F.w[F.n + c];
                    if (F.nph > 1 && (((l + 1) % F.nph) >> P.sp) != (l >> P.sp)) wp += F.w[2 * F.n + c];
                }
        C.s[cc] = sum;
        C.w[cc] = wr;
        C.w[C.n + cc] = wt;
        C.w[2 * C.n + cc] = wp;
    }
}

// inverse diagonal of a level
__global__ void __launch_bounds__(256) k_mg_diag(const MgLevel L)
{
    const unsigned n = L.n, plane = (unsigned)L.nr * (unsigned)L.nth;
    MG_LOOP(c, n)
    {
        int k, j, l;
        cell_ijk(c, L.nr, L.nth, L.dnr, L.dnth, k, j, l);
        float d = L.s[c];
        if (k + 1 < L.nr) d += L.w[c];
        if (k > 0) d += L.w[c - 1];
        if (j + 1 < L.nth) d += L.w[n + c];
        if (j > 0) d += L.w[n + c - L.nr];
        if (L.nph > 1) {
            const unsigned ca = l > 0 ? c - plane : c + (unsigned)(L.nph - 1) * plane;
            d += L.w[2 * n + c] + L.w[2 * n + ca];
        }
        L.idg[c] = d > 0.0f ? 1.0f / d : 0.0f;
    }
}

// coarse right-hand side: the aggregate's sum of the fine residuals after the
// first Jacobi step x0 = omega b / dg (the 2 x 2 x 2 loop unrolled, so that the
// loads of all eight fine cells are in flight together)
__global__ void __launch_bounds__(256) k_mg_down(const MgPair P)
{
    if (P.cg.scal[kDone] != 0.0) return;
    const MgLevel &F = P.f, &C = P.c;
    const float *idg = F.idg, *b = F.b;
    auto x0 = [=](unsigned i) { return kMgOmega * idg[i] * b[i]; };
    MG_LOOP(cc, C.n)
    {
        int K, J, L;
        cell_ijk(cc, C.nr, C.nth, C.dnr, C.dnth, K, J, L);
        float sum = 0.0f;
#pragma unroll
        for (int dl = 0; dl < 2; ++dl)
#pragma unroll
            for (int dj = 0; dj < 2; ++dj)
#pragma unroll
                for (int dk = 0; dk < 2; ++dk) {
                    const int l = (L << P.sp) + dl, j = (J << P.st) + dj, k = (K << P.sr) + dk;
                    const bool in = (dl <= P.sp && l < F.nph) && (dj <= P.st && j < F.nth) && (dk <= P.sr && k < F.nr);
                    if (in) {
                        const unsigned c = ((unsigned)l * F.nth + j) * F.nr + k;
                        sum += b[c] - apply_lv(F, x0, c, k, j, l, x0(c));
                    }
                }
        C.b[cc] = sum;
    }
}

// the coarsest level (n <= 1024): kMgCoarseSweeps damped Jacobi sweeps from zero,
// the level's operator staged in shared memory once
__global__ void __launch_bounds__(256) k_mg_coarsest(const MgLevel L, const double *scal)
{
    if (scal[kDone] != 0.0) return;
    __shared__ float xs[1024], ss[1024], wr[1024], wt[1024], wp[1024], id[1024], bs[1024];
    const unsigned n = L.n;
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
        ss[i] = L.s[i];
        wr[i] = L.w[i];
        wt[i] = L.w[n + i];
        wp[i] = L.w[2 * n + i];
        id[i] = L.idg[i];
        bs[i] = L.b[i];
        xs[i] = kMgOmega * L.idg[i] * L.b[i];
    }
    __syncthreads();
    const unsigned plane = (unsigned)L.nr * (unsigned)L.nth;
    for (int sweep = 1; sweep < kMgCoarseSweeps; ++sweep) {
        float nv[4];
        int m = 0;
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x, ++m) {
            int k, j, l;
            cell_ijk(i, L.nr, L.nth, L.dnr, L.dnth, k, j, l);
            const float xi = xs[i];
            float acc = ss[i] * xi;
            if (k + 1 < L.nr) acc = fmaf(wr[i], xi - xs[i + 1], acc);
            if (k > 0) acc = fmaf(wr[i - 1], xi - xs[i - 1], acc);
            if (j + 1 < L.nth) acc = fmaf(wt[i], xi - xs[i + L.nr], acc);
            if (j > 0) acc = fmaf(wt[i - L.nr], xi - xs[i - L.nr], acc);
            if (L.nph > 1) {
                const unsigned cb = l + 1 < L.nph ? i + plane : i - (unsigned)l * plane;
                const unsigned ca = l > 0 ? i - plane : i + (unsigned)(L.nph - 1) * plane;
                acc = fmaf(wp[i], xi - xs[cb], acc);
                acc = fmaf(wp[ca], xi - xs[ca], acc);
            }
            nv[m] = fmaf(kMgOmega * id[i], bs[i] - acc, xi);
        }
        __syncthreads();
        m = 0;
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x, ++m) xs[i] = nv[m];
        __syncthreads();
    }
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) L.x[i] = xs[i];
}

// prolonged correction and the second Jacobi step: x = x1 + omega (b - A x1) / dg,
// x1 = omega b / dg + x_coarse[aggregate]. On the finest pair (top) x is z = M^-1 r
// and its r.z closes the CG step: init sets rz0 and beta = 0, otherwise beta, rz,
// the iteration count and the convergence flag.
__global__ void __launch_bounds__(256) k_mg_up(const MgPair P, int top, int init)
{
    if (P.cg.scal[kDone] != 0.0) return;
    const MgLevel &F = P.f, &C = P.c;
    const unsigned n = F.n, plane = (unsigned)F.nr * (unsigned)F.nth;
    const float *idg = F.idg, *b = F.b, *xc = C.x;
    auto x1 = [&](unsigned i, int k, int j, int l) {
        return fmaf(kMgOmega * idg[i], b[i], xc[((unsigned)(l >> P.sp) * C.nth + (j >> P.st)) * C.nr + (k >> P.sr)]);
    };
    KSum rz;
    MG_LOOP(c, n)
    {
        int k, j, l;
        cell_ijk(c, F.nr, F.nth, F.dnr, F.dnth, k, j, l);
        const float vc = x1(c, k, j, l);
        float acc = F.s[c] * vc;
        if (k + 1 < F.nr) acc = fmaf(F.w[c], vc - x1(c + 1, k + 1, j, l), acc);
        if (k > 0) acc = fmaf(F.w[c - 1], vc - x1(c - 1, k - 1, j, l), acc);
        if (j + 1 < F.nth) acc = fmaf(F.w[n + c], vc - x1(c + F.nr, k, j + 1, l), acc);
        if (j > 0) acc = fmaf(F.w[n + c - F.nr], vc - x1(c - F.nr, k, j - 1, l), acc);
        if (F.nph > 1) {
            const int lb = l + 1 < F.nph ? l + 1 : 0, la = l > 0 ? l - 1 : F.nph - 1;
            const unsigned cb = c + (unsigned)(lb - l) * plane, ca = c + (unsigned)(la - l) * plane;
            acc = fmaf(F.w[2 * n + c], vc - x1(cb, k, j, lb), acc);
            acc = fmaf(F.w[2 * n + ca], vc - x1(ca, k, j, la), acc);
        }
        const float xv = fmaf(kMgOmega * idg[c], b[c] - acc, vc);
        F.x[c] = xv;
        if (top) rz.add(b[c] * xv);
    }
    if (!top) return;
    double tot;
    if (grid_reduce<false>(P.cg, rz.value(), &tot)) {
        double *sc = P.cg.scal;
        if (init) {
            sc[kRz] = tot;
            sc[kRz0] = tot;
            sc[kBeta] = 0.0;
            sc[kDone] = tot > 0.0 ? 0.0 : 1.0;
        } else {
            sc[kBeta] = sc[kRz] > 0.0 ? tot / sc[kRz] : 0.0;
            sc[kRz] = tot;
            sc[kIters] += 1.0;
            if (!(tot > kInnerDropMg * kInnerDropMg * sc[kRz0])) sc[kDone] = 1.0;
        }
    }
}

// Finest level with nr % 4 == 0: four cells of one ray per thread; the BF16 operator
// in 64-bit loads. A_h v on the quad c .. c+3 at (k .. k+3, j, l), the value of the quad
// at the same k of row (j', l') from vrow(c0, k, j', l') and of one cell from
// vone(i, k', j, l).
__device__ __forceinline__ float4 ldh4(const unsigned short *p)
{
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u));
}
__device__ __forceinline__ float ldh1(const unsigned short *p) { return __uint_as_float((unsigned)*p << 16); }

template <class VR, class V1>
__device__ __forceinline__ float4 apply_quad(const MgLevel &F, const HalfOp &h, const VR &vrow, const V1 &vone,
                                             unsigned c, int k, int j, int l, float4 vc)
{
    const unsigned n = F.n, plane = (unsigned)F.nr * (unsigned)F.nth;
    const float4 s = ldh4(h.s + c), wr = ldh4(h.w + c);
    float4 acc = make_float4(s.x * vc.x, s.y * vc.y, s.z * vc.z, s.w * vc.w);
    acc.x = fmaf(wr.x, vc.x - vc.y, acc.x);
    acc.y = fmaf(wr.y, vc.y - vc.z, acc.y);
    acc.z = fmaf(wr.z, vc.z - vc.w, acc.z);
    acc.y = fmaf(wr.x, vc.y - vc.x, acc.y);
    acc.z = fmaf(wr.y, vc.z - vc.y, acc.z);
    acc.w = fmaf(wr.z, vc.w - vc.z, acc.w);
    if (k + 4 < F.nr) acc.w = fmaf(wr.w, vc.w - vone(c + 4, k + 4, j, l), acc.w);
    if (k > 0) acc.x = fmaf(ldh1(h.w + c - 1), vc.x - vone(c - 1, k - 1, j, l), acc.x);
    auto face4 = [&](float4 w, float4 u) {
        acc.x = fmaf(w.x, vc.x - u.x, acc.x);
        acc.y = fmaf(w.y, vc.y - u.y, acc.y);
        acc.z = fmaf(w.z, vc.z - u.z, acc.z);
        acc.w = fmaf(w.w, vc.w - u.w, acc.w);
    };
    if (j + 1 < F.nth) face4(ldh4(h.w + n + c), vrow(c + F.nr, k, j + 1, l));
    if (j > 0) face4(ldh4(h.w + n + c - F.nr), vrow(c - F.nr, k, j - 1, l));
    if (F.nph > 1) {
        const int lb = l + 1 < F.nph ? l + 1 : 0, la = l > 0 ? l - 1 : F.nph - 1;
        const unsigned cb = c + (unsigned)(lb - l) * plane, ca = c + (unsigned)(la - l) * plane;
        face4(ldh4(h.w + 2 * n + c), vrow(cb, k, j, lb));
        face4(ldh4(h.w + 2 * n + ca), vrow(ca, k, j, la));
    }
    return acc;
}

// k_mg_down on the finest level: one thread per pair of coarse cells (K0, K0 + 1)
// of one coarse row, i.e. the four-cell quads of the fine rows in the aggregate.
// (Five CTAs per SM: 48 registers and a few bytes of spill measured 1.2 % faster per
// FLD step than four CTAs at 54 registers; the same for k_mg_up4.)
__global__ void __launch_bounds__(256, 5) k_mg_down4(const MgPair P)
{
    if (P.cg.scal[kDone] != 0.0) return;
    const MgLevel &F = P.f, &C = P.c;
    const unsigned short *idg = P.h.idg;
    const float *b = F.b;
    auto vrow = [=](unsigned c0, int, int, int) {
        const float4 d = ldh4(idg + c0), bb = ld4(b + c0);
        return make_float4(kMgOmega * d.x * bb.x, kMgOmega * d.y * bb.y, kMgOmega * d.z * bb.z, kMgOmega * d.w * bb.w);
    };
    auto vone = [=](unsigned i, int, int, int) { return kMgOmega * ldh1(idg + i) * b[i]; };
    const unsigned nq = (unsigned)(F.nr / 4) * (unsigned)C.nth * (unsigned)C.nph;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < nq; t += gridDim.x * blockDim.x) {
        const unsigned qr = (unsigned)(F.nr / 4);
        const unsigned rest = t / qr;
        const int m = (int)(t - rest * qr);
        const int J = (int)(rest % (unsigned)C.nth), L = (int)(rest / (unsigned)C.nth);
        const int k = 4 * m;
        float lo = 0.0f, hi = 0.0f;
        for (int l = L << P.sp; l < min((L + 1) << P.sp, F.nph); ++l)
            for (int j = J << P.st; j < min((J + 1) << P.st, F.nth); ++j) {
                const unsigned c = ((unsigned)l * F.nth + j) * F.nr + k;
                const float4 vc = vrow(c, k, j, l), bb = ld4(b + c);
                const float4 ax = apply_quad(F, P.h, vrow, vone, c, k, j, l, vc);
                lo += (bb.x - ax.x) + (bb.y - ax.y);
                hi += (bb.z - ax.z) + (bb.w - ax.w);
            }
        const unsigned cc = ((unsigned)L * C.nth + J) * C.nr + 2 * m;
        C.b[cc] = lo;
        C.b[cc + 1] = hi;
    }
}

// k_mg_up on the finest level (top), four cells per thread
__global__ void __launch_bounds__(256, 5) k_mg_up4(const MgPair P, int init)
{
    if (P.cg.scal[kDone] != 0.0) return;
    const MgLevel &F = P.f, &C = P.c;
    const unsigned short *idg = P.h.idg;
    const float *b = F.b, *xc = C.x;
    const int st = P.st, sp = P.sp, cnr = C.nr, cnth = C.nth;
    auto crow = [=](int j, int l) { return ((unsigned)(l >> sp) * cnth + (j >> st)) * cnr; };
    auto vrow = [=](unsigned c0, int k, int j, int l) {
        const unsigned K0 = crow(j, l) + (k >> 1);
        const float2 x2 = make_float2(xc[K0], xc[K0 + 1]);
        const float4 d = ldh4(idg + c0), bb = ld4(b + c0);
        return make_float4(fmaf(kMgOmega * d.x, bb.x, x2.x), fmaf(kMgOmega * d.y, bb.y, x2.x),
                           fmaf(kMgOmega * d.z, bb.z, x2.y), fmaf(kMgOmega * d.w, bb.w, x2.y));
    };
    auto vone = [=](unsigned i, int k, int j, int l) {
        return fmaf(kMgOmega * ldh1(idg + i), b[i], xc[crow(j, l) + (k >> 1)]);
    };
    KSum rz;
    for (unsigned c = 4u * (blockIdx.x * blockDim.x + threadIdx.x); c < F.n; c += 4u * gridDim.x * blockDim.x) {
        int k, j, l;
        cell_ijk(c, F.nr, F.nth, F.dnr, F.dnth, k, j, l);
        const float4 vc = vrow(c, k, j, l);
        const float4 ax = apply_quad(F, P.h, vrow, vone, c, k, j, l, vc);
        const float4 d = ldh4(idg + c), bb = ld4(b + c);
        const float4 z = make_float4(fmaf(kMgOmega * d.x, bb.x - ax.x, vc.x), fmaf(kMgOmega * d.y, bb.y - ax.y, vc.y),
                                     fmaf(kMgOmega * d.z, bb.z - ax.z, vc.z), fmaf(kMgOmega * d.w, bb.w - ax.w, vc.w));
        st4(F.x + c, z);
        rz.add(bb.x * z.x);
        rz.add(bb.y * z.y);
        rz.add(bb.z * z.z);
        rz.add(bb.w * z.w);
    }
    double tot;
    if (grid_reduce<false>(P.cg, rz.value(), &tot)) {
        double *sc = P.cg.scal;
        if (init) {
            sc[kRz] = tot;
            sc[kRz0] = tot;
            sc[kBeta] = 0.0;
            sc[kDone] = tot > 0.0 ? 0.0 : 1.0;
        } else {
            sc[kBeta] = sc[kRz] > 0.0 ? tot / sc[kRz] : 0.0;
            sc[kRz] = tot;
            sc[kIters] += 1.0;
            if (!(tot > kInnerDropMg * kInnerDropMg * sc[kRz0])) sc[kDone] = 1.0;
        }
    }
}

#undef MG_LOOP

// CG steps of the multigrid path (the preconditioned residual z comes from k_mg_up)
// r = b - A x, d = 0, p = 0
__global__ void __launch_bounds__(256) k_cg_residual_mg(const CgArgs a)
{
    FLD_CELLS(c)
    {
        a.r[c] = a.b[c] - apply_flux(a, a.x, c);
        a.d[c] = 0.0f;
        a.p[c] = 0.0f;
    }
}

// d += alpha p, r -= alpha q (four cells per thread; n % 4 == 0)
__global__ void __launch_bounds__(256) k_cg_update_mg4(const CgArgs a)
{
    if (a.scal[kDone] != 0.0) return;
    const float alpha = (float)a.scal[kAlpha];
    for (unsigned c = 4u * (blockIdx.x * blockDim.x + threadIdx.x); c < (unsigned)a.n; c += 4u * gridDim.x * blockDim.x) {
        const float4 p = ld4(a.p + c), q = ld4(a.q + c);
        float4 d = ld4(a.d + c), r = ld4(a.r + c);
        d = make_float4(fmaf(alpha, p.x, d.x), fmaf(alpha, p.y, d.y), fmaf(alpha, p.z, d.z), fmaf(alpha, p.w, d.w));
        r = make_float4(fmaf(-alpha, q.x, r.x), fmaf(-alpha, q.y, r.y), fmaf(-alpha, q.z, r.z),
                        fmaf(-alpha, q.w, r.w));
        st4(a.d + c, d);
        st4(a.r + c, r);
    }
}

__global__ void __launch_bounds__(256) k_cg_update_mg(const CgArgs a)
{
    if (a.scal[kDone] != 0.0) return;
    const float alpha = (float)a.scal[kAlpha];
    FLD_CELLS(c)
    {
        a.d[c] = fmaf(alpha, a.p[c], a.d[c]);
        a.r[c] = fmaf(-alpha, a.q[c], a.r[c]);
    }
}

// p = z + beta p (z: the finest level's multigrid result)
__global__ void __launch_bounds__(256) k_cg_direction_mg4(const CgArgs a, const float *z)
{
    if (a.scal[kDone] != 0.0) return;
    const float beta = (float)a.scal[kBeta];
    for (unsigned c = 4u * (blockIdx.x * blockDim.x + threadIdx.x); c < (unsigned)a.n; c += 4u * gridDim.x * blockDim.x) {
        const float4 zz = ld4(z + c), p = ld4(a.p + c);
        st4(a.p + c, make_float4(fmaf(beta, p.x, zz.x), fmaf(beta, p.y, zz.y), fmaf(beta, p.z, zz.z),
                                 fmaf(beta, p.w, zz.w)));
    }
}

__global__ void __launch_bounds__(256) k_cg_direction_mg(const CgArgs a, const float *z)
{
    if (a.scal[kDone] != 0.0) return;
    const float beta = (float)a.scal[kBeta];
    FLD_CELLS(c) a.p[c] = fmaf(beta, a.p[c], z[c]);
}

#undef FLD_CELLS

int rosseland_nodes(const CtxInfo &in, const std::vector<double> &t_nodes, double *kr_host, float *lkr_dev,
                    cudaStream_t st, std::string &err)
{
    const int n = (int)t_nodes.size();
    const int n_t = in.n_t > 0 ? in.n_t : 1;
    const double *kap_h = in.n_t > 0 ? in.kappa_t_h : in.kappa_h;
    double *tn = nullptr, *nu = nullptr, *ka = nullptr, *tg = nullptr, *kr = nullptr;
    bool ok = cudaMalloc(&tn, sizeof(double) * n) == cudaSuccess &&
              cudaMalloc(&nu, sizeof(double) * in.n_nu) == cudaSuccess &&
              cudaMalloc(&ka, sizeof(double) * in.n_nu * n_t) == cudaSuccess &&
              cudaMalloc(&tg, sizeof(double) * n_t) == cudaSuccess && cudaMalloc(&kr, sizeof(double) * n) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(tn, t_nodes.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(nu, in.nu_h, sizeof(double) * in.n_nu, cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(ka, kap_h, sizeof(double) * in.n_nu * n_t, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok && in.n_t > 0)
        ok = cudaMemcpyAsync(tg, in.t_grid_h, sizeof(double) * n_t, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok) {
        k_rosseland<<<(n + 7) / 8, 256, 0, st>>>(n, tn, in.n_nu, nu, ka, n_t, tg, kr, lkr_dev);
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (ok && kr_host) ok = cudaMemcpyAsync(kr_host, kr, sizeof(double) * n, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) err = std::string("Rosseland-mean kernel: ") + cudaGetErrorString(cudaGetLastError());
    cudaFree(tn);
    cudaFree(nu);
    cudaFree(ka);
    cudaFree(tg);
    cudaFree(kr);
    return ok ? RT_OK : RT_ERR_CUDA;
}

// the axis tables of FldGeo, in units of the outer radius, computed in FP64
std::vector<float> geometry_tables(const CtxInfo &in)
{
    const int nr = in.nr, nth = in.ntheta, nph = in.nphi;
    const double *ri = in.r_if_h, *ti = in.theta_if_h, *pi = in.phi_if_h;
    const double L = ri[nr];
    std::vector<float> h;
    auto rc = [&](int k) { return 0.5 * (ri[k] + ri[k + 1]) / L; };
    auto thc = [&](int j) { return 0.5 * (ti[j] + ti[j + 1]); };
    auto phc = [&](int l) { return 0.5 * (pi[l] + pi[l + 1]); };
    for (int k = 0; k <= nr; ++k) h.push_back((float)(ri[k] / L));
    for (int k = 0; k < nr; ++k) h.push_back((float)rc(k));
    for (int k = 0; k < nr; ++k) h.push_back(k + 1 < nr ? (float)(rc(k + 1) - rc(k)) : 0.0f);
    for (int k = 0; k < nr; ++k) {
        const double a = ri[k] / L, b = ri[k + 1] / L;
        h.push_back((float)((b - a) * (a * a + a * b + b * b) / 3.0));
    }
    for (int k = 0; k < nr; ++k) {
        const double a = ri[k] / L, b = ri[k + 1] / L;
        h.push_back((float)(0.5 * (b - a) * (a + b)));
    }
    for (int j = 0; j <= nth; ++j) h.push_back((float)sin(ti[j]));
    for (int j = 0; j < nth; ++j) h.push_back(j + 1 < nth ? (float)(thc(j + 1) - thc(j)) : 0.0f);
    for (int j = 0; j < nth; ++j) h.push_back((float)sin(thc(j)));
    for (int j = 0; j < nth; ++j) h.push_back((float)(cos(ti[j]) - cos(ti[j + 1])));
    for (int j = 0; j < nth; ++j) h.push_back((float)(ti[j + 1] - ti[j]));
    for (int l = 0; l < nph; ++l) h.push_back((float)(pi[l + 1] - pi[l]));
    for (int l = 0; l < nph; ++l) {
        double d = fmod(phc((l + 1) % nph) - phc(l), 2.0 * kPi);
        if (d < 0.0) d += 2.0 * kPi;
        h.push_back((float)d);
    }
    return h;
}

FldGeo geo_view(const float *gp, int nr, int nth, int nph)
{
    FldGeo g;
    g.rif = gp; gp += nr + 1;
    g.rc = gp; gp += nr;
    g.drc = gp; gp += nr;
    g.d3 = gp; gp += nr;
    g.dr2 = gp; gp += nr;
    g.sin_thif = gp; gp += nth + 1;
    g.dthc = gp; gp += nth;
    g.sin_thc = gp; gp += nth;
    g.dcos = gp; gp += nth;
    g.dth = gp; gp += nth;
    g.dph = gp; gp += nph;
    g.dphc = gp;
    g.nr = nr;
    g.nth = nth;
    g.nph = nph;
    g.div_nr = FastDiv::make((unsigned)nr);
    g.div_nth = FastDiv::make((unsigned)nth);
    return g;
}

double radiation_constant()
{
    const double sigma = 2.0 * pow(kPi, 5) * pow(kKB, 4) / (15.0 * kH * kH * kH * kC * kC);
    return 4.0 * sigma / kC;
}

}  // namespace

void fld_free(FldState *s)
{
    if (!s) return;
    cudaFree(s->buf);
    cudaFree(s->mg_buf);
    cudaFree(s->part);
    cudaFree(s->scal);
    cudaFree(s->bad);
    cudaFree(s->count);
    cudaFree(s->geo);
    cudaFree(s->lkr);
    if (s->burst) cudaGraphExecDestroy(s->burst);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->gs) cudaStreamDestroy(s->gs);
    delete s;
}

}  // namespace rt

using namespace rt;

extern "C" {

int rt_rosseland_mean_opacity(rt_ctx *ctx, double t, double *kappa_r)
{
    if (!ctx || !kappa_r) return RT_ERR_INVALID_ARG;
    CtxInfo in;
    ctx_info(ctx, &in);
    if (!in.configured) return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "call rt_set_star and rt_set_opacity_table first");
    if (!(t > 0.0) || !isfinite(t)) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "t must be finite and > 0");
    if (cudaSetDevice(in.dev) != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, "cudaSetDevice");
    std::string err;
    const int rc = rosseland_nodes(in, std::vector<double>{t}, kappa_r, nullptr, in.stream, err);
    return rc == RT_OK ? RT_OK : ctx_fail(ctx, rc, err);
}

int rt_fld_step(rt_ctx *ctx, const float *rho, const float *t_gas, const float *q_abs, const float *e_old,
                float *e_new, double dt, double c_v, double t_bg, double tol, int max_iter, rt_fld_stats *stats)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    CtxInfo in;
    ctx_info(ctx, &in);
    if (!in.configured) return ctx_fail(ctx, RT_ERR_NOT_CONFIGURED, "call rt_set_star and rt_set_opacity_table first");
    if (!rho || !t_gas || !q_abs || !e_old || !e_new) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "NULL field pointer");
    if (!(dt > 0.0) || !(c_v >= 0.0) || !isfinite(c_v) || !(t_bg >= 0.0) || !isfinite(t_bg) || !(tol > 0.0) ||
        max_iter < 1)
        return ctx_fail(ctx, RT_ERR_INVALID_ARG, "need dt > 0, finite c_v >= 0 and t_bg >= 0, tol > 0, max_iter >= 1");
    if (e_new == e_old) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "e_new must not alias e_old");
    if (in.ncells >= (1LL << 31) - 1) return ctx_fail(ctx, RT_ERR_INVALID_ARG, "FLD step needs fewer than 2^31 cells");
    if (cudaSetDevice(in.dev) != cudaSuccess) return ctx_fail(ctx, RT_ERR_CUDA, "cudaSetDevice");
    FldState *&fs = ctx_fld(ctx);
    if (!fs) fs = new FldState();
    if (!fs->gs) {
        if (cudaStreamCreateWithFlags(&fs->gs, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&fs->ev_in, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(ctx, RT_ERR_CUDA, "FLD stream");
        }
    }
    // everything below runs on the private stream, after the context stream's work so far
    if (cudaEventRecord(fs->ev_in, in.stream) != cudaSuccess || cudaStreamWaitEvent(fs->gs, fs->ev_in, 0) != cudaSuccess)
        return ctx_fail(ctx, RT_ERR_CUDA, "FLD stream order");
    cudaStream_t st = fs->gs;
    const long long n = in.ncells;
    const int nr = in.nr, nth = in.ntheta, nph = in.nphi;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, in.dev);
    if (nsm < 1) nsm = 1;
    const int grid = (int)std::max(1LL, std::min<long long>((n + 255) / 256, 8LL * nsm));
    if (fs->cap < n) {
        cudaFree(fs->buf);
        fs->buf = nullptr;
        fs->cap = 0;
        if (cudaMalloc(&fs->buf, sizeof(float) * 18 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(ctx, RT_ERR_NO_MEMORY, "FLD workspace");
        }
        fs->cap = n;
    }
    const int grid_max = 8 * nsm;  // 256-thread CTAs resident per SM are at most 8
    if (fs->part_cap < grid_max) {
        cudaFree(fs->part);
        fs->part = nullptr;
        fs->part_cap = 0;
        if (cudaMalloc(&fs->part, sizeof(double) * grid_max) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(ctx, RT_ERR_NO_MEMORY, "FLD partials");
        }
        fs->part_cap = grid_max;
    }
    if (!fs->scal) {
        if (cudaMalloc(&fs->scal, sizeof(double) * kNScal) != cudaSuccess ||
            cudaMalloc(&fs->bad, sizeof(unsigned)) != cudaSuccess ||
            cudaMalloc(&fs->count, sizeof(unsigned)) != cudaSuccess ||
            cudaMemset(fs->count, 0, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(fs->scal);
            cudaFree(fs->bad);
            cudaFree(fs->count);
            fs->scal = nullptr;
            fs->bad = fs->count = nullptr;
            return ctx_fail(ctx, RT_ERR_NO_MEMORY, "FLD scalars");
        }
    }
    if (!fs->geo) {
        const std::vector<float> h = geometry_tables(in);
        if (cudaMalloc(&fs->geo, sizeof(float) * h.size()) != cudaSuccess ||
            cudaMemcpy(fs->geo, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(fs->geo);
            fs->geo = nullptr;
            return ctx_fail(ctx, RT_ERR_CUDA, "FLD geometry tables");
        }
    }
    if (fs->mg_dims.empty()) {  // multigrid levels: halve every direction longer than one cell
        int a = nr, b2 = nth, c3 = nph;
        size_t coarse = 0;
        fs->mg_dims = {a, b2, c3};
        while ((unsigned long long)a * b2 * c3 > kMgCoarsest && (a > 1 || b2 > 1 || c3 > 1)) {
            a = a > 1 ? (a + 1) / 2 : 1;
            b2 = b2 > 1 ? (b2 + 1) / 2 : 1;
            c3 = c3 > 1 ? (c3 + 1) / 2 : 1;
            fs->mg_dims.insert(fs->mg_dims.end(), {a, b2, c3});
            coarse += (size_t)a * b2 * c3;
        }
        if (coarse > 0 && cudaMalloc(&fs->mg_buf, sizeof(float) * 7 * coarse) != cudaSuccess) {
            cudaGetLastError();
            fs->mg_dims.clear();
            return ctx_fail(ctx, RT_ERR_NO_MEMORY, "FLD multigrid levels");
        }
    }
    if (!fs->lkr_valid || fs->lkr_fp != in.table_fingerprint) {
        if (!fs->lkr && cudaMalloc(&fs->lkr, sizeof(float) * kRossNodes) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(ctx, RT_ERR_NO_MEMORY, "Rosseland table");
        }
        std::vector<double> tn(kRossNodes);
        for (int i = 0; i < kRossNodes; ++i) tn[i] = exp(kRossLnLo + (kRossLnHi - kRossLnLo) * i / (kRossNodes - 1));
        std::string err;
        const int rc = rosseland_nodes(in, tn, nullptr, fs->lkr, st, err);
        if (rc != RT_OK) return ctx_fail(ctx, rc, err);
        fs->lkr_fp = in.table_fingerprint;
        fs->lkr_valid = true;
    }
    const FldGeo g = geo_view(fs->geo, nr, nth, nph);
    const double L = in.r_if_h[nr];
    const double a_rad = radiation_constant();
    float *F = fs->buf, *tc = F + n, *b0 = tc + n, *w = b0 + n, *sv = w + 3 * n, *idg = sv + n, *b = idg + n;
    float *d = b + n, *r = d + n, *p = r + n, *q = p + n, *z = q + n;
    unsigned short *hs = reinterpret_cast<unsigned short *>(z + n), *hw = hs + n, *hidg = hw + 3 * n;

    FldCellArgs ca;
    ca.g = g;
    ca.rho = rho;
    ca.t = t_gas;
    ca.q = q_abs;
    ca.e = e_old;
    ca.lkr = fs->lkr;
    ca.y0 = (float)kRossLnLo;
    ca.inv_dy = (float)((kRossNodes - 1) / (kRossLnHi - kRossLnLo));
    ca.L = (float)L;
    ca.c_v = (float)c_v;
    ca.four_a = (float)(4.0 * a_rad);
    ca.inv_tau = (float)(L / (kC * dt));
    ca.q_scale = (float)(L / kC);
    ca.F = F;
    ca.tc = tc;
    ca.b0 = b0;
    ca.bad = fs->bad;
    ca.n = n;
    FldFaceArgs fa;
    fa.g = g;
    fa.F = F;
    fa.tc = tc;
    fa.b0 = b0;
    fa.e_bg = (float)(a_rad * pow(t_bg, 4));
    fa.w = w;
    fa.s = sv;
    fa.idg = idg;
    fa.b = b;
    fa.hs = hs;
    fa.hw = hw;
    fa.hidg = hidg;
    fa.n = n;
    CgArgs cg;
    cg.nr = nr;
    cg.nth = nth;
    cg.nph = nph;
    cg.div_nr = g.div_nr;
    cg.div_nth = g.div_nth;
    cg.n = n;
    cg.w = w;
    cg.s = sv;
    cg.idg = idg;
    cg.b = b;
    cg.x = e_new;
    cg.d = d;
    cg.r = r;
    cg.p = p;
    cg.q = q;
    cg.part = fs->part;
    cg.scal = fs->scal;
    cg.count = fs->count;

    // multigrid levels and pairs (level 0: the fine operator, b = r, x = z)
    const int n_lv = (int)fs->mg_dims.size() / 3;
    const bool use_mg = n_lv > 1;
    std::vector<MgLevel> lv(n_lv);
    {
        float *cursor = fs->mg_buf;
        for (int i = 0; i < n_lv; ++i) {
            MgLevel &L = lv[i];
            L.nr = fs->mg_dims[3 * i];
            L.nth = fs->mg_dims[3 * i + 1];
            L.nph = fs->mg_dims[3 * i + 2];
            L.dnr = FastDiv::make((unsigned)L.nr);
            L.dnth = FastDiv::make((unsigned)L.nth);
            L.n = (unsigned)L.nr * (unsigned)L.nth * (unsigned)L.nph;
            if (i == 0) {
                L.s = sv;
                L.w = w;
                L.idg = idg;
                L.b = r;
                L.x = z;
            } else {
                L.s = cursor;
                L.w = L.s + L.n;
                L.idg = L.w + 3 * (size_t)L.n;
                L.b = L.idg + L.n;
                L.x = L.b + L.n;
                cursor = L.x + L.n;
            }
        }
    }
    std::vector<MgPair> pairs(n_lv > 0 ? n_lv - 1 : 0);
    for (int i = 0; i + 1 < n_lv; ++i) {
        pairs[i].f = lv[i];
        pairs[i].c = lv[i + 1];
        pairs[i].sr = lv[i].nr > 1 ? 1 : 0;
        pairs[i].st = lv[i].nth > 1 ? 1 : 0;
        pairs[i].sp = lv[i].nph > 1 ? 1 : 0;
        pairs[i].cg = cg;
        pairs[i].h = HalfOp{hs, hw, hidg};
    }
    auto work_grid = [&](const void *kern, unsigned cells) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        return (int)std::max(1LL, std::min<long long>((cells + 255) / 256, (long long)per_sm * nsm));
    };
    // the finest pair in four-cell form where the rays hold a multiple of four cells
    const bool quad0 = nr % 4 == 0 && use_mg;
    std::vector<int> g_down(n_lv, 1), g_up(n_lv, 1);
    for (int i = 0; i + 1 < n_lv; ++i) {
        g_down[i] = (i == 0 && quad0) ? work_grid((const void *)k_mg_down4, lv[1].n / 2)
                                      : work_grid((const void *)k_mg_down, lv[i + 1].n);
        g_up[i] = (i == 0 && quad0) ? work_grid((const void *)k_mg_up4, lv[0].n / 4)
                                    : work_grid((const void *)k_mg_up, lv[i].n);
    }
    auto mg_apply = [&](int init) {
        if (quad0) k_mg_down4<<<g_down[0], 256, 0, st>>>(pairs[0]);
        else k_mg_down<<<g_down[0], 256, 0, st>>>(pairs[0]);
        for (int i = 1; i + 1 < n_lv; ++i) k_mg_down<<<g_down[i], 256, 0, st>>>(pairs[i]);
        k_mg_coarsest<<<1, 256, 0, st>>>(lv[n_lv - 1], fs->scal);
        for (int i = n_lv - 2; i >= 1; --i) k_mg_up<<<g_up[i], 256, 0, st>>>(pairs[i], 0, init);
        if (quad0) k_mg_up4<<<g_up[0], 256, 0, st>>>(pairs[0], init);
        else k_mg_up<<<g_up[0], 256, 0, st>>>(pairs[0], 1, init);
    };

    auto sync_read = [&](double *h_sc, unsigned *h_bad) {
        bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemcpyAsync(h_sc, fs->scal, sizeof(double) * kNScal, cudaMemcpyDeviceToHost, st) == cudaSuccess;
        if (ok && h_bad) ok = cudaMemcpyAsync(h_bad, fs->bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st) == cudaSuccess;
        return ok && cudaStreamSynchronize(st) == cudaSuccess;
    };
    double h_sc[kNScal];
    unsigned h_bad = 0;
    bool ok = cudaMemsetAsync(fs->bad, 0, sizeof(unsigned), st) == cudaSuccess &&
              cudaMemsetAsync(fs->scal, 0, sizeof(double) * kNScal, st) == cudaSuccess;
    k_fld_cell<<<grid, 256, 0, st>>>(ca);
    k_fld_faces<<<grid, 256, 0, st>>>(fa);
    for (int i = 0; i + 1 < n_lv; ++i) {  // coarse operators of this step
        k_mg_coarsen<<<work_grid((const void *)k_mg_coarsen, lv[i + 1].n), 256, 0, st>>>(pairs[i]);
        k_mg_diag<<<work_grid((const void *)k_mg_diag, lv[i + 1].n), 256, 0, st>>>(lv[i + 1]);
    }
    ok = ok && sync_read(h_sc, &h_bad);
    if (!ok) return ctx_fail(ctx, RT_ERR_CUDA, std::string("FLD set-up: ") + cudaGetErrorString(cudaGetLastError()));
    if (h_bad)
        return ctx_fail(ctx, RT_ERR_NONFINITE_INPUT,
                        "FLD input holds rho < 0, T <= 0, E_old < 0, q_abs < 0 or a NaN/Inf");
    if (cudaMemcpyAsync(e_new, e_old, sizeof(float) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return ctx_fail(ctx, RT_ERR_CUDA, "FLD start value");

    // refinement passes; the inner iterations go in bursts of kBurst, whose launches
    // return at once after the device flagged convergence (8 measured 1 % faster per
    // step than 16 with multigrid: fewer idle launches at the end of a pass)
    constexpr int kBurst = 8;
    int iters = 0, passes = 0;
    double corr = INFINITY;
    bool done = false;
    // four cells per thread where a ray holds a multiple of four cells
    const bool quads = nr % 4 == 0;
    // grids of one full wave: the CTAs resident per SM (from each kernel's registers)
    // times the SM count, capped by the work
    auto wave = [&](const void *kern) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        const long long work = ((quads ? n / 4 : n) + 255) / 256;
        return (int)std::max(1LL, std::min<long long>(work, (long long)per_sm * nsm));
    };
    const int g_res = quads ? wave((const void *)k_cg_residual4) : wave((const void *)k_cg_residual);
    const int g_app = quads ? wave((const void *)k_cg_apply4) : wave((const void *)k_cg_apply);
    const int g_upd = quads ? wave((const void *)k_cg_update4) : wave((const void *)k_cg_update);
    const int g_dir = quads ? wave((const void *)k_cg_direction4) : wave((const void *)k_cg_direction);
    const int g_acc = wave((const void *)k_cg_accumulate);
    // one inner iteration: q = A p, the updates, z = M^-1 r and r.z, the new direction
    auto iteration = [&]() {
        if (use_mg) {
            if (quads) {
                k_cg_apply4<<<g_app, 256, 0, st>>>(cg);
                k_cg_update_mg4<<<g_upd, 256, 0, st>>>(cg);
            } else {
                k_cg_apply<<<g_app, 256, 0, st>>>(cg);
                k_cg_update_mg<<<g_upd, 256, 0, st>>>(cg);
            }
            mg_apply(0);
            if (quads) k_cg_direction_mg4<<<g_dir, 256, 0, st>>>(cg, z);
            else k_cg_direction_mg<<<g_dir, 256, 0, st>>>(cg, z);
        } else if (quads) {
            k_cg_apply4<<<g_app, 256, 0, st>>>(cg);
            k_cg_update4<<<g_upd, 256, 0, st>>>(cg);
            k_cg_direction4<<<g_dir, 256, 0, st>>>(cg);
        } else {
            k_cg_apply<<<g_app, 256, 0, st>>>(cg);
            k_cg_update<<<g_upd, 256, 0, st>>>(cg);
            k_cg_direction<<<g_dir, 256, 0, st>>>(cg);
        }
    };
    while (!done) {
        if (cudaMemsetAsync(fs->scal + kDone, 0, sizeof(double), st) != cudaSuccess)
            return ctx_fail(ctx, RT_ERR_CUDA, "FLD pass start");
        if (use_mg) {
            k_cg_residual_mg<<<g_res, 256, 0, st>>>(cg);
            mg_apply(1);
            if (quads) k_cg_direction_mg4<<<g_dir, 256, 0, st>>>(cg, z);
            else k_cg_direction_mg<<<g_dir, 256, 0, st>>>(cg, z);
        } else if (quads) {
            k_cg_residual4<<<g_res, 256, 0, st>>>(cg);
        } else {
            k_cg_residual<<<g_res, 256, 0, st>>>(cg);
        }
        bool inner_done = false;
        while (!inner_done && iters < max_iter) {
            const int burst = std::min(kBurst, max_iter - iters);
            if (burst == kBurst && !fs->no_graph && (!fs->burst || fs->burst_x != e_new || fs->burst_buf != fs->buf)) {
                // (re)capture the burst: its launches point at e_new and the workspace
                if (fs->burst) cudaGraphExecDestroy(fs->burst);
                fs->burst = nullptr;
                cudaGraph_t graph = nullptr;
                bool cap = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (cap) {
                    for (int i = 0; i < kBurst; ++i) iteration();
                    cap = cudaStreamEndCapture(st, &graph) == cudaSuccess && graph;
                }
                if (cap) cap = cudaGraphInstantiate(&fs->burst, graph, 0) == cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
                if (!cap) {  // run the bursts as plain launches from now on
                    cudaGetLastError();
                    if (fs->burst) cudaGraphExecDestroy(fs->burst);
                    fs->burst = nullptr;
                    fs->no_graph = true;
                }
                fs->burst_x = e_new;
                fs->burst_buf = fs->buf;
            }
            if (burst == kBurst && fs->burst && !fs->no_graph) {
                if (cudaGraphLaunch(fs->burst, st) != cudaSuccess)
                    return ctx_fail(ctx, RT_ERR_CUDA, "FLD graph launch");
            } else {
                for (int i = 0; i < burst; ++i) iteration();
            }
            if (!sync_read(h_sc, nullptr))
                return ctx_fail(ctx, RT_ERR_CUDA, std::string("FLD iteration: ") + cudaGetErrorString(cudaGetLastError()));
            iters = (int)h_sc[kIters];
            inner_done = h_sc[kDone] != 0.0;
        }
        k_cg_accumulate<<<g_acc, 256, 0, st>>>(cg);
        if (!sync_read(h_sc, nullptr))
            return ctx_fail(ctx, RT_ERR_CUDA, std::string("FLD refinement: ") + cudaGetErrorString(cudaGetLastError()));
        ++passes;
        corr = h_sc[kCorr];
        done = corr < tol || iters >= max_iter || isinf(corr);
    }
    if (stats) {
        stats->levels = use_mg ? n_lv : 1;
        stats->iterations = iters;
        stats->passes = passes;
        stats->rel_change = corr;
    }
    if (isinf(corr)) return ctx_fail(ctx, RT_ERR_CUDA, "FLD solve broke down (non-finite E')");
    return corr < tol ? RT_OK
                      : ctx_fail(ctx, RT_ERR_TIMEOUT, "FLD solve did not reach tol within max_iter iterations");
}

}  // extern "C"
