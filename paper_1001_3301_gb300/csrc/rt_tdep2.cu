// Tracer for temperature-dependent opacity tables of low rank R (2 <= R <= 4): every
// entry of the table is
//   kappa_i(T_j) = sum_r A_ir B_rj,
// as for a mixture of R dust species whose abundances change with T. Linear
// interpolation in T keeps that form (b_r(T) interpolates B_r), so the optical depth
// of every bin is a combination of R columns shared by all bins (Eq. 19):
//   tau_i,in(k) = sum_r A_ir N_r,in(k),   N_r,in(k) = sum_{k' < k} b_r(T_k') rho_k' dr_k'.
// The R columns are scanned once per ray, not once per bin as in rt_tdep.cu; per
// (cell, bin) the kernel forms the exponent and the cell's own optical depth from
// them (R FMAs each), then the attenuated flux (Eq. 17) and the absorbed fraction
// (Eqs. 31-32, 36) in the Taylor and mixed classes of rt_device.cuh. For R = 2 the
// factors are two of the table's own columns and their non-negative weights (every
// term of every sum non-negative); for R = 3, 4 they come from the table's singular
// vectors and may carry either sign (the set-up accepts them where they reproduce
// every entry to 1e-10 of its row's largest value).
//
// One warp per ray, lane l owns cells [l C, (l+1) C), pairs of cells in f32x2
// registers. The bins are ordered by their largest tabulated kappa, which bounds the
// cell's dtau_i for the classes (kappa_i(T) <= max_j kappa_i(T_j) between the points).
// Two kernels: k_ray_tdep_two for R = 2 (two named columns) and k_ray_tdep2 for R = 3, 4.
#include "rt_device.cuh"

namespace rt {
namespace {

struct RankTab {
    const float4 *kr;  // [nnu_pad] (-A_i1 log2 e, .., -A_iR log2 e) of every sorted bin
    const float4 *bw;  // [n_t] (B_1j, .., B_Rj) at every grid point
    const float *tg;   // [n_t] temperature grid (K)
    int n_t;
};

// component r of v (r a compile-time constant where it is called)
__device__ __forceinline__ float comp(const float4 &v, int r)
{
    return r == 0 ? v.x : (r == 1 ? v.y : (r == 2 ? v.z : v.w));
}

// The two-column kernel (rank two; the per-bin loops with two named columns, which
// compile to fewer instructions than the rank-R form below instantiated for R = 2).
// Bins [i0, i1) of one class for the lane's cells. Zero-density dust cells carry
// (b_1, b_2) in place of their (zero) column steps, so y = -kappa_i(T) log2 e there:
// their a_rad limit sums g kappa_i = -g y ln 2 (a02; ZERO: the warp holds such a cell).
// Class 1 (one Taylor term, 1 - 2^y = p0 y) in the moment form: with y = k1 d1 + k2 d2,
// sum_i g_i p0 y_i = p0 (d1 sum_i g_i k1_i + d2 sum_i g_i k2_i), two FMAs per (cell, bin).
template <int CLASS, int C, bool ZERO>
__device__ __forceinline__ void rank2_range(int i0, int i1, const float *s_lf, const float4 *s_ab,
                                            const float2 (&n1)[C / 2], const float2 (&n2)[C / 2],
                                            const float2 (&d1)[C / 2], const float2 (&d2)[C / 2],
                                            float2 (&a2)[C / 2], float2 (&a02)[C / 2])
{
    if constexpr (CLASS == 1) {
        if (i0 >= i1) return;  // warp-uniform
        float2 m1[C / 2], m2[C / 2];
#pragma unroll
        for (int m = 0; m < C / 2; ++m) m1[m] = m2[m] = f2(0.0f);
#pragma unroll 2
        for (int i = i0; i < i1; ++i) {
            const float4 e = s_ab[i];
            const float2 k1 = f2(e.x), k2 = f2(e.y), lf = f2(s_lf[i]);
#pragma unroll
            for (int m = 0; m < C / 2; ++m) {
                const float2 g = ex2_approx2(__ffma2_rn(k1, n1[m], __ffma2_rn(k2, n2[m], lf)));
                m1[m] = __ffma2_rn(g, k1, m1[m]);
                m2[m] = __ffma2_rn(g, k2, m2[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float2 gy = __ffma2_rn(d1[m], m1[m], __fmul2_rn(d2[m], m2[m]));  // sum_i g_i y_i
            a2[m] = __ffma2_rn(f2((float)taylor_coeff(0)), gy, a2[m]);
            if constexpr (ZERO) a02[m] = __fadd2_rn(a02[m], gy);
        }
        return;
    }
#pragma unroll(CLASS <= 2 ? 2 : 1)
    for (int i = i0; i < i1; ++i) {
        const float4 e = s_ab[i];
        const float2 k1 = f2(e.x), k2 = f2(e.y), lf = f2(s_lf[i]);
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float2 g = ex2_approx2(__ffma2_rn(k1, n1[m], __ffma2_rn(k2, n2[m], lf)));
            const float2 y = __ffma2_rn(k1, d1[m], __fmul2_rn(k2, d2[m]));  // -dtau log2 e
            float2 om;                                                       // 1 - 2^y
            if constexpr (CLASS <= 5) {
                om = taylor_fraction<CLASS>(y);
            } else {
                // the smaller of the 5-term series and 1 - ex2(y) + 2^-22, as in bin_range
                const float2 big = __ffma2_rn(ex2_approx2(y), f2(-1.0f), f2(1.0f + 0x1p-22f));
                const float2 small = taylor_fraction<5>(y);
                om = make_float2(fminf(small.x, big.x), fminf(small.y, big.y));
            }
            a2[m] = __ffma2_rn(g, om, a2[m]);
            if constexpr (ZERO) a02[m] = __ffma2_rn(g, y, a02[m]);
        }
    }
}

// every class range of one warp
template <int C, bool ZERO>
__device__ __forceinline__ void rank2_ranges(const BinClasses &bc, int na, const float *s_lf, const float4 *s_ab,
                                             const float2 (&n1)[C / 2], const float2 (&n2)[C / 2],
                                             const float2 (&d1)[C / 2], const float2 (&d2)[C / 2],
                                             float2 (&a2)[C / 2], float2 (&a02)[C / 2])
{
    rank2_range<1, C, ZERO>(0, bc.b1, s_lf, s_ab, n1, n2, d1, d2, a2, a02);
    rank2_range<2, C, ZERO>(bc.b1, bc.b2, s_lf, s_ab, n1, n2, d1, d2, a2, a02);
    rank2_range<3, C, ZERO>(bc.b2, bc.b3, s_lf, s_ab, n1, n2, d1, d2, a2, a02);
    rank2_range<5, C, ZERO>(bc.b3, bc.b5, s_lf, s_ab, n1, n2, d1, d2, a2, a02);
    rank2_range<6, C, ZERO>(bc.b5, na, s_lf, s_ab, n1, n2, d1, d2, a2, a02);
}

template <int C, int W, int MINB>
__global__ void __launch_bounds__(W * 32, MINB) k_ray_tdep_two(const TraceArgs p, const RankTab t)
{
    static_assert(C % 2 == 0, "pairs of cells");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nr = p.nr;
    const int c0 = lane * C;
    const int nv = nr - c0 < 0 ? 0 : (nr - c0 > C ? C : nr - c0);

    __shared__ float s_dr[C][32], s_gq[C][32], s_ga[C][32];
    __shared__ float s_tg[kMaxTdepPoints], s_idt[kMaxTdepPoints];  // grid, 1 / (T_{j+1} - T_j)
    __shared__ float4 s_bw[kMaxTdepPoints];
    __shared__ KahanSum s_red[W][2];
    extern __shared__ float4 smem4[];
    float4 *s_nu = smem4;                                       // [nnu_pad] (nk_max, ., lf, .)
    float4 *s_ab = s_nu + p.nnu_pad;                            // [nnu_pad] (-A_1 log2 e, -A_2 log2 e, ., .)
    float *s_lf = reinterpret_cast<float *>(s_ab + p.nnu_pad);  // [nnu_pad]

    for (int i = tid; i < p.nnu_pad; i += W * 32) {
        const NuEntry e = p.nu[i];
        s_nu[i] = make_float4(e.nk, e.nk, e.lf, e.lf);
        s_lf[i] = e.lf;
        s_ab[i] = t.kr[i];
    }
    for (int i = tid; i < t.n_t; i += W * 32) {  // the weights of both ends of every interval
        s_tg[i] = t.tg[i];
        s_idt[i] = i + 1 < t.n_t ? 1.0f / (t.tg[i + 1] - t.tg[i]) : 0.0f;
        const float4 b0 = t.bw[i], b1 = t.bw[i + 1 < t.n_t ? i + 1 : i];
        s_bw[i] = make_float4(b0.x, b1.x, b0.y, b1.y);
    }
    for (int i = tid; i < 32 * C; i += W * 32) {
        const int l = i / C, j = i % C, k = l * C + j;
        const float4 g = (k < nr) ? __ldg(&p.rtab[k]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        s_dr[j][l] = g.x;
        s_gq[j][l] = g.y;
        s_ga[j][l] = g.z;
    }
    __syncthreads();
    const int nt = t.n_t;
    const int na = p.n_active;

    KahanSum eabs, eesc;
    eabs.zero();
    eesc.zero();
    for (unsigned ray = blockIdx.x * W + warp; ray < p.nrays; ray += gridDim.x * W) {
        const size_t base = (size_t)ray * nr + c0;
        float2 d1[C / 2], d2[C / 2], n1[C / 2], n2[C / 2], acc[C / 2], acc0[C / 2];
        float dc[C];  // the cell's column rho dr (dust only)
        float b1z[C], b2z[C];
        unsigned zero_m = 0;
        bool bad = false;
        float dmax = 0.0f;
        float ls1 = 0.0f, ls2 = 0.0f;  // the lane's sums (plain FP32, at most C terms)
#pragma unroll
        for (int j = 0; j < C; ++j) {
            float rho = 0.0f, td = 0.0f;
            if (j < nv) {
                rho = __ldg(p.rho + base + j);
                td = __ldg(p.tdust + base + j);
                bad |= !(rho >= 0.0f && rho <= FLT_MAX) || (td != td);
            }
            const bool dust = j < nv && td <= p.t_sub;
            const float dj = dust ? rho * s_dr[j][lane] : 0.0f;
            dc[j] = dj;
            if (dust && dj == 0.0f) zero_m |= 1u << j;
            dmax = fmaxf(dmax, dj);
            // bracketing temperature points, the weights of the upper and the lower one,
            // and the two column weights (sums of non-negative terms)
            int lo = 0;
            for (int s = 16; s > 0; s >>= 1)
                if (lo + s < nt - 1 && s_tg[lo + s] <= td) lo += s;
            const float wt = fminf(fmaxf((td - s_tg[lo]) * s_idt[lo], 0.0f), 1.0f);
            const float wb = fminf(fmaxf((s_tg[lo + 1] - td) * s_idt[lo], 0.0f), 1.0f);
            const float4 bw = s_bw[lo];
            b1z[j] = fmaf(bw.y, wt, bw.x * wb);
            b2z[j] = fmaf(bw.w, wt, bw.z * wb);
            const float e1 = b1z[j] * dj, e2 = b2z[j] * dj;
            if (j % 2 == 0) {
                d1[j / 2].x = e1;
                d2[j / 2].x = e2;
            } else {
                d1[j / 2].y = e1;
                d2[j / 2].y = e2;
            }
            ls1 += e1;
            ls2 += e2;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(p.bad_input, p.seq);
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        const bool any_zero = __any_sync(0xffffffffu, zero_m != 0u);

        // compensated warp scans of the two lane sums, interleaved
        KahanSum i1, i2;
        i1.zero();
        i2.zero();
        i1.add(ls1);
        i2.add(ls2);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const KahanSum v1 = i1.shfl_up(o), v2 = i2.shfl_up(o);
            if (lane >= o) {
                i1.add(v1);
                i2.add(v2);
            }
        }
        const float tot1 = __shfl_sync(0xffffffffu, i1.value(), 31);
        const float tot2 = __shfl_sync(0xffffffffu, i2.value(), 31);
        KahanSum p1 = i1.shfl_up(1), p2 = i2.shfl_up(1);
        if (lane == 0) {
            p1.zero();
            p2.zero();
        }
        // each cell's columns in front of it: the warp offset (hi + lo) plus the lane's
        // plain partial sum
        float q1 = 0.0f, q2 = 0.0f;
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            n1[m].x = p1.hi + (p1.lo + q1);
            n2[m].x = p2.hi + (p2.lo + q2);
            q1 += d1[m].x;
            q2 += d2[m].x;
            n1[m].y = p1.hi + (p1.lo + q1);
            n2[m].y = p2.hi + (p2.lo + q2);
            q1 += d1[m].y;
            q2 += d2[m].y;
            acc[m] = f2(0.0f);
            acc0[m] = f2(0.0f);
        }
        // zero-density dust cells: their column steps (zero) become (b_1, b_2)
        if (any_zero) {
#pragma unroll
            for (int j = 0; j < C; ++j)
                if ((zero_m >> j) & 1u) {
                    if (j % 2 == 0) {
                        d1[j / 2].x = b1z[j];
                        d2[j / 2].x = b2z[j];
                    } else {
                        d1[j / 2].y = b1z[j];
                        d2[j / 2].y = b2z[j];
                    }
                }
        }

        const BinClasses bc = classify_bins(s_nu, na, lane, dmax, 0.0f);
        if (any_zero) rank2_ranges<C, true>(bc, na, s_lf, s_ab, n1, n2, d1, d2, acc, acc0);
        else rank2_ranges<C, false>(bc, na, s_lf, s_ab, n1, n2, d1, d2, acc, acc0);

        // the flux leaving the ray, bins spread over the lanes (Eq. 33)
        float esc = 0.0f;
        for (int i = lane; i < na; i += 32) {
            const float4 e = s_ab[i];
            esc += ex2_approx(fmaf(e.x, tot1, fmaf(e.y, tot2, s_lf[i])));
        }
        const float w = __ldg(p.domega32 + ray);
        eesc.add(esc * w);
        float lane_abs = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const bool zc = (zero_m >> j) & 1u;
            const float aj = j % 2 == 0 ? acc[j / 2].x : acc[j / 2].y;
            const float a0 = (j % 2 == 0 ? acc0[j / 2].x : acc0[j / 2].y) * -(float)kLn2;
            const float dj = dc[j];
            const float qv = zc ? 0.0f : s_gq[j][lane] * aj;
            const float av = s_ga[j][lane] * (zc ? a0 : (dj > 0.0f ? __fdividef(aj, dj) : 0.0f));
            lane_abs += (j < nv && !zc) ? aj : 0.0f;
            if (j < nv) {
                p.q[base + j] = qv;
                p.a[base + j] = av;
            }
        }
        eabs.add(lane_abs * w);
    }

    for (int o = 16; o > 0; o >>= 1) {
        eabs.add(eabs.shfl_xor(o));
        eesc.add(eesc.shfl_xor(o));
    }
    if (lane == 0) {
        s_red[warp][0] = eabs;
        s_red[warp][1] = eesc;
    }
    __syncthreads();
    if (tid == 0) {
        KahanSum sa = s_red[0][0], se = s_red[0][1];
        for (int w2 = 1; w2 < W; ++w2) {
            sa.add(s_red[w2][0]);
            se.add(s_red[w2][1]);
        }
        p.partials[blockIdx.x] = make_double2(to_double(sa), to_double(se));
    }
}

// Bins [i0, i1) of one class for the lane's cells. Zero-density dust cells carry
// (b_1, .., b_R) in place of their (zero) column steps, so y = -kappa_i(T) log2 e there:
// their a_rad limit sums g kappa_i = -g y ln 2 (a02; ZERO: the warp holds such a cell).
// Class 1 (one Taylor term, 1 - 2^y = p0 y) in the moment form: with y = sum_r k_r d_r,
// sum_i g_i p0 y_i = p0 sum_r d_r sum_i g_i k_ri, R FMAs per (cell, bin).
template <int CLASS, int C, int R, bool ZERO>
__device__ __forceinline__ void rank_range(int i0, int i1, const float *s_lf, const float4 *s_kr,
                                           const float2 (&n)[R][C / 2], const float2 (&d)[R][C / 2],
                                           float2 (&a2)[C / 2], float2 (&a02)[C / 2])
{
    if constexpr (CLASS == 1) {
        if (i0 >= i1) return;  // warp-uniform
        float2 mo[R][C / 2];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int m = 0; m < C / 2; ++m) mo[r][m] = f2(0.0f);
#pragma unroll 2
        for (int i = i0; i < i1; ++i) {
            const float4 e = s_kr[i];
            const float2 lf = f2(s_lf[i]);
            float2 kk[R];  // the bin's coefficients, splat once per bin
#pragma unroll
            for (int r = 0; r < R; ++r) kk[r] = f2(comp(e, r));
#pragma unroll
            for (int m = 0; m < C / 2; ++m) {
                float2 x = lf;
#pragma unroll
                for (int r = R - 1; r >= 0; --r) x = __ffma2_rn(kk[r], n[r][m], x);
                const float2 g = ex2_approx2(x);
#pragma unroll
                for (int r = 0; r < R; ++r) mo[r][m] = __ffma2_rn(g, kk[r], mo[r][m]);
            }
        }
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            float2 gy = __fmul2_rn(d[R - 1][m], mo[R - 1][m]);  // sum_i g_i y_i
#pragma unroll
            for (int r = R - 2; r >= 0; --r) gy = __ffma2_rn(d[r][m], mo[r][m], gy);
            a2[m] = __ffma2_rn(f2((float)taylor_coeff(0)), gy, a2[m]);
            if constexpr (ZERO) a02[m] = __fadd2_rn(a02[m], gy);
        }
        return;
    }
#pragma unroll(CLASS <= 2 ? 2 : 1)
    for (int i = i0; i < i1; ++i) {
        const float4 e = s_kr[i];
        const float2 lf = f2(s_lf[i]);
        float2 kk[R];  // the bin's coefficients, splat once per bin
#pragma unroll
        for (int r = 0; r < R; ++r) kk[r] = f2(comp(e, r));
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            float2 x = lf;
#pragma unroll
            for (int r = R - 1; r >= 0; --r) x = __ffma2_rn(kk[r], n[r][m], x);
            const float2 g = ex2_approx2(x);
            float2 y = __fmul2_rn(kk[R - 1], d[R - 1][m]);  // -dtau log2 e
#pragma unroll
            for (int r = R - 2; r >= 0; --r) y = __ffma2_rn(kk[r], d[r][m], y);
            float2 om;  // 1 - 2^y
            if constexpr (CLASS <= 5) {
                om = taylor_fraction<CLASS>(y);
            } else {
                // the smaller of the 5-term series and 1 - ex2(y) + 2^-22, as in bin_range
                const float2 big = __ffma2_rn(ex2_approx2(y), f2(-1.0f), f2(1.0f + 0x1p-22f));
                const float2 small = taylor_fraction<5>(y);
                om = make_float2(fminf(small.x, big.x), fminf(small.y, big.y));
            }
            a2[m] = __ffma2_rn(g, om, a2[m]);
            if constexpr (ZERO) a02[m] = __ffma2_rn(g, y, a02[m]);
        }
    }
}

// every class range of one warp
template <int C, int R, bool ZERO>
__device__ __forceinline__ void rank_ranges(const BinClasses &bc, int na, const float *s_lf, const float4 *s_kr,
                                            const float2 (&n)[R][C / 2], const float2 (&d)[R][C / 2],
                                            float2 (&a2)[C / 2], float2 (&a02)[C / 2])
{
    rank_range<1, C, R, ZERO>(0, bc.b1, s_lf, s_kr, n, d, a2, a02);
    rank_range<2, C, R, ZERO>(bc.b1, bc.b2, s_lf, s_kr, n, d, a2, a02);
    rank_range<3, C, R, ZERO>(bc.b2, bc.b3, s_lf, s_kr, n, d, a2, a02);
    rank_range<5, C, R, ZERO>(bc.b3, bc.b5, s_lf, s_kr, n, d, a2, a02);
    rank_range<6, C, R, ZERO>(bc.b5, na, s_lf, s_kr, n, d, a2, a02);
}

// the column weights b_r(T) of one cell: T's bracketing points found by a five-step
// binary search, then linear in T between them (the end values beyond the grid)
template <int R>
__device__ __forceinline__ void column_weights(float td, const float *s_tg, const float *s_idt, const float4 *s_bw,
                                               int nt, float (&b)[R])
{
    int lo = 0;
    for (int s = 16; s > 0; s >>= 1)
        if (lo + s < nt - 1 && s_tg[lo + s] <= td) lo += s;
    const float wt = fminf(fmaxf((td - s_tg[lo]) * s_idt[lo], 0.0f), 1.0f);
    const float wb = fminf(fmaxf((s_tg[lo + 1] - td) * s_idt[lo], 0.0f), 1.0f);
    const float4 b0 = s_bw[lo], b1 = s_bw[lo + 1];
#pragma unroll
    for (int r = 0; r < R; ++r) b[r] = fmaf(comp(b1, r), wt, comp(b0, r) * wb);
}

template <int C, int W, int MINB, int R>
__global__ void __launch_bounds__(W * 32, MINB) k_ray_tdep2(const TraceArgs p, const RankTab t)
{
    static_assert(C % 2 == 0, "pairs of cells");
    static_assert(R >= 3 && R <= 4, "three or four columns (two: k_ray_tdep_two)");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nr = p.nr;
    const int c0 = lane * C;
    const int nv = nr - c0 < 0 ? 0 : (nr - c0 > C ? C : nr - c0);

    __shared__ float s_dr[C][32], s_gq[C][32], s_ga[C][32];
    __shared__ float s_tg[kMaxTdepPoints], s_idt[kMaxTdepPoints];  // grid, 1 / (T_{j+1} - T_j)
    __shared__ float4 s_bw[kMaxTdepPoints];
    __shared__ KahanSum s_red[W][2];
    extern __shared__ float4 smem4[];
    float4 *s_nu = smem4;                                       // [nnu_pad] (nk_max, ., lf, .)
    float4 *s_kr = s_nu + p.nnu_pad;                            // [nnu_pad]
    float *s_lf = reinterpret_cast<float *>(s_kr + p.nnu_pad);  // [nnu_pad]

    for (int i = tid; i < p.nnu_pad; i += W * 32) {
        const NuEntry e = p.nu[i];
        s_nu[i] = make_float4(e.nk, e.nk, e.lf, e.lf);
        s_lf[i] = e.lf;
        s_kr[i] = t.kr[i];
    }
    for (int i = tid; i < t.n_t; i += W * 32) {
        s_tg[i] = t.tg[i];
        s_idt[i] = i + 1 < t.n_t ? 1.0f / (t.tg[i + 1] - t.tg[i]) : 0.0f;
        s_bw[i] = t.bw[i];
    }
    for (int i = tid; i < 32 * C; i += W * 32) {
        const int l = i / C, j = i % C, k = l * C + j;
        const float4 g = (k < nr) ? __ldg(&p.rtab[k]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        s_dr[j][l] = g.x;
        s_gq[j][l] = g.y;
        s_ga[j][l] = g.z;
    }
    __syncthreads();
    const int nt = t.n_t;
    const int na = p.n_active;

    KahanSum eabs, eesc;
    eabs.zero();
    eesc.zero();
    for (unsigned ray = blockIdx.x * W + warp; ray < p.nrays; ray += gridDim.x * W) {
        const size_t base = (size_t)ray * nr + c0;
        float2 d[R][C / 2], n[R][C / 2], acc[C / 2], acc0[C / 2];
        float dc[C];      // the cell's column rho dr (dust only)
        float bz[R][C];   // its column weights (kept for the zero-density cells)
        unsigned zero_m = 0;
        bool bad = false;
        float dmax = 0.0f;
        float ls[R];  // the lane's sums (plain FP32, at most C terms)
#pragma unroll
        for (int r = 0; r < R; ++r) ls[r] = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            float rho = 0.0f, td = 0.0f;
            if (j < nv) {
                rho = __ldg(p.rho + base + j);
                td = __ldg(p.tdust + base + j);
                bad |= !(rho >= 0.0f && rho <= FLT_MAX) || (td != td);
            }
            const bool dust = j < nv && td <= p.t_sub;
            const float dj = dust ? rho * s_dr[j][lane] : 0.0f;
            dc[j] = dj;
            if (dust && dj == 0.0f) zero_m |= 1u << j;
            dmax = fmaxf(dmax, dj);
            float b[R];
            column_weights<R>(td, s_tg, s_idt, s_bw, nt, b);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                bz[r][j] = b[r];
                const float e = b[r] * dj;
                if (j % 2 == 0) d[r][j / 2].x = e;
                else d[r][j / 2].y = e;
                ls[r] += e;
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(p.bad_input, p.seq);
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        const bool any_zero = __any_sync(0xffffffffu, zero_m != 0u);

        // compensated warp scans of the R lane sums, interleaved
        KahanSum inc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            inc[r].zero();
            inc[r].add(ls[r]);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            KahanSum v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = inc[r].shfl_up(o);
            if (lane >= o) {
#pragma unroll
                for (int r = 0; r < R; ++r) inc[r].add(v[r]);
            }
        }
        float tot[R];
        float q[R];
        KahanSum pre[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            tot[r] = __shfl_sync(0xffffffffu, inc[r].value(), 31);
            pre[r] = inc[r].shfl_up(1);
            if (lane == 0) pre[r].zero();
            q[r] = 0.0f;
        }
        // each cell's columns in front of it: the warp offset (hi + lo) plus the lane's
        // plain partial sum
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                n[r][m].x = pre[r].hi + (pre[r].lo + q[r]);
                q[r] += d[r][m].x;
                n[r][m].y = pre[r].hi + (pre[r].lo + q[r]);
                q[r] += d[r][m].y;
            }
            acc[m] = f2(0.0f);
            acc0[m] = f2(0.0f);
        }
        // zero-density dust cells: their column steps (zero) become (b_1, .., b_R)
        if (any_zero) {
#pragma unroll
            for (int j = 0; j < C; ++j)
                if ((zero_m >> j) & 1u) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (j % 2 == 0) d[r][j / 2].x = bz[r][j];
                        else d[r][j / 2].y = bz[r][j];
                    }
                }
        }

        const BinClasses bc = classify_bins(s_nu, na, lane, dmax, 0.0f);
        if (any_zero) rank_ranges<C, R, true>(bc, na, s_lf, s_kr, n, d, acc, acc0);
        else rank_ranges<C, R, false>(bc, na, s_lf, s_kr, n, d, acc, acc0);

        // the flux leaving the ray, bins spread over the lanes (Eq. 33)
        float esc = 0.0f;
        for (int i = lane; i < na; i += 32) {
            const float4 e = s_kr[i];
            float x = s_lf[i];
#pragma unroll
            for (int r = R - 1; r >= 0; --r) x = fmaf(comp(e, r), tot[r], x);
            esc += ex2_approx(x);
        }
        const float w = __ldg(p.domega32 + ray);
        eesc.add(esc * w);
        float lane_abs = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const bool zc = (zero_m >> j) & 1u;
            const float aj = j % 2 == 0 ? acc[j / 2].x : acc[j / 2].y;
            const float a0 = (j % 2 == 0 ? acc0[j / 2].x : acc0[j / 2].y) * -(float)kLn2;
            const float dj = dc[j];
            const float qv = zc ? 0.0f : s_gq[j][lane] * aj;
            const float av = s_ga[j][lane] * (zc ? a0 : (dj > 0.0f ? __fdividef(aj, dj) : 0.0f));
            lane_abs += (j < nv && !zc) ? aj : 0.0f;
            if (j < nv) {
                p.q[base + j] = qv;
                p.a[base + j] = av;
            }
        }
        eabs.add(lane_abs * w);
    }

    for (int o = 16; o > 0; o >>= 1) {
        eabs.add(eabs.shfl_xor(o));
        eesc.add(eesc.shfl_xor(o));
    }
    if (lane == 0) {
        s_red[warp][0] = eabs;
        s_red[warp][1] = eesc;
    }
    __syncthreads();
    if (tid == 0) {
        KahanSum sa = s_red[0][0], se = s_red[0][1];
        for (int w2 = 1; w2 < W; ++w2) {
            sa.add(s_red[w2][0]);
            se.add(s_red[w2][1]);
        }
        p.partials[blockIdx.x] = make_double2(to_double(sa), to_double(se));
    }
}

// kr[a] = (-A_a1 log2 e, .., -A_aR log2 e) of the sorted active bin a (A: [n_nu][4],
// FP64); padding bins get zero opacity
__global__ void k_build_rank(int n_active, int nnu_pad, const double *fac_a, const int *order, float4 *kr)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nnu_pad) return;
    if (a >= n_active) {
        kr[a] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    const double *f = fac_a + 4 * order[a];
    kr[a] = make_float4((float)(-f[0] * kLog2e), (float)(-f[1] * kLog2e), (float)(-f[2] * kLog2e),
                        (float)(-f[3] * kLog2e));
}

template <int C, int W, int MINB, int R>
constexpr auto rank_kernel()
{
    if constexpr (R == 2) return k_ray_tdep_two<C, W, MINB>;
    else return k_ray_tdep2<C, W, MINB, R>;
}

template <int C, int W, int MINB, int R>
cudaError_t launch_rank_shape(const TraceArgs &a, const RankTab &t, cudaStream_t stream, unsigned *grid_out)
{
    const size_t smem = (size_t)a.nnu_pad * (16 + 16 + 4);
    auto kern = rank_kernel<C, W, MINB, R>();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    unsigned grid = (unsigned)nsm * (unsigned)per_sm;
    const unsigned need = (a.nrays + W - 1) / W;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<grid, W * 32, smem, stream>>>(a, t);
    *grid_out = grid;
    return cudaGetLastError();
}

struct RankEntry {
    int rank, c, w, minb;
    cudaError_t (*fn)(const TraceArgs &, const RankTab &, cudaStream_t, unsigned *);
};
#define RT_RK(R, C, W, MB) {R, C, W, MB, &launch_rank_shape<C, W, MB, R>}
const RankEntry kRankShapes[] = {
    RT_RK(2, 2, 4, 8), RT_RK(2, 4, 4, 8), RT_RK(2, 8, 4, 6), RT_RK(2, 8, 4, 4), RT_RK(2, 16, 4, 2), RT_RK(2, 32, 4, 1),
    RT_RK(3, 2, 4, 8), RT_RK(3, 4, 4, 6), RT_RK(3, 8, 4, 3), RT_RK(3, 16, 4, 2), RT_RK(3, 32, 4, 1),
    RT_RK(4, 2, 4, 8), RT_RK(4, 4, 4, 6), RT_RK(4, 8, 4, 3), RT_RK(4, 16, 4, 2), RT_RK(4, 32, 4, 1)};
#undef RT_RK

}  // namespace

// The shapes of rank R whose rays fill the warp: the fewest cells per lane that hold nr.
int tdep2_shapes(int rank, int nr, Shape *out, int max_out)
{
    int c_fit = 0;
    for (const RankEntry &s : kRankShapes)
        if (s.rank == rank && 32 * s.c >= nr && (c_fit == 0 || s.c < c_fit)) c_fit = s.c;
    int n = 0;
    for (const RankEntry &s : kRankShapes)
        if (s.rank == rank && s.c == c_fit && n < max_out) out[n++] = Shape{kKindRay, s.c, s.w, s.minb};
    return n;
}

cudaError_t launch_tdep2(int rank, Shape s, const TraceArgs &args, const float4 *kr, const float4 *bw, const float *tg,
                         int n_t, cudaStream_t stream, unsigned *grid_out)
{
    const RankTab t{kr, bw, tg, n_t};
    for (const RankEntry &e : kRankShapes)
        if (e.rank == rank && e.c == s.cells_per_lane && e.w == s.warps &&
            (s.min_blocks == 0 || e.minb == s.min_blocks) && 32 * e.c >= args.nr)
            return e.fn(args, t, stream, grid_out);
    return cudaErrorInvalidValue;
}

cudaError_t launch_build_rank2(int n_active, int nnu_pad, const double *fac_a, const int *order, float4 *kr,
                               cudaStream_t stream)
{
    k_build_rank<<<(nnu_pad + 127) / 128, 128, 0, stream>>>(n_active, nnu_pad, fac_a, order, kr);
    return cudaGetLastError();
}

}  // namespace rt
