// Tracer for temperature-dependent opacity tables of rank two: every entry of the
// table is a non-negative combination of two of its own columns,
//   kappa_i(T_j) = A_i1 B_1j + A_i2 B_2j,   A, B >= 0,
// as for a mixture of two dust species whose abundances change with T. Linear
// interpolation in T keeps that form (b_r(T) interpolates B_r), so the optical depth
// of every bin is a combination of two columns shared by all bins (Eq. 19):
//   tau_i,in(k) = A_i1 N_1,in(k) + A_i2 N_2,in(k),   N_r,in(k) = sum_{k' < k} b_r(T_k') rho_k' dr_k'.
// The two columns are scanned once per ray, not once per bin as in rt_tdep.cu; per
// (cell, bin) the kernel forms the exponent and the cell's own optical depth from
// them (two FMAs each), then the attenuated flux (Eq. 17) and the absorbed fraction
// (Eqs. 31-32, 36) in the Taylor, mixed and MUFU classes of rt_device.cuh.
//
// One warp per ray, lane l owns cells [l C, (l+1) C), pairs of cells in f32x2
// registers. The bins are ordered by their largest tabulated kappa, which bounds the
// cell's dtau_i for the classes (kappa_i(T) <= max_j kappa_i(T_j) between the points).
#include "rt_device.cuh"

namespace rt {
namespace {

struct Rank2Tab {
    const float4 *ab;  // [nnu_pad] (-A_1 log2 e, -A_2 log2 e, A_1, A_2) of every sorted bin
    const float4 *bw;  // [kMaxTdepPoints] (B_1j, B_1,j+1, B_2j, B_2,j+1)
    const float *tg;   // [n_t] temperature grid (K)
    int n_t;
};

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
__global__ void __launch_bounds__(W * 32, MINB) k_ray_tdep2(const TraceArgs p, const Rank2Tab t)
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
    float4 *s_ab = s_nu + p.nnu_pad;                            // [nnu_pad]
    float *s_lf = reinterpret_cast<float *>(s_ab + p.nnu_pad);  // [nnu_pad]

    for (int i = tid; i < p.nnu_pad; i += W * 32) {
        const NuEntry e = p.nu[i];
        s_nu[i] = make_float4(e.nk, e.nk, e.lf, e.lf);
        s_lf[i] = e.lf;
        s_ab[i] = t.ab[i];
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

// ab[a] = (-A_1 log2 e, -A_2 log2 e, A_1, A_2) of the sorted active bin a (A: [n_nu][2],
// FP64); padding bins get zero opacity
__global__ void k_build_rank2(int n_active, int nnu_pad, const double *fac_a, const int *order, float4 *ab)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nnu_pad) return;
    if (a >= n_active) {
        ab[a] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    const double a1 = fac_a[2 * order[a]], a2 = fac_a[2 * order[a] + 1];
    ab[a] = make_float4((float)(-a1 * kLog2e), (float)(-a2 * kLog2e), (float)a1, (float)a2);
}

template <int C, int W, int MINB>
cudaError_t launch_rank2_shape(const TraceArgs &a, const Rank2Tab &t, cudaStream_t stream, unsigned *grid_out)
{
    const size_t smem = (size_t)a.nnu_pad * (16 + 16 + 4);
    auto kern = k_ray_tdep2<C, W, MINB>;
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

struct Rank2Entry {
    int c, w, minb;
    cudaError_t (*fn)(const TraceArgs &, const Rank2Tab &, cudaStream_t, unsigned *);
};
#define RT_R2(C, W, MB) {C, W, MB, &launch_rank2_shape<C, W, MB>}
const Rank2Entry kRank2Shapes[] = {RT_R2(2, 4, 8), RT_R2(4, 4, 8), RT_R2(8, 4, 6), RT_R2(8, 4, 4),
                                   RT_R2(16, 4, 3), RT_R2(32, 4, 2)};
#undef RT_R2

}  // namespace

// The shapes whose rays fill the warp: the fewest cells per lane that hold nr.
int tdep2_shapes(int nr, Shape *out, int max_out)
{
    int c_fit = 0;
    for (const Rank2Entry &s : kRank2Shapes)
        if (32 * s.c >= nr && (c_fit == 0 || s.c < c_fit)) c_fit = s.c;
    int n = 0;
    for (const Rank2Entry &s : kRank2Shapes)
        if (s.c == c_fit && n < max_out) out[n++] = Shape{kKindRay, s.c, s.w, s.minb};
    return n;
}

cudaError_t launch_tdep2(Shape s, const TraceArgs &args, const float4 *ab, const float4 *bw, const float *tg, int n_t,
                         cudaStream_t stream, unsigned *grid_out)
{
    const Rank2Tab t{ab, bw, tg, n_t};
    for (const Rank2Entry &e : kRank2Shapes)
        if (e.c == s.cells_per_lane && e.w == s.warps && (s.min_blocks == 0 || e.minb == s.min_blocks) &&
            32 * e.c >= args.nr)
            return e.fn(args, t, stream, grid_out);
    return cudaErrorInvalidValue;
}

cudaError_t launch_build_rank2(int n_active, int nnu_pad, const double *fac_a, const int *order, float4 *ab,
                               cudaStream_t stream)
{
    k_build_rank2<<<(nnu_pad + 127) / 128, 128, 0, stream>>>(n_active, nnu_pad, fac_a, order, ab);
    return cudaGetLastError();
}

}  // namespace rt
