// Tracer with temperature-dependent opacity tables: kappa_i(T) per bin, linear in T
// between the points of a temperature grid (the ends beyond it), zero above the
// sublimation temperature. Each cell has its own kappa per bin, so the optical
// depth of every bin is its own scan along the ray (Eq. 19; no single column serves
// all bins as in rt_ray.cu):
//   tau_i,in(k) = sum_{k' < k} kappa_i(T_k') rho_k' dr_k',
// then the attenuated flux (Eq. 17) and the absorbed fraction of the cell
// (Eqs. 31-32, 36) per (cell, bin) as in the per-bin loop of rt_device.cuh.
//
// One warp per ray, lane l owns cells [l C, (l+1) C). The bins go in pairs (2p, 2p + 1),
// one f32x2 register per cell holding both: every cell's two kappa from the table (one
// 16-byte shared-memory read of both rows' bracketing points), the lane's two sums (C
// terms, plain FP32), one compensated warp scan of both (packed: half the scan
// instructions per bin), then a second pass over the lane's cells carrying the
// exclusive prefix (no per-cell prefix is stored).
// The bins are ordered by their largest tabulated kappa; the Taylor classes of the
// absorbed fraction (1, 2, 3, 5 terms) come from that largest kappa and the warp's
// largest column, the remaining bins take the per-cell select between the 5-term
// series and 1 - ex2 (kappa's smallest value need not follow the same order). A pair
// takes the class of its upper bin, which holds for the lower one too.
#include "rt_device.cuh"

namespace rt {
namespace {

struct TdepTab {
    const float2 *kt2;  // [nnu_pad][n_t] (kappa_j, kappa_{j+1}) of every sorted bin (global)
    const float *tg;    // [n_t] temperature grid (K)
    int n_t;
};

// Bins [i0, i1) of one class: scan, attenuation, absorption for the lane's cells,
// two cells per f32x2 register pair (packed FMA/ADD/MUL on the column, the exponent,
// the absorbed fraction and the accumulators; the two cells' kappa come from
// different table rows, so the interpolation itself stays scalar).
template <int CLASS, int C>
__device__ __forceinline__ void tdep_range(int i0, int i1, const float *s_lf, const float2 *s_kt, int n_t,
                                           const int (&jt)[C], const float (&wt)[C], const float (&wb)[C],
                                           const float2 (&d2)[C / 2],
                                           float2 (&a2)[C / 2], float2 (&a02)[C / 2], bool any_zero, int lane,
                                           float &esc)
{
    const float2 nl2e = f2(-(float)kLog2e);
    for (int i = i0; i < i1; ++i) {
        const float lf = s_lf[i];
        const float2 *row = s_kt + i * n_t;
        auto kappa2 = [&](int m) {  // the two cells' kappa of this bin
            // kappa_j (T_{j+1} - T) / dT + kappa_{j+1} (T - T_j) / dT: two non-negative
            // terms, no cancellation where the row falls towards zero
            const float2 k0 = row[jt[2 * m]], k1 = row[jt[2 * m + 1]];
            return make_float2(fmaf(k0.y, wt[2 * m], k0.x * wb[2 * m]), fmaf(k1.y, wt[2 * m + 1], k1.x * wb[2 * m + 1]));
        };
        float2 dt2[C / 2];
        float2 ls2 = f2(0.0f);  // the lane's sum, at most C terms in two halves (plain FP32)
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            dt2[m] = __fmul2_rn(kappa2(m), d2[m]);
            ls2 = __fadd2_rn(ls2, dt2[m]);
        }
        // compensated warp scan of the lane sums (the ray-long sum)
        KahanSum inc;
        inc.zero();
        inc.add(ls2.x + ls2.y);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const KahanSum v = inc.shfl_up(o);
            if (lane >= o) inc.add(v);
        }
        KahanSum pre = inc.shfl_up(1);
        if (lane == 0) pre.zero();
        if (lane == 31) esc += ex2_approx(fmaf(-(float)kLog2e, inc.value(), lf));
        // the lane's exclusive prefix: the warp offset (hi + lo) plus a plain partial sum
        const float2 bhi = f2(pre.hi), blo = f2(pre.lo), lf2 = f2(lf);
        float part = 0.0f;
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float2 p2 = make_float2(part, part + dt2[m].x);
            const float2 tau = __fadd2_rn(bhi, __fadd2_rn(blo, p2));
            const float2 g = ex2_approx2(__ffma2_rn(nl2e, tau, lf2));
            const float2 y = __fmul2_rn(nl2e, dt2[m]);  // -dtau log2(e)
            float2 om;                                   // 1 - 2^y
            if constexpr (CLASS <= 5) {
                om = taylor_fraction<CLASS>(y);
            } else {
                const float2 big = __ffma2_rn(ex2_approx2(y), f2(-1.0f), f2(1.0f));
                const float2 small = taylor_fraction<5>(y);
                om = make_float2(y.x > -kYSplit ? small.x : big.x, y.y > -kYSplit ? small.y : big.y);
            }
            a2[m] = __ffma2_rn(g, om, a2[m]);
            if (any_zero) a02[m] = __ffma2_rn(g, kappa2(m), a02[m]);  // (rare: re-read, not kept)
            part = p2.y + dt2[m].y;
        }
    }
}

// Bin pairs [p0, p1) of one class: scan, attenuation, absorption for the lane's cells,
// one cell per f32x2 register pair holding the pair's two bins (packed FMA/ADD/MUL on the
// opacity, the column, the exponent, the absorbed fraction). s_kt4[p n_t + j] =
// (kappa_2p(T_j), kappa_2p+1(T_j), kappa_2p(T_j+1), kappa_2p+1(T_j+1)).
template <int CLASS, int C>
__device__ __forceinline__ void tdep_pairs(int p0, int p1, const float *s_lf, const float4 *s_kt4, int n_t,
                                           const int (&jt)[C], const float (&wt)[C], const float (&wb)[C],
                                           const Cells<float, C> &dc, Cells<float, C> &ac, Cells<float, C> &ac0,
                                           bool any_zero, int lane, float &esc)
{
    const float2 nl2e = f2(-(float)kLog2e);
    for (int pp = p0; pp < p1; ++pp) {
        const float2 lf2 = make_float2(s_lf[2 * pp], s_lf[2 * pp + 1]);
        const float4 *row = s_kt4 + pp * n_t;
        auto kappa2 = [&](int j) {  // the pair's kappa in cell j
            // kappa_j (T_{j+1} - T) / dT + kappa_{j+1} (T - T_j) / dT: two non-negative
            // terms, no cancellation where the row falls towards zero
            const float4 k = row[jt[j]];
            return __ffma2_rn(make_float2(k.z, k.w), f2(wt[j]), __fmul2_rn(make_float2(k.x, k.y), f2(wb[j])));
        };
        float2 dt2[C];
        float2 ls2 = f2(0.0f);  // the lane's two sums, C terms each (plain FP32)
#pragma unroll
        for (int j = 0; j < C; ++j) {
            dt2[j] = __fmul2_rn(kappa2(j), f2(dc.get(j)));
            ls2 = __fadd2_rn(ls2, dt2[j]);
        }
        // compensated warp scan of both bins' lane sums (the ray-long sums): a Kahan pair
        // per bin, the two bins side by side
        float2 ih = ls2, il = f2(0.0f);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float2 vh = make_float2(__shfl_up_sync(0xffffffffu, ih.x, o), __shfl_up_sync(0xffffffffu, ih.y, o));
            const float2 vl = make_float2(__shfl_up_sync(0xffffffffu, il.x, o), __shfl_up_sync(0xffffffffu, il.y, o));
            if (lane >= o) {
                // two_sum(vh, ih) exactly, then the low parts
                const float2 sm = __fadd2_rn(vh, ih);
                const float2 bb = __fadd2_rn(sm, __fmul2_rn(vh, f2(-1.0f)));
                const float2 ea = __fadd2_rn(vh, __fmul2_rn(__fadd2_rn(sm, __fmul2_rn(bb, f2(-1.0f))), f2(-1.0f)));
                const float2 eb = __fadd2_rn(ih, __fmul2_rn(bb, f2(-1.0f)));
                il = __fadd2_rn(__fadd2_rn(il, vl), __fadd2_rn(ea, eb));
                ih = sm;
            }
        }
        // exclusive prefix: the inclusive one of the lane before
        float2 bhi = make_float2(__shfl_up_sync(0xffffffffu, ih.x, 1), __shfl_up_sync(0xffffffffu, ih.y, 1));
        float2 blo = make_float2(__shfl_up_sync(0xffffffffu, il.x, 1), __shfl_up_sync(0xffffffffu, il.y, 1));
        if (lane == 0) bhi = blo = f2(0.0f);
        if (lane == 31) {
            const float2 tot = __fadd2_rn(ih, il);
            const float2 ee = ex2_approx2(__ffma2_rn(nl2e, tot, lf2));
            esc += ee.x + ee.y;
        }
        // the lane's exclusive prefix: the warp offset (hi + lo) plus a plain partial sum
        float2 part = f2(0.0f);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float2 tau = __fadd2_rn(bhi, __fadd2_rn(blo, part));
            const float2 g = ex2_approx2(__ffma2_rn(nl2e, tau, lf2));
            const float2 y = __fmul2_rn(nl2e, dt2[j]);  // -dtau log2(e)
            float2 om;                                  // 1 - 2^y
            if constexpr (CLASS <= 5) {
                om = taylor_fraction<CLASS>(y);
            } else {
                const float2 big = __ffma2_rn(ex2_approx2(y), f2(-1.0f), f2(1.0f));
                const float2 small = taylor_fraction<5>(y);
                om = make_float2(y.x > -kYSplit ? small.x : big.x, y.y > -kYSplit ? small.y : big.y);
            }
            ac.set(j, fmaf(g.y, om.y, fmaf(g.x, om.x, ac.get(j))));
            if (any_zero) {  // (rare: the kappa read again, not kept)
                const float2 k2 = kappa2(j);
                ac0.set(j, fmaf(g.y, k2.y, fmaf(g.x, k2.x, ac0.get(j))));
            }
            part = __fadd2_rn(part, dt2[j]);
        }
    }
}

// PAIRS: the bins in pairs (tdep_pairs; 2C more registers for both bins' column
// increments), else one at a time (tdep_range), for the shapes whose register cap the
// pair form overflows
template <int C, int W, int MINB, bool PAIRS>
__global__ void __launch_bounds__(W * 32, MINB) k_ray_tdep(const TraceArgs p, const TdepTab t)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nr = p.nr;
    const int c0 = lane * C;
    const int nv = nr - c0 < 0 ? 0 : (nr - c0 > C ? C : nr - c0);

    __shared__ float s_dr[C][32], s_gq[C][32], s_ga[C][32];
    __shared__ float s_tg[32], s_idt[32];  // grid, 1 / (T_{j+1} - T_j)
    __shared__ KahanSum s_red[W][2];
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *s_nu = reinterpret_cast<float4 *>(smem);                 // [nnu_pad] (nk_max, ., lf, .)
    float *s_lf = reinterpret_cast<float *>(s_nu + p.nnu_pad);        // [nnu_pad]
    // [nnu_pad][n_t] rows of (kappa_j, kappa_j+1), or [nnu_pad / 2][n_t] bin-pair rows of
    // both bins' (kappa_j, kappa_j+1) (the same bytes); 16-byte aligned
    float4 *s_kt4 = reinterpret_cast<float4 *>((reinterpret_cast<size_t>(s_lf + p.nnu_pad) + 15) & ~size_t(15));
    float2 *s_kt = reinterpret_cast<float2 *>(s_kt4);

    for (int i = tid; i < p.nnu_pad; i += W * 32) {
        const NuEntry e = p.nu[i];
        s_nu[i] = make_float4(e.nk, e.nk, e.lf, e.lf);
        s_lf[i] = e.lf;
    }
    if constexpr (PAIRS) {
        for (int i = tid; i < (p.nnu_pad / 2) * t.n_t; i += W * 32) {
            const int pp = i / t.n_t, j = i - pp * t.n_t;
            const float2 a = t.kt2[2 * pp * t.n_t + j], b = t.kt2[(2 * pp + 1) * t.n_t + j];
            s_kt4[i] = make_float4(a.x, b.x, a.y, b.y);
        }
    } else {
        for (int i = tid; i < p.nnu_pad * t.n_t; i += W * 32) s_kt[i] = t.kt2[i];
    }
    for (int i = tid; i < t.n_t; i += W * 32) {
        s_tg[i] = t.tg[i];
        s_idt[i] = i + 1 < t.n_t ? 1.0f / (t.tg[i + 1] - t.tg[i]) : 0.0f;
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

    KahanSum eabs, eesc;
    eabs.zero();
    eesc.zero();
    for (unsigned ray = blockIdx.x * W + warp; ray < p.nrays; ray += gridDim.x * W) {
        const size_t base = (size_t)ray * nr + c0;
        Cells<float, C> d, acc, acc0;
        float wt[C], wb[C];  // the weights of the upper and the lower point
        int jt[C];
        unsigned zero_m = 0;
        bool bad = false;
        float dmax = 0.0f;
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
            d.set(j, dj);
            if (dust && dj == 0.0f) zero_m |= 1u << j;
            dmax = fmaxf(dmax, dj);
            acc.set(j, 0.0f);
            acc0.set(j, 0.0f);
            // bracketing temperature points and the weight of the upper one
            int lo = 0;
            for (int s = 16; s > 0; s >>= 1)
                if (lo + s < nt - 1 && s_tg[lo + s] <= td) lo += s;
            jt[j] = lo;
            wt[j] = fminf(fmaxf((td - s_tg[lo]) * s_idt[lo], 0.0f), 1.0f);
            wb[j] = fminf(fmaxf((s_tg[lo + 1] - td) * s_idt[lo], 0.0f), 1.0f);
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(p.bad_input, p.seq);
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        const bool any_zero = __any_sync(0xffffffffu, zero_m != 0u);

        const int na = p.n_active;
        const BinClasses bc = classify_bins(s_nu, na, lane, dmax, 0.0f);
        float esc = 0.0f;
        if constexpr (PAIRS) {
            // pair p (bins 2p, 2p + 1) belongs to the class of its upper bin: the pairs
            // below a class boundary b are those with 2p + 1 < b; a last odd bin pairs with
            // a padding bin (kappa 0, no flux: it adds nothing)
            const int q1 = bc.b1 / 2, q2 = max(bc.b2 / 2, q1), q3 = max(bc.b3 / 2, q2), q5 = max(bc.b5 / 2, q3);
            const int qn = (na + 1) / 2;
            tdep_pairs<1, C>(0, q1, s_lf, s_kt4, nt, jt, wt, wb, d, acc, acc0, any_zero, lane, esc);
            tdep_pairs<2, C>(q1, q2, s_lf, s_kt4, nt, jt, wt, wb, d, acc, acc0, any_zero, lane, esc);
            tdep_pairs<3, C>(q2, q3, s_lf, s_kt4, nt, jt, wt, wb, d, acc, acc0, any_zero, lane, esc);
            tdep_pairs<5, C>(q3, q5, s_lf, s_kt4, nt, jt, wt, wb, d, acc, acc0, any_zero, lane, esc);
            tdep_pairs<6, C>(q5, qn, s_lf, s_kt4, nt, jt, wt, wb, d, acc, acc0, any_zero, lane, esc);
        } else {
            tdep_range<1, C>(0, bc.b1, s_lf, s_kt, nt, jt, wt, wb, d.v, acc.v, acc0.v, any_zero, lane, esc);
            tdep_range<2, C>(bc.b1, bc.b2, s_lf, s_kt, nt, jt, wt, wb, d.v, acc.v, acc0.v, any_zero, lane, esc);
            tdep_range<3, C>(bc.b2, bc.b3, s_lf, s_kt, nt, jt, wt, wb, d.v, acc.v, acc0.v, any_zero, lane, esc);
            tdep_range<5, C>(bc.b3, bc.b5, s_lf, s_kt, nt, jt, wt, wb, d.v, acc.v, acc0.v, any_zero, lane, esc);
            tdep_range<6, C>(bc.b5, na, s_lf, s_kt, nt, jt, wt, wb, d.v, acc.v, acc0.v, any_zero, lane, esc);
        }

        const float w = __ldg(p.domega32 + ray);
        if (lane == 31) eesc.add(esc * w);
        float lane_abs = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const bool zc = (zero_m >> j) & 1u;
            const float aj = acc.get(j), dj = d.get(j);
            const float qv = zc ? 0.0f : s_gq[j][lane] * aj;
            const float av = s_ga[j][lane] * (zc ? acc0.get(j) : (dj > 0.0f ? __fdividef(aj, dj) : 0.0f));
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

// kt2[a][j] = (kappa[order[a]][j], kappa[order[a]][j + 1]) for the sorted active
// bins; padding bins get zero opacity
__global__ void k_build_tdep(int n_active, int nnu_pad, int n_t, const double *kappa_t, const int *order,
                             float2 *kt2)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nnu_pad * n_t) return;
    const int a = idx / n_t, j = idx % n_t;
    if (a >= n_active) {
        kt2[idx] = make_float2(0.0f, 0.0f);
        return;
    }
    const double *row = kappa_t + (size_t)order[a] * n_t;
    kt2[idx] = make_float2((float)row[j], (float)row[j + 1 < n_t ? j + 1 : j]);
}

template <int C, int W, int MINB, bool PAIRS>
cudaError_t launch_tdep_shape(const TraceArgs &a, const TdepTab &t, cudaStream_t stream, unsigned *grid_out)
{
    const size_t smem = (size_t)a.nnu_pad * (16 + 4) + 16 + (size_t)(a.nnu_pad / 2) * t.n_t * sizeof(float4);
    auto kern = k_ray_tdep<C, W, MINB, PAIRS>;
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

struct TdepEntry {
    int c, w, minb;
    cudaError_t (*fn)(const TraceArgs &, const TdepTab &, cudaStream_t, unsigned *);
};
// the bin-pair form where its registers fit the cap without more than a few bytes of spill
#define RT_TD(C, W, MB, PR) {C, W, MB, &launch_tdep_shape<C, W, MB, PR>}
const TdepEntry kTdepShapes[] = {RT_TD(2, 4, 8, true),  RT_TD(4, 4, 8, false),  RT_TD(4, 4, 6, true),
                                 RT_TD(8, 4, 6, false), RT_TD(8, 4, 4, true),   RT_TD(16, 4, 3, false),
                                 RT_TD(32, 4, 2, false)};
#undef RT_TD

}  // namespace

// The shapes whose rays fill the warp: the fewest cells per lane that hold nr
// (with each of its register caps); a wider one would leave lanes idle.
int tdep_shapes(int nr, Shape *out, int max_out)
{
    int c_fit = 0;
    for (const TdepEntry &s : kTdepShapes)
        if (32 * s.c >= nr && (c_fit == 0 || s.c < c_fit)) c_fit = s.c;
    int n = 0;
    for (const TdepEntry &s : kTdepShapes)
        if (s.c == c_fit && n < max_out) out[n++] = Shape{kKindRay, s.c, s.w, s.minb};
    return n;
}

cudaError_t launch_tdep(Shape s, const TraceArgs &args, const float2 *kt2, const float *tg, int n_t,
                        cudaStream_t stream, unsigned *grid_out)
{
    const TdepTab t{kt2, tg, n_t};
    for (const TdepEntry &e : kTdepShapes)
        if (e.c == s.cells_per_lane && e.w == s.warps && (s.min_blocks == 0 || e.minb == s.min_blocks) &&
            32 * e.c >= args.nr)
            return e.fn(args, t, stream, grid_out);
    return cudaErrorInvalidValue;
}

cudaError_t launch_build_tdep(int n_active, int nnu_pad, int n_t, const double *kappa_t, const int *order,
                              float2 *kt2, cudaStream_t stream)
{
    const int n = nnu_pad * n_t;
    k_build_tdep<<<(n + 255) / 256, 256, 0, stream>>>(n_active, nnu_pad, n_t, kappa_t, order, kt2);
    return cudaGetLastError();
}

}  // namespace rt
