// The warp-per-ray body of the frequency-dependent tracer (Kuiper et al. 2010,
// Sect. 2.2-2.3, 3.3.4), shared by the single-grid kernel (rt_ray.cu) and the
// multi-grid batch (rt_batch.cu).
//
// A segment of G lanes traces one radial ray (a warp holds 32 / G rays at a time,
// so rays shorter than 32 C cells keep every lane busy), or P = 2 warps of a CTA
// trace one ray together (64 C cells: fewer cells per lane, fewer registers, more
// warps per SM); lane l of a segment owns the cells [l C, (l+1) C) of its ray, so the radial constants of a lane never
// change and the ray's fields are read straight from HBM in 16-byte vectors (no
// staging, no block barrier in the ray loop). While it traces one warp-slot, the
// warp asks L2 for the fields of its next one (a bulk prefetch: nothing to wait
// for). Per ray:
//   - dN = [T <= t_sub] rho dr per cell, and its exclusive prefix along the ray
//     (Eq. 19, tau = 0 at the inner radius) in one compensated pass: each lane keeps
//     the column u from its own first cell, and a compensated warp scan of the lane
//     sums gives the column N0 in front of the lane, so N_in = N0 + u;
//   - every exponent is taken about the lane's N0: e^{-kappa N_in} =
//     e^{-kappa N0} e^{-kappa u};
//   - the bins optically thin along all the warp's rays (one power series in the
//     column for the lot, whose rows the set-up builds) and the bins thin within
//     every lane's own cells (expanded about N0 per lane) are summed as one series
//     in u per lane (lane_series); the others go bin by bin (rt_device.cuh: Eqs.
//     17, 20, 31-32) with the warp's bin classes from its largest and smallest
//     column; all into one accumulator per cell;
//   - escaping power sum_i F_i/F_max e^{-kappa_i N_total} (Eqs. 33-35), the lanes
//     sharing the bins outside the thin series (that part from the series row);
//   - q_abs = Gq acc and a_rad = q/(rho c) = Ga0 acc / dN (Sect. 5; the rho -> 0
//     limit where dN = 0 with dust), stored as 16-byte vectors;
//   - energy sums per lane.
// Chunked form (MC): a segment of G lanes holds G C cells of its ray at a time and
// walks the ray outward chunk by chunk, the column in front of the chunk carried
// (compensated) from one chunk to the next. Every per-warp decision (thin series,
// tier, bin classes) is then taken over the cells of one chunk of R neighbouring
// rays, a narrow range of radii, and the bins whose attenuation underflows in every
// cell of the chunk (kappa_i N_in >= 127 / log2 e at the smallest N_in of the warp:
// 2^{-127} and below flush to zero) are skipped, which changes no bit of the result.
#pragma once

#include "rt_device.cuh"

namespace rt {
namespace {

// Radial constants of every lane's cells, stored [j / 2][lane] as pairs of
// consecutive cells (lane l's cell j is radial index (l mod G) C + j), so that the
// lanes of a warp read consecutive words and every read yields the packed pair the
// f32x2 arithmetic works on: dr as (dr_j, dr_j+1), (Gq_j, Gq_j+1, Ga0_j, Ga0_j+1).
template <int C, int P = 1>
struct RayShared {
    float2 dr[P][C / 2][32];
    float4 gqa[P][C / 2][32];
};

// dynamic shared memory of the bin tables: kappa, (nk, nk, lf, lf) and the series
// moments' constants (two float4 per bin)
__host__ __device__ constexpr size_t ray_bin_smem(int nnu_pad) { return (size_t)nnu_pad * (4 + 16 + 32); }
// chunked form: the pairs of radial constants of all chunks (chunks x C/2 x G)
__host__ __device__ constexpr int ray_chunk_pairs(int c, int g, int nr) { return (nr + g * c - 1) / (g * c) * (c / 2) * g; }

// The tables of grid p for G lanes per ray, or P warps per ray (call from every
// thread of the CTA, then __syncthreads()).
template <int C, int W, int P = 1>
__device__ __forceinline__ void ray_tables(const TraceArgs &p, int G, RayShared<C, P> &rs, float *s_kap,
                                           float4 *s_nu, float4 *s_mom)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < p.nnu_pad; i += W * 32) {
        s_kap[i] = p.kap[i];
        const NuEntry e = p.nu[i];
        s_nu[i] = make_float4(e.nk, e.nk, e.lf, e.lf);
        fill_moments(s_mom, i, e.nk);
    }
    for (int i = tid; i < P * 16 * C; i += W * 32) {
        const int h = i / (16 * C), l = (i / (C / 2)) % 32, m = i % (C / 2);
        const int k = (P > 1 ? h * 32 + l : l % G) * C + 2 * m;
        const float4 g0 = (k < p.nr) ? __ldg(&p.rtab[k]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float4 g1 = (k + 1 < p.nr) ? __ldg(&p.rtab[k + 1]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        rs.dr[h][m][l] = make_float2(g0.x, g1.x);
        rs.gqa[h][m][l] = make_float4(g0.y, g1.y, g0.z, g1.z);
    }
}

// the hardware log2 (absolute error near 2^-22)
__device__ __forceinline__ float ex_lg2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Ask L2 for `bytes` bytes from p (16-byte aligned, a multiple of 16): a hint with
// no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// One lane's series in v = s2 u: Q(v) = sum_{k=1..K} F_k v^k. A cell with column u
// in front of it (from the lane's first cell) and dN in it absorbs
// Q(s2 (u + dN)) - Q(s2 u) = s2 dN sum_k F_k h_{k-1}(a, c), a = s2 (u + dN), c = s2 u,
// evaluated by the paired Horner recurrence of thin_series (no a - c cancellation).
template <int C>
__device__ __forceinline__ void lane_series(const float (&F)[kThinTerms + 1], float s2, const float2 (&u2)[C / 2],
                                            const float2 (&d2)[C / 2], float2 (&a2)[C / 2])
{
    const float2 s22 = f2(s2);
    float2 Fk[kThinTerms + 1];
#pragma unroll
    for (int k = 1; k <= kThinTerms; ++k) Fk[k] = f2(F[k]);
#pragma unroll
    for (int m = 0; m < C / 2; ++m) {
        const float2 cc = __fmul2_rn(s22, u2[m]);
        const float2 aa = __ffma2_rn(s22, d2[m], cc);
        float2 dd = Fk[kThinTerms];
        float2 pc = __ffma2_rn(dd, cc, Fk[kThinTerms - 1]);
#pragma unroll
        for (int k = kThinTerms - 2; k >= 1; --k) {
            dd = __ffma2_rn(dd, aa, pc);
            pc = __ffma2_rn(pc, cc, Fk[k]);
        }
        dd = __ffma2_rn(dd, aa, pc);
        a2[m] = __ffma2_rn(__fmul2_rn(d2[m], dd), s22, a2[m]);
    }
}

// The coefficients F_1..F_K of a lane's series (lane_series) and its scale s2:
//   - the bins i < bt, thin along all the warp's rays: their set-up row holds
//     P(x) = sum_k C_k x^k with x = s N (s = kappa_{bt-1}), so that a cell absorbs
//     P(s N_out) - P(s N_in). Shifted to the lane's column N0 (Taylor shift,
//     synthetic division: E_k = P^(k)(x0) / k!, x0 = s N0 <= kThinX) and rescaled to
//     v = s2 u: F_k += E_k (s / s2)^k.
//   - the bins bt <= i < bt2, thin within every lane's own cells (kappa_i u <=
//     kThinX for every u of the lane): expanded about N0,
//     sum_i g_i (1 - e^{-kappa_i u}) = sum_k T_k v^k, g_i = F_i/F_max e^{-kappa_i N0},
//     T_k = (-1)^{k+1} / k! sum_i g_i (kappa_i / s2)^k, s2 = kappa_{bt2-1}.
// Every power sum of the tier has one sign (no cancellation); the shifted row
// alternates with |x0| <= kThinX (precision loss below e^{2 kThinX}). Both parts
// are truncated after K terms with |v| <= kThinX: the first omitted term is below
// kThinX^K / K! of the leading one.
__device__ __forceinline__ float lane_coefficients(const float *thin_row, int bt, int bt2, const float4 *s_nu,
                                                   float n0, float (&F)[kThinTerms + 1])
{
    constexpr int K = kThinTerms;
#pragma unroll
    for (int k = 0; k <= K; ++k) F[k] = 0.0f;
    // s2 in the units of -nk (the ratio of two bins' nk is the ratio of their kappa);
    // without tier bins the row's own s
    const float nks2 = s_nu[bt2 - 1].x;
    const float s2 = (bt2 > bt || bt == 0) ? -nks2 * (float)kLn2 : __ldg(thin_row);
    if (bt > 0) {
        const float s = __ldg(thin_row);
        float c[K + 1];
        c[0] = 0.0f;
#pragma unroll
        for (int k = 1; k <= K; ++k) c[k] = __ldg(thin_row + k);
        const float x0 = s * n0;
#pragma unroll
        for (int i = 0; i < K; ++i)
#pragma unroll
            for (int j = K - 1; j >= (i > 1 ? i : 1); --j) c[j] = fmaf(x0, c[j + 1], c[j]);
        if (bt2 > bt) {
            const float rho = s / s2;
            float pk = rho;
#pragma unroll
            for (int k = 1; k <= K; ++k) {
                F[k] = c[k] * pk;
                pk *= rho;
            }
        } else {
#pragma unroll
            for (int k = 1; k <= K; ++k) F[k] = c[k];
        }
    }
    if (bt2 > bt) {
        const float inv = 1.0f / nks2;
        float2 m[K + 1];
#pragma unroll
        for (int k = 1; k <= K; ++k) m[k] = f2(0.0f);
        const float2 n02 = f2(n0);
        for (int i = bt; i < bt2; i += 2) {  // warp-uniform; bins in pairs
            const float4 e0 = s_nu[i];
            const float4 e1 = s_nu[i + 1 < bt2 ? i + 1 : i];
            const float2 nk = make_float2(e0.x, e1.x);
            float2 g = ex2_approx2(__ffma2_rn(nk, n02, make_float2(e0.z, e1.z)));
            if (i + 1 >= bt2) g.y = 0.0f;
            const float2 r = __fmul2_rn(nk, f2(inv));
            float2 pw = g;
#pragma unroll
            for (int k = 1; k <= K; ++k) {
                pw = __fmul2_rn(pw, r);
                m[k] = __fadd2_rn(m[k], pw);
            }
        }
#pragma unroll
        for (int k = 1; k <= K; ++k) {
            const float t = (m[k].x + m[k].y) * (float)inv_factorial(k);
            F[k] += (k & 1) ? t : -t;
        }
    }
    return s2;
}

// Column weight b(T) of a separable kappa(nu, T) table (TraceArgs::tw_t, tw_b): T
// clamped to the grid, its interval found by a five-step binary search over the
// 32-entry grid (padded with +Inf), then linear in T as
// (b_j (T_{j+1} - T) + b_{j+1} (T - T_j)) / dT: two non-negative terms, so no
// cancellation where b falls towards zero. t_lo, t_hi: the grid's ends.
__device__ __forceinline__ float tw_weight(const float *tg, const float4 *tb, float t_lo, float t_hi, float t)
{
    t = fminf(fmaxf(t, t_lo), t_hi);
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (tg[j + step] <= t) j += step;
    const float4 e = tb[j];
    return fmaf(e.z, e.y - t, e.w * (t - e.x));
}

// Bar.sync on a named barrier of n threads (the P warps of one group).
__device__ __forceinline__ void group_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Bins (sorted by kappa) whose attenuation over a column n stays at or above 2^-127:
// (-nk_i) n <= 127, a prefix of the sorted bins (warp-uniform count).
__device__ __forceinline__ int live_count(const float4 *s_nu, int n_active, int lane, float n)
{
    n = fmaxf(n, 0.0f);  // as in thin_count: padding lanes (ak = inf) never count
    int b = 0;
    for (int c0 = 0; c0 < n_active; c0 += 32) {
        const int i = c0 + lane;
        const float ak = (i < n_active) ? -s_nu[i].x : INFINITY;
        b += __popc(__ballot_sync(0xffffffffu, ak * n <= 127.0f));
    }
    return b;
}

// The radial constants of every chunk for the chunked form (G lanes of C cells per
// chunk): s_dr[(ch C/2 + m) G + l] = (dr, dr) of cells (ch G + l) C + 2m, +1, and
// s_gqa the (Gq, Gq, Ga0, Ga0) pairs. Call from every thread of the CTA, then
// __syncthreads().
template <int C, int W, int G>
__device__ __forceinline__ void ray_tables_mc(const TraceArgs &p, float2 *s_dr, float4 *s_gqa)
{
    const int nch = (p.nr + G * C - 1) / (G * C);
    for (int i = threadIdx.x; i < nch * (C / 2) * G; i += W * 32) {
        const int l = i % G, m = (i / G) % (C / 2), ch = i / (G * (C / 2));
        const int k = (ch * G + l) * C + 2 * m;
        const float4 g0 = (k < p.nr) ? __ldg(&p.rtab[k]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float4 g1 = (k + 1 < p.nr) ? __ldg(&p.rtab[k + 1]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        s_dr[i] = make_float2(g0.x, g1.x);
        s_gqa[i] = make_float4(g0.y, g1.y, g0.z, g1.z);
    }
}

// Warp-slots wr = wr_begin, wr_begin + step, ... (< wr_end) of grid p, R = 32 / G rays
// each (or, with P > 1, one ray per group of P consecutive warps, which all walk the
// same slots); the lanes' energy sums are added to eabs / eesc. TW: the table is a
// separable kappa(nu, T) (TraceArgs::n_tw > 0) and each cell's column carries the
// weight b(T). LUT: the absorbed power of the cells comes from the lookup table of
// TraceArgs::lut (the per-bin sum only in warp-slots that hold a flagged cell).
// MC: the chunked form; s_dr_mc / s_gqa_mc hold the radial constants of every chunk,
// [chunk][j / 2][lane in the segment] (ray_tables_mc).
template <int C, int W, int MODE, int G, int P = 1, bool TW = false, bool LUT = false, bool MC = false>
__device__ __forceinline__ void ray_slots(const TraceArgs &p, unsigned wr_begin, unsigned wr_end, unsigned step,
                                          const RayShared<C, P> &rs, const float *s_kap, const float4 *s_nu,
                                          const float4 *s_mom, KahanSum &eabs, KahanSum &eesc,
                                          const float2 *s_dr_mc = nullptr, const float4 *s_gqa_mc = nullptr)
{
    static_assert(MODE != RT_FP64, "the FP64 mode uses the tile kernel");
    static_assert(!MC || (P == 1 && !TW && !LUT), "chunks: one warp per segment, the plain table");
    static_assert(C % 2 == 0, "cells per lane must be even");
    static_assert(G == 8 || G == 16 || G == 32, "lanes per ray");
    static_assert(P == 1 || (G == 32 && W % P == 0 && P == 2), "warps per ray");
    using Sum = ColSum<MODE>;
    constexpr int V = (C % 4 == 0) ? 4 : 2;  // vector width of the field loads
    constexpr int R = 32 / G;                // rays per warp

    const int lane = threadIdx.x & 31;
    const int half = P > 1 ? (int)(threadIdx.x >> 5) % P : 0;  // warp within its group
    const int group = (int)(threadIdx.x >> 5) / P;
    // lane totals of the group's warps, double buffered by slot parity
    __shared__ Sum s_grp[P > 1 ? W / P : 1][2][P];
    // separable table: each warp's copy of the weight table, and its cells' weights
    __shared__ float s_twt[TW ? W : 1][kMaxTdepPoints];
    __shared__ float4 s_twb[TW ? W : 1][kMaxTdepPoints];
    __shared__ float2 s_bw[TW ? W : 1][C / 2][32];
    const int wid = TW ? (int)(threadIdx.x >> 5) : 0;
    float tw_lo = 0.0f, tw_hi = 0.0f;
    if constexpr (TW) {
        s_twt[wid][lane] = __ldg(p.tw_t + lane);
        s_twb[wid][lane] = __ldg(p.tw_b + lane);
        tw_lo = __ldg(p.tw_t);
        tw_hi = __ldg(p.tw_t + p.n_tw - 1);
        __syncwarp();
    }
    const int seg = lane / G, ll = half * 32 + lane % G;  // ray slot of the lane, lane within the ray
    const int nr = p.nr;
    const int nch = MC ? (nr + G * C - 1) / (G * C) : 1;  // chunks per ray
    // vector access needs every lane start and the field bases 4V-byte aligned
    const bool vec = (nr % V == 0) &&
                     ((reinterpret_cast<size_t>(p.rho) | reinterpret_cast<size_t>(p.tdust) |
                       reinterpret_cast<size_t>(p.q) | reinterpret_cast<size_t>(p.a)) % (4 * V) == 0);
    // a warp-slot's fields are R consecutive rays: one contiguous run per field
    const bool pf = (nr % 4 == 0) &&
                    ((reinterpret_cast<size_t>(p.rho) | reinterpret_cast<size_t>(p.tdust)) % 16 == 0);
    const int na = p.n_active;
    const float2 tiny2 = f2(FLT_MIN);

    for (unsigned wr = wr_begin; wr < wr_end; wr += step) {
        const unsigned ray = wr * R + seg;
        const bool live = ray < p.nrays;  // the last warp may hold fewer than R rays
        const float w = live ? __ldg(p.domega32 + ray) : 0.0f;
        Sum carry;  // chunked form: the ray's column in front of the chunk
        carry.zero();
        for (int ch = 0; ch < nch; ++ch) {
        const int c0 = (ch * G + ll) * C;  // the lane's first cell in the ray
        const int nv = !live ? 0 : (nr - c0 < 0 ? 0 : (nr - c0 > C ? C : nr - c0));  // its valid cells
        const size_t base = (size_t)(live ? ray : 0u) * nr + c0;

        // the fields, straight from HBM (or from L2, where the prefetch got there first)
        float2 rho2[C / 2], td2[C / 2];
        if (vec && nv == C) {
#pragma unroll
            for (int j = 0; j < C; j += V) {
                if constexpr (V == 4) {
                    const float4 r4 = __ldg(reinterpret_cast<const float4 *>(p.rho + base + j));
                    const float4 t4 = __ldg(reinterpret_cast<const float4 *>(p.tdust + base + j));
                    rho2[j / 2] = make_float2(r4.x, r4.y);
                    rho2[j / 2 + 1] = make_float2(r4.z, r4.w);
                    td2[j / 2] = make_float2(t4.x, t4.y);
                    td2[j / 2 + 1] = make_float2(t4.z, t4.w);
                } else {
                    rho2[j / 2] = __ldg(reinterpret_cast<const float2 *>(p.rho + base + j));
                    td2[j / 2] = __ldg(reinterpret_cast<const float2 *>(p.tdust + base + j));
                }
            }
        } else {
            // cells past the ray's end: no density, no dust (their column is 0 with any t_sub)
#pragma unroll
            for (int j = 0; j < C; j += 2) {
                rho2[j / 2] = make_float2(j < nv ? __ldg(p.rho + base + j) : 0.0f,
                                          j + 1 < nv ? __ldg(p.rho + base + j + 1) : 0.0f);
                td2[j / 2] = make_float2(j < nv ? __ldg(p.tdust + base + j) : INFINITY,
                                         j + 1 < nv ? __ldg(p.tdust + base + j + 1) : INFINITY);
            }
        }
        // the fields of this warp's next slot, on their way to L2 (with P > 1 the group's
        // first warp asks for the whole ray); in the chunked form each segment's first
        // lane asks for its ray's next chunk (the first chunk of its next ray after the
        // last), the same distance ahead as one slot of the one-chunk form
        if constexpr (MC) {
            if (pf && lane % G == 0) {
                const bool last = ch + 1 == nch;
                const unsigned rn = last ? (wr + step) * R + seg : ray;
                const int k0 = last ? 0 : (ch + 1) * G * C;
                if ((!last || wr + step < wr_end) && rn < p.nrays) {
                    const unsigned bytes = (unsigned)min(G * C, nr - k0) * 4u;
                    prefetch_l2(p.rho + (size_t)rn * nr + k0, bytes);
                    prefetch_l2(p.tdust + (size_t)rn * nr + k0, bytes);
                }
            }
        } else if (pf && lane == 0 && half == 0 && wr + step < wr_end) {
            const unsigned r0 = (wr + step) * R;
            if (r0 < p.nrays) {
                const unsigned nrs = p.nrays - r0 < (unsigned)R ? p.nrays - r0 : (unsigned)R;
                const unsigned bytes = nrs * (unsigned)nr * 4u;
                prefetch_l2(p.rho + (size_t)r0 * nr, bytes);
                prefetch_l2(p.tdust + (size_t)r0 * nr, bytes);
            }
        }

        // column density of the dust in each cell, its compensated prefix u from the
        // lane's first cell, and the invalid-input and no-column flags
        // (a cell without dust gets the column -0, one with dust but no density +0: the
        // sign tells the two apart where the force needs it, and -0 adds nothing)
        float2 D[C / 2], U[C / 2], acc[C / 2];
        unsigned rho_bits = 0u, d_min = 0xffffffffu;
        float td_max = 0.0f;  // NaN as soon as one t_dust is NaN
        Sum lsum;
        lsum.zero();
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float2 dr = MC ? s_dr_mc[(ch * (C / 2) + m) * G + ll] : rs.dr[half][m][lane];
            const bool d0 = td2[m].x <= p.t_sub, d1 = td2[m].y <= p.t_sub;
            // rho must be finite and >= 0 (-0 counts as 0): the bits of rho + 0 stay
            // below those of +Inf; t_dust must not be NaN
            const float2 rz = __fadd2_rn(rho2[m], f2(0.0f));
            rho_bits = max(rho_bits, max(__float_as_uint(rz.x), __float_as_uint(rz.y)));
            td_max = max_nan(td_max, max_nan(td2[m].x, td2[m].y));
            float2 mw = make_float2(d0 ? dr.x : -0.0f, d1 ? dr.y : -0.0f);
            if constexpr (TW) {
                // kappa_i(T) = kappa_i b(T): the weight enters the column (0 without dust)
                const float2 bw = make_float2(d0 ? tw_weight(s_twt[wid], s_twb[wid], tw_lo, tw_hi, td2[m].x) : 0.0f,
                                              d1 ? tw_weight(s_twt[wid], s_twb[wid], tw_lo, tw_hi, td2[m].y) : 0.0f);
                s_bw[wid][m][lane] = bw;
                mw = make_float2(d0 ? mw.x * bw.x : -0.0f, d1 ? mw.y * bw.y : -0.0f);
            }
            D[m] = __fmul2_rn(rz, mw);
            // +0 (dust, no column) has the smallest bits of all columns a valid input gives
            d_min = min(d_min, min(__float_as_uint(D[m].x), __float_as_uint(D[m].y)));
            acc[m] = f2(0.0f);
            U[m].x = lsum.value();
            lsum.add(D[m].x);
            U[m].y = lsum.value();
            lsum.add(D[m].y);
        }
        const bool zc = d_min == 0u;
        if (__any_sync(0xffffffffu, rho_bits >= 0x7f800000u || td_max != td_max) && lane == 0)
            atomicMax(p.bad_input, p.seq);

        // column in front of each lane: compensated scan of the lane sums within the segment
        Sum inc = lsum;
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const Sum o = inc.shfl_up(d, G);
            if ((ll % G) >= d) inc.add(o);
        }
        Sum pre = inc.shfl_up(1, G);
        if ((ll % G) == 0) pre.zero();
        float n0, ntot;
        if constexpr (P > 1) {
            // the group's warps exchange their totals: the warps before this one give its
            // offset, all of them the ray's total
            const int par = (int)(((wr - wr_begin) / step) & 1u);
            Sum wt;
            wt.hi = __shfl_sync(0xffffffffu, inc.hi, 31);
            if constexpr (MODE == RT_FP32_KAHAN) wt.lo = __shfl_sync(0xffffffffu, inc.lo, 31);
            if (lane == 0) s_grp[group][par][half] = wt;
            group_sync(1 + group, 32 * P);
            Sum off, tot;
            off.zero();
            tot.zero();
#pragma unroll
            for (int h = 0; h < P; ++h) {
                const Sum t = s_grp[group][par][h];
                if (h < half) off.add(t);
                tot.add(t);
            }
            off.add(pre);
            n0 = off.value();
            ntot = tot.value();
        } else if constexpr (MC) {
            // the chunk's offset: the carried column plus the segment's exclusive prefix;
            // then the carry moves past the chunk (ntot: the column at its end)
            Sum off = carry;
            off.add(pre);
            n0 = off.value();
            Sum st;
            st.hi = __shfl_sync(0xffffffffu, inc.hi, G - 1, G);
            if constexpr (MODE == RT_FP32_KAHAN) st.lo = __shfl_sync(0xffffffffu, inc.lo, G - 1, G);
            carry.add(st);
            ntot = carry.value();
        } else {
            n0 = pre.value();
            ntot = __shfl_sync(0xffffffffu, inc.value(), G - 1, G);
        }

        // bins thin along all the warp's rays (bt of them) and, after those, bins thin
        // within every lane's cells (up to bt2): one series per lane; the rest bin by bin
        float nmax = ntot;
        for (int o = G; o < 32; o <<= 1) nmax = fmaxf(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        float cmax = lsum.value();
        for (int o = 16; o > 0; o >>= 1) cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        int bt, bc;
        thin_counts(s_nu, na, lane, nmax, cmax, bt, bc);
        // chunked form: the bins from na_live on underflow in every cell of the chunk
        // (e^{-kappa N_in} <= 2^{-127} at the warp's smallest column in front of a lane)
        int na_live = na;
        if constexpr (MC) {
            float n0min = n0;
            for (int o = 16; o > 0; o >>= 1) n0min = fminf(n0min, __shfl_xor_sync(0xffffffffu, n0min, o));
            na_live = live_count(s_nu, na, lane, n0min);
        }
        // with no row to shift, a few tier bins do not pay for the series
        const int bt2 = (bc > bt && (bt > 0 || bc >= 4)) ? bc : bt;
        const float *thin_row = p.kap + kKapTable + bt * kThinStride;
        bool per_bin = true;
        if constexpr (LUT) {
            // acc = G kappa_ref dN with log2 G bilinear in (s, d); per_bin where a cell's
            // square is flagged or the cell lies off the table (warp-uniform)
            bool flagged = false;
            const float kr = p.lut_kref;
#pragma unroll
            for (int m = 0; m < C / 2; ++m) {
                float g2[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float dn = h ? D[m].y : D[m].x, uu = h ? U[m].y : U[m].x;
                    const float fs = (ex_lg2(fmaf(kr, n0 + uu, 0x1p-20f)) - kLutS0) * kLutInvH;
                    const float fd = (ex_lg2(fmaf(kr, dn, 0x1p-30f)) - kLutD0) * kLutInvH;
                    flagged |= !(fs >= 0.0f && fs < (float)(kLutNs - 1) && fd >= 0.0f && fd < (float)(kLutNd - 1));
                    // clamped into the table (NaN to 0), so every read stays inside it
                    const float fsc = fminf(fmaxf(fs, 0.0f), (float)(kLutNs - 1));
                    const float fdc = fminf(fmaxf(fd, 0.0f), (float)(kLutNd - 1));
                    const int i = min((int)fsc, kLutNs - 2), j = min((int)fdc, kLutNd - 2);
                    const float ts = fsc - (float)i, tdd = fdc - (float)j;
                    // (s_i, s_{i+1}) at d_j and at d_{j+1}: two 8-byte reads, s the fast index
                    const float2 *row = p.lut + (size_t)j * kLutNs + i;
                    const float2 a = __ldg(row), b = __ldg(row + kLutNs);
                    flagged |= (__float_as_uint(a.x) & 1u) != 0u;
                    const float v0 = fmaf(tdd, b.x - a.x, a.x), v1 = fmaf(tdd, b.y - a.y, a.y);
                    g2[h] = ex2_approx(fmaf(ts, v1 - v0, v0));
                }
                acc[m] = __fmul2_rn(__fmul2_rn(make_float2(g2[0], g2[1]), f2(kr)), D[m]);
            }
            per_bin = __any_sync(0xffffffffu, flagged);
            if (per_bin) {
                if (lane == 0 && p.lut_fallback) atomicAdd(p.lut_fallback, 1u);
#pragma unroll
                for (int m = 0; m < C / 2; ++m) acc[m] = f2(0.0f);
            }
        }
        if (per_bin && bt2 > 0) {
            float F[kThinTerms + 1];
            const float s2 = lane_coefficients(thin_row, bt, bt2, s_nu, n0, F);
            lane_series<C>(F, s2, U, D, acc);
        }
        if (per_bin && bt2 < na_live) {  // warp-uniform
            // the warp's largest and smallest non-zero column decide each bin's class
            float dmax = 0.0f, dmin = INFINITY;
#pragma unroll
            for (int m = 0; m < C / 2; ++m) {
                dmax = fmaxf(dmax, fmaxf(D[m].x, D[m].y));
                dmin = fminf(dmin, fminf(D[m].x > 0.0f ? D[m].x : INFINITY, D[m].y > 0.0f ? D[m].y : INFINITY));
            }
            for (int o = 16; o > 0; o >>= 1) {
                dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
                dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
            }
            const BinClasses bc = classify_bins(s_nu, na_live, lane, dmax, dmin, bt2);
            const int t1 = max(bc.b1, bt2), t2 = max(bc.b2, bt2), t3 = max(bc.b3, bt2), t5 = max(bc.b5, bt2);
            const int tb = max(bc.bb, bt2);
            moment_range<1, C>(bt2, t1, s_nu, s_mom, n0, U, D, acc);
            moment_range<2, C>(t1, t2, s_nu, s_mom, n0, U, D, acc);
            bin_range<3, C>(t2, t3, s_nu, n0, U, D, acc);
            bin_range<5, C>(t3, t5, s_nu, n0, U, D, acc);
            bin_range<6, C>(t5, tb, s_nu, n0, U, D, acc);
            bin_range<7, C>(tb, na_live, s_nu, n0, U, D, acc);
        }

        // escaping power of the ray, the lanes of its segment (all P warps of a group)
        // sharing the bins (chunked form: after its last chunk)
        if (!MC || ch == nch - 1) {
            float s = 0.0f;
            for (int i = bt + ll; i < na; i += G * P) s += ex2_approx(fmaf(s_nu[i].x, ntot, s_nu[i].z));
            for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if ((ll % G) == 0) {
                if (bt > 0 && half == 0) s += thin_escape(thin_row, ntot);
                eesc.add(s * w);
            }
        }

        // outputs and the lane's absorbed power: q = Gq acc, a = Ga0 acc / dN (a cell
        // with no column, past the ray or without dust or density, absorbed 0)
        float2 lane_abs2 = f2(0.0f);
        float2 qv[C / 2];
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float4 g = MC ? s_gqa_mc[(ch * (C / 2) + m) * G + ll] : rs.gqa[half][m][lane];
            qv[m] = __fmul2_rn(make_float2(g.x, g.y), acc[m]);
            lane_abs2 = __fadd2_rn(lane_abs2, acc[m]);
            const float2 dd = make_float2(fmaxf(D[m].x, tiny2.x), fmaxf(D[m].y, tiny2.y));
            acc[m] = __fmul2_rn(make_float2(g.z, g.w), __fmul2_rn(acc[m], make_float2(rcp_approx(dd.x), rcp_approx(dd.y))));
            if constexpr (TW) acc[m] = __fmul2_rn(acc[m], s_bw[wid][m][lane]);  // per mass: dN b / (rho dr)
        }
        // cells with dust but no column: the rho -> 0 force limit Ga0 sum_i kappa_i g_i
        if (__any_sync(0xffffffffu, zc)) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const float dj = (j & 1) ? D[j / 2].y : D[j / 2].x;
                const bool zj = zc && __float_as_uint(dj) == 0u;
                if (__any_sync(0xffffffffu, zj)) {
                    const float uj = (j & 1) ? U[j / 2].y : U[j / 2].x;
                    float s = 0.0f;
                    for (int i = 0; i < na; ++i)
                        s = fmaf(s_kap[i], ex2_approx(fmaf(s_nu[i].x, uj, fmaf(s_nu[i].x, n0, s_nu[i].z))), s);
                    if (zj) {
                        const float4 g = MC ? s_gqa_mc[(ch * (C / 2) + j / 2) * G + ll] : rs.gqa[half][j / 2][lane];
                        if constexpr (TW) {  // kappa_i(T) = kappa_i b(T)
                            const float2 bw = s_bw[wid][j / 2][lane];
                            s *= (j & 1) ? bw.y : bw.x;
                        }
                        if (j & 1) acc[j / 2].y = g.w * s;
                        else acc[j / 2].x = g.z * s;
                    }
                }
            }
        }
        eabs.add((lane_abs2.x + lane_abs2.y) * w);
        if (vec && nv == C) {
#pragma unroll
            for (int j = 0; j < C; j += V) {
                if constexpr (V == 4) {
                    *reinterpret_cast<float4 *>(p.q + base + j) =
                        make_float4(qv[j / 2].x, qv[j / 2].y, qv[j / 2 + 1].x, qv[j / 2 + 1].y);
                    *reinterpret_cast<float4 *>(p.a + base + j) =
                        make_float4(acc[j / 2].x, acc[j / 2].y, acc[j / 2 + 1].x, acc[j / 2 + 1].y);
                } else {
                    *reinterpret_cast<float2 *>(p.q + base + j) = qv[j / 2];
                    *reinterpret_cast<float2 *>(p.a + base + j) = acc[j / 2];
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (j < nv) {
                    p.q[base + j] = (j & 1) ? qv[j / 2].y : qv[j / 2].x;
                    p.a[base + j] = (j & 1) ? acc[j / 2].y : acc[j / 2].x;
                }
            }
        }
        }  // chunks
    }
}


// The kernel over all rays of one grid (persistent CTAs striding over the warp-slots),
// then the CTA's energy partial.
template <int C, int W, int MODE, int MINB, int G, int P, bool TW, bool LUT, bool MC>
__global__ void __launch_bounds__(W * 32, MINB) k_ray(const TraceArgs p)
{
    using ESum = KahanSum;
    constexpr int R = 32 / G;  // rays per warp
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ RayShared<C, P> rs;
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_kap = reinterpret_cast<float *>(smem);
    float4 *s_nu = reinterpret_cast<float4 *>(s_kap + p.nnu_pad);
    float4 *s_mom = s_nu + p.nnu_pad;
    // chunked form: the radial constants of every chunk after the bin tables
    float2 *s_dr_mc = reinterpret_cast<float2 *>(s_mom + 2 * p.nnu_pad);
    float4 *s_gqa_mc = reinterpret_cast<float4 *>(s_dr_mc + (MC ? ray_chunk_pairs(C, G, p.nr) : 0));
    __shared__ ESum s_red[W][2];
    ray_tables<C, W, P>(p, G, rs, s_kap, s_nu, s_mom);
    if constexpr (MC) ray_tables_mc<C, W, G>(p, s_dr_mc, s_gqa_mc);
    __syncthreads();

    ESum eabs, eesc;
    eabs.zero();
    eesc.zero();
    const unsigned slots = (p.nrays + R - 1) / R;
    constexpr int WG = W / P;  // ray groups per CTA
    ray_slots<C, W, MODE, G, P, TW, LUT, MC>(p, blockIdx.x * WG + warp / P, slots, gridDim.x * WG, rs, s_kap, s_nu,
                                             s_mom, eabs, eesc, s_dr_mc, s_gqa_mc);

    for (int o = 16; o > 0; o >>= 1) {
        eabs.add(eabs.shfl_xor(o));
        eesc.add(eesc.shfl_xor(o));
    }
    if (lane == 0) { s_red[warp][0] = eabs; s_red[warp][1] = eesc; }
    __syncthreads();
    if (tid == 0) {
        ESum sa = s_red[0][0], se = s_red[0][1];
        for (int w2 = 1; w2 < W; ++w2) { sa.add(s_red[w2][0]); se.add(s_red[w2][1]); }
        p.partials[blockIdx.x] = make_double2(to_double(sa), to_double(se));
    }
}

template <int C, int W, int MODE, int MINB, int G, int P, bool TW, bool LUT, bool MC = false>
cudaError_t launch_ray_g(const TraceArgs &a, cudaStream_t stream, unsigned *grid_out, unsigned max_grid)
{
    constexpr int R = 32 / G;
    const size_t smem = ray_bin_smem(a.nnu_pad) + 16 + (MC ? (size_t)ray_chunk_pairs(C, G, a.nr) * (8 + 16) : 0);
    auto kern = k_ray<C, W, MODE, MINB, G, P, TW, LUT, MC>;
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
    const unsigned need = (a.nrays * P + W * R - 1) / (W * R);
    if (grid > need) grid = need;
    if (max_grid > 0 && grid > max_grid) grid = max_grid;
    if (grid < 1) grid = 1;
    kern<<<grid, W * 32, smem, stream>>>(a);
    *grid_out = grid;
    return cudaGetLastError();
}

}  // namespace
}  // namespace rt
