// The warp-per-ray body of the frequency-dependent tracer (Kuiper et al. 2010,
// Sect. 2.2-2.3, 3.3.4), shared by the single-grid kernel (rt_ray.cu) and the
// multi-grid batch (rt_batch.cu).
//
// A segment of G lanes traces one radial ray (a warp holds 32 / G rays at a time,
// so rays shorter than 32 C cells keep every lane busy); lane l of a segment owns
// the cells [l C, (l+1) C) of its ray, so the radial constants of a lane never
// change and the ray's fields are read straight from HBM in 16-byte vectors (no
// staging, no block barrier in the ray loop). Per ray:
//   - dN = [T <= t_sub] rho dr per cell, and its exclusive prefix N_in along the
//     ray (Eq. 19, tau = 0 at the inner radius): compensated lane sums, then a
//     compensated warp scan;
//   - the bins optically thin along all the warp's rays as one power series in the
//     column (thin_series), the others by the per-bin loop of rt_device.cuh
//     (Eqs. 17, 20, 31-32), into one accumulator per cell, with the warp's bin
//     classes chosen from its largest and smallest column;
//   - escaping power sum_i F_i/F_max e^{-kappa_i N_total} (Eqs. 33-35), the lanes
//     sharing the bins outside the thin series (that part from the series row);
//   - q_abs = Gq acc and a_rad = q/(rho c) = Ga0 acc / dN (Sect. 5; the rho -> 0
//     limit where dN = 0 with dust), stored as 16-byte vectors;
//   - energy sums per lane.
#pragma once

#include "rt_device.cuh"

namespace rt {
namespace {

// Radial constants of every lane's cells, stored [j][lane] so that the lanes of a
// warp read consecutive words (lane l's cell j is radial index (l mod G) C + j; a
// [k] layout would put all 32 lanes on one shared-memory bank).
template <int C>
struct RayShared {
    float dr[C][32], gq[C][32], ga[C][32];
};

// dynamic shared memory of the bin tables: kappa, (nk, nk, lf, lf) and the series
// moments' constants (two float4 per bin)
__host__ __device__ constexpr size_t ray_bin_smem(int nnu_pad) { return (size_t)nnu_pad * (4 + 16 + 32); }

// The tables of grid p for G lanes per ray (call from every thread of the CTA,
// then __syncthreads()).
template <int C, int W>
__device__ __forceinline__ void ray_tables(const TraceArgs &p, int G, RayShared<C> &rs, float *s_kap, float4 *s_nu,
                                           float4 *s_mom)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < p.nnu_pad; i += W * 32) {
        s_kap[i] = p.kap[i];
        const NuEntry e = p.nu[i];
        s_nu[i] = make_float4(e.nk, e.nk, e.lf, e.lf);
        fill_moments(s_mom, i, e.nk);
    }
    for (int i = tid; i < 32 * C; i += W * 32) {
        const int l = i / C, j = i % C, k = (l % G) * C + j;
        const float4 g = (k < p.nr) ? __ldg(&p.rtab[k]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        rs.dr[j][l] = g.x;
        rs.gq[j][l] = g.y;
        rs.ga[j][l] = g.z;
    }
}

// Warp-slots wr = wr_begin, wr_begin + step, ... (< wr_end) of grid p, R = 32 / G rays
// each; the lanes' energy sums are added to eabs / eesc.
template <int C, int W, int MODE, int G>
__device__ __forceinline__ void ray_slots(const TraceArgs &p, unsigned wr_begin, unsigned wr_end, unsigned step,
                                          const RayShared<C> &rs, const float *s_kap, const float4 *s_nu,
                                          const float4 *s_mom, KahanSum &eabs, KahanSum &eesc)
{
    static_assert(MODE != RT_FP64, "the FP64 mode uses the tile kernel");
    static_assert(C % 2 == 0, "cells per lane must be even");
    static_assert(G == 8 || G == 16 || G == 32, "lanes per ray");
    using Sum = ColSum<MODE>;
    constexpr int V = (C % 4 == 0) ? 4 : 2;  // vector width of the field loads
    constexpr int R = 32 / G;                // rays per warp

    const int lane = threadIdx.x & 31;
    const int seg = lane / G, ll = lane % G;  // ray slot of the lane, lane within the ray
    const int nr = p.nr;
    const int c0 = ll * C;
    const int nv_ray = nr - c0 < 0 ? 0 : (nr - c0 > C ? C : nr - c0);  // valid cells of this lane
    // vector access needs every lane start and the field bases 4V-byte aligned
    const bool vec = (nr % V == 0) &&
                     ((reinterpret_cast<size_t>(p.rho) | reinterpret_cast<size_t>(p.tdust) |
                       reinterpret_cast<size_t>(p.q) | reinterpret_cast<size_t>(p.a)) % (4 * V) == 0);

    for (unsigned wr = wr_begin; wr < wr_end; wr += step) {
        const unsigned ray = wr * R + seg;
        const bool live = ray < p.nrays;  // the last warp may hold fewer than R rays
        const int nv = live ? nv_ray : 0;
        const size_t base = (size_t)(live ? ray : 0u) * nr + c0;
        float rho[C], td[C];
        if (vec && nv == C) {
#pragma unroll
            for (int j = 0; j < C; j += V) {
                if constexpr (V == 4) {
                    const float4 r4 = __ldg(reinterpret_cast<const float4 *>(p.rho + base + j));
                    const float4 t4 = __ldg(reinterpret_cast<const float4 *>(p.tdust + base + j));
                    rho[j] = r4.x; rho[j + 1] = r4.y; rho[j + 2] = r4.z; rho[j + 3] = r4.w;
                    td[j] = t4.x; td[j + 1] = t4.y; td[j + 2] = t4.z; td[j + 3] = t4.w;
                } else {
                    const float2 r2 = __ldg(reinterpret_cast<const float2 *>(p.rho + base + j));
                    const float2 t2 = __ldg(reinterpret_cast<const float2 *>(p.tdust + base + j));
                    rho[j] = r2.x; rho[j + 1] = r2.y;
                    td[j] = t2.x; td[j + 1] = t2.y;
                }
            }
        } else {
            // cells past the ray's end: no density, no dust (their column is 0 with any t_sub)
#pragma unroll
            for (int j = 0; j < C; ++j) {
                rho[j] = 0.0f;
                td[j] = INFINITY;
                if (j < nv) {
                    rho[j] = __ldg(p.rho + base + j);
                    td[j] = __ldg(p.tdust + base + j);
                }
            }
        }

        // column density of the dust in each cell, and invalid-input flags
        Cells<float, C> D, N, acc;
        unsigned zero_m = 0;
        bool bad = false;
        Sum lsum;
        lsum.zero();
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const bool dust = td[j] <= p.t_sub;
            const float d = dust ? rho[j] * rs.dr[j][lane] : 0.0f;
            D.set(j, d);
            bad |= !(rho[j] >= 0.0f && rho[j] <= FLT_MAX) || (td[j] != td[j]);
            if (dust && d == 0.0f) zero_m |= 1u << j;
            lsum.add(d);
        }
        zero_m &= nv >= 32 ? 0xffffffffu : (1u << nv) - 1u;  // cells of the ray only
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(p.bad_input, p.seq);

        // exclusive prefix along the ray: scan of the lane sums within the segment
        Sum inc = lsum;
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const Sum o = inc.shfl_up(d, G);
            if (ll >= d) inc.add(o);
        }
        Sum pre = inc.shfl_up(1, G);
        if (ll == 0) pre.zero();
#pragma unroll
        for (int j = 0; j < C; ++j) {
            N.set(j, pre.value());
            pre.add(D.get(j));
            acc.set(j, 0.0f);
        }
        const float ntot = __shfl_sync(0xffffffffu, pre.value(), G - 1, G);

        const int na = p.n_active;
        // bins thin along all the warp's rays: one series for the lot, the rest bin by bin
        float nmax = ntot;
        for (int o = G; o < 32; o <<= 1) nmax = fmaxf(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        const int bt = thin_count(s_nu, na, lane, nmax);
        const float *thin_row = p.kap + kKapTable + bt * kThinStride;
        if (bt > 0) thin_series<C>(thin_row, N.v, D.v, acc.v);
        if (bt < na) {  // warp-uniform
            // the warp's largest and smallest non-zero column decide each bin's class
            float dmax = 0.0f, dmin = INFINITY;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                dmax = fmaxf(dmax, D.get(j));
                if (D.get(j) > 0.0f) dmin = fminf(dmin, D.get(j));
            }
            for (int o = 16; o > 0; o >>= 1) {
                dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
                dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
            }
            const BinClasses bc = classify_bins(s_nu, na, lane, dmax, dmin, bt);
            const int t1 = max(bc.b1, bt), t2 = max(bc.b2, bt), t3 = max(bc.b3, bt), t5 = max(bc.b5, bt);
            const int tb = max(bc.bb, bt);
            moment_range<1, C>(bt, t1, s_nu, s_mom, N.v, D.v, acc.v);
            moment_range<2, C>(t1, t2, s_nu, s_mom, N.v, D.v, acc.v);
            bin_range<3, C>(t2, t3, s_nu, N.v, D.v, acc.v);
            bin_range<5, C>(t3, t5, s_nu, N.v, D.v, acc.v);
            bin_range<6, C>(t5, tb, s_nu, N.v, D.v, acc.v);
            bin_range<7, C>(tb, na, s_nu, N.v, D.v, acc.v);
        }

        // cells with dust but no column: the rho -> 0 force limit sum_i kappa_i g_i
        if (__any_sync(0xffffffffu, zero_m != 0u)) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (__any_sync(0xffffffffu, (zero_m >> j) & 1u)) {
                    float s = 0.0f;
                    for (int i = 0; i < p.nnu_pad; ++i)
                        s = fmaf(s_kap[i], ex2_approx(fmaf(s_nu[i].x, N.get(j), s_nu[i].z)), s);
                    if ((zero_m >> j) & 1u) D.set(j, s);
                }
            }
        }

        // escaping power of the ray, the lanes of its segment sharing the bins
        const float w = live ? __ldg(p.domega32 + ray) : 0.0f;
        {
            float s = 0.0f;
            for (int i = bt + ll; i < na; i += G) s += ex2_approx(fmaf(s_nu[i].x, ntot, s_nu[i].z));
            for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (ll == 0) {
                if (bt > 0) s += thin_escape(thin_row, ntot);
                eesc.add(s * w);
            }
        }

        // outputs and the lane's absorbed power
        // (a cell with no column, past the ray or without dust or density, absorbed 0)
        float qv[C], av[C];
        float lane_abs = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float aj = acc.get(j), dj = D.get(j);
            const bool zc = (zero_m >> j) & 1u;
            qv[j] = rs.gq[j][lane] * aj;
            av[j] = rs.ga[j][lane] * (zc ? dj : (dj > 0.0f ? __fdividef(aj, dj) : 0.0f));
            lane_abs += aj;
        }
        eabs.add(lane_abs * w);
        if (vec && nv == C) {
#pragma unroll
            for (int j = 0; j < C; j += V) {
                if constexpr (V == 4) {
                    *reinterpret_cast<float4 *>(p.q + base + j) = make_float4(qv[j], qv[j + 1], qv[j + 2], qv[j + 3]);
                    *reinterpret_cast<float4 *>(p.a + base + j) = make_float4(av[j], av[j + 1], av[j + 2], av[j + 3]);
                } else {
                    *reinterpret_cast<float2 *>(p.q + base + j) = make_float2(qv[j], qv[j + 1]);
                    *reinterpret_cast<float2 *>(p.a + base + j) = make_float2(av[j], av[j + 1]);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (j < nv) {
                    p.q[base + j] = qv[j];
                    p.a[base + j] = av[j];
                }
            }
        }
    }
}

}  // namespace
}  // namespace rt
