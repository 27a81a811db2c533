// The flattened-tile tracer body shared by the single-grid kernel (rt_trace.cu)
// and the multi-grid batch kernel (rt_batch.cu): one CTA traces a contiguous range
// of tiles of one grid. See rt_trace.cu for the decomposition.
#pragma once

#include "rt_device.cuh"

namespace rt {
namespace {

// radial table staged in shared memory up to this many cells per ray
constexpr int kRtabSmemMax = 1024;

// Shared-memory index with one padding word per 32: lanes that own C consecutive
// cells read at stride C, which this skew spreads over distinct banks.
__device__ __forceinline__ int skew(int i) { return i + (i >> 5); }
// (rounded up to 4 floats so the float4 tables after the buffers stay 16-byte aligned)
template <int T>
constexpr int skewed_len() { return (T + T / 32 + 1 + 3) & ~3; }

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// energy sums of the tile kernel: compensated FP32 (the FP64 pipe of this part is
// far narrower than its FP32 pipes), plain FP64 in the FP64 mode
template <int MODE>
struct TileTypes {
    using ESum = typename std::conditional<MODE == RT_FP64, PlainSum<double>, KahanSum>::type;
};

// One CTA traces the tiles [t_begin, t_end) of the grid described by p,
// prefetching tile t+1 (cp.async, double buffer) while it computes tile t and
// handing the column of the ray that runs into the next tile over in shared
// memory; only the first tile of the range re-reads an earlier tile. The CTA's
// energy sums are added to eabs / eesc (per lane).
template <int C, int W, int MODE>
__device__ __forceinline__ void trace_tile_range(const TraceArgs &p, unsigned t_begin, unsigned t_end,
                                                 typename TileTypes<MODE>::ESum &eabs,
                                                 typename TileTypes<MODE>::ESum &eesc)
{
    using Real = typename std::conditional<MODE == RT_FP64, double, float>::type;
    using Sum = ColSum<MODE>;
    constexpr int T = 32 * W * C;
    static_assert(C % 2 == 0, "cells per lane must be even");

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nr = p.nr;
    const unsigned R1 = (unsigned)nr + 1u;
    const bool rt_staged = (MODE != RT_FP64) && nr <= kRtabSmemMax;

    // dynamic shared memory: input double buffer, output staging, radial table,
    // bin tables
    constexpr int TS = skewed_len<T>();
    const int nrs = rt_staged ? ((nr + nr / 32 + 1 + 3) & ~3) : 0;  // skewed radial length
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_in = reinterpret_cast<float *>(smem);  // [2][rho | tdust][TS]
    float *s_out = s_in + 4 * TS;                    // [q | a][TS]
    float *s_rdr = s_out + 2 * TS;                   // radial dr, Gq, Ga0 [nrs] each
    float *s_rgq = s_rdr + nrs;
    float *s_rga = s_rgq + nrs;
    float *s_kap = s_rga + nrs;
    // (nk, nk, lf, lf): each bin's constants duplicated for packed f32x2 math
    float4 *s_nu = reinterpret_cast<float4 *>(s_kap + p.nnu_pad);
    double2 *s_nu64 = reinterpret_cast<double2 *>(s_kap + p.nnu_pad);
    float4 *s_mom = s_nu + p.nnu_pad;  // series moments' constants (FP32 modes), two per bin

    __shared__ Sum s_wsum[W];
    __shared__ int s_whead[W];
    // The column of the ray that enters a tile crosses tile (and, for the first tile
    // of a CTA, block) boundaries in FP64: the re-summed part in front of the CTA's
    // first tile is added up in FP64, and the carry from tile to tile is held as an
    // FP64 value. Inside a tile the mode's own sum (compensated FP32 by default)
    // continues from it.
    __shared__ double s_cpart[W];  // first tile: per-warp shares of the re-summed column
    __shared__ double s_carry[2];  // column handed from tile to tile (double buffered)

    __syncthreads();  // a previous range of this CTA may still read the tables

    // tile t covers flattened cells [t T, min((t+1) T, L)); its real cells are the
    // contiguous field elements [m0, m0 + nreal)
    auto tile_bounds = [&](unsigned t, unsigned &f0, unsigned &f1, unsigned &m0, int &nreal, int &k0) {
        f0 = t * (unsigned)T;
        f1 = (f0 + (unsigned)T < p.L) ? f0 + (unsigned)T : p.L;
        const unsigned ray0 = p.r1div.div(f0);
        k0 = (int)(f0 - ray0 * R1);
        m0 = ray0 * (unsigned)nr + (unsigned)(k0 < nr ? k0 : nr);
        const unsigned rayE = p.r1div.div(f1);
        const int kE = (int)(f1 - rayE * R1);
        nreal = (int)(rayE * (unsigned)nr + (unsigned)(kE < nr ? kE : nr) - m0);
    };
    auto prefetch = [&](unsigned t, int buf) {
        unsigned f0, f1, m0;
        int nreal, k0;
        tile_bounds(t, f0, f1, m0, nreal, k0);
        float *dr = s_in + buf * 2 * TS;
        for (int i = tid; i < nreal; i += W * 32) {
            cp_async4(dr + skew(i), p.rho + m0 + i);
            cp_async4(dr + TS + skew(i), p.tdust + m0 + i);
        }
        cp_async_commit();
    };
    auto rad_dr = [&](int k) -> float { return rt_staged ? s_rdr[skew(k)] : __ldg(&p.rtab[k].x); };
    auto rad_gq = [&](int k) -> float { return rt_staged ? s_rgq[skew(k)] : __ldg(&p.rtab[k].y); };
    auto rad_ga = [&](int k) -> float { return rt_staged ? s_rga[skew(k)] : __ldg(&p.rtab[k].z); };
    auto column = [&](float rho, float td, int k) -> Real {
        if constexpr (MODE == RT_FP64) return (td <= p.t_sub) ? (double)rho * __ldg(&p.rtab64[k].x) : 0.0;
        else return (td <= p.t_sub) ? rho * rad_dr(k) : 0.0f;
    };

    // prologue: tables, first prefetch, the first tile's incoming column
    if (t_begin < t_end) prefetch(t_begin, 0);
    for (int i = tid; i < p.nnu_pad; i += W * 32) {
        s_kap[i] = p.kap[i];
        if constexpr (MODE == RT_FP64) {
            s_nu64[i] = p.nu64[i];
        } else {
            const NuEntry e = p.nu[i];
            s_nu[i] = make_float4(e.nk, e.nk, e.lf, e.lf);
            fill_moments(s_mom, i, e.nk);
        }
    }
    if (rt_staged)
        for (int k = tid; k < nr; k += W * 32) {
            const float4 g = __ldg(&p.rtab[k]);
            s_rdr[skew(k)] = g.x;
            s_rgq[skew(k)] = g.y;
            s_rga[skew(k)] = g.z;
        }
    __syncthreads();  // radial table visible before the column re-sum uses it
    if (t_begin < t_end) {
        unsigned f0, f1, m0;
        int nreal, k0;
        tile_bounds(t_begin, f0, f1, m0, nreal, k0);
        const unsigned ray0 = p.r1div.div(f0);
        double c = 0.0;
        const int kc = k0 < nr ? k0 : nr;
        const float *rr = p.rho + (size_t)ray0 * nr;
        const float *tt = p.tdust + (size_t)ray0 * nr;
        for (int k = tid; k < kc; k += W * 32) c += (double)column(__ldg(rr + k), __ldg(tt + k), k);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) s_cpart[warp] = c;
    }

    using ESum = typename TileTypes<MODE>::ESum;

    for (unsigned t = t_begin; t < t_end; ++t) {
        const int buf = (int)((t - t_begin) & 1u);
        if (t + 1 < t_end) prefetch(t + 1, buf ^ 1);
        else cp_async_commit();  // keep one group per iteration
        cp_async_wait_prev();    // this thread's copies of tile t have landed
        __syncthreads();         // ... and everyone else's

        unsigned f0, f1, m0;
        int nreal, k0;
        tile_bounds(t, f0, f1, m0, nreal, k0);
        const float *s_rho = s_in + buf * 2 * TS;
        const float *s_t = s_rho + TS;

        // this lane's cells: slot j is flattened cell fl + j with radial index k
        // (k == nr is the escape cell); real cells sit at consecutive tile
        // indices from idx0
        const unsigned fl = f0 + (unsigned)(warp * 32 + lane) * C;
        const unsigned rayl = p.r1div.div(fl);
        const int kl = (int)(fl - rayl * R1);
        const int idx0 = (int)(rayl * (unsigned)nr + (unsigned)(kl < nr ? kl : nr) - m0);
        Cells<Real, C> D, N;
        unsigned real_m = 0, virt_m = 0, head_m = 0, zero_m = 0;
        bool bad = false;
        {
            int k = kl, idx = idx0;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                D.set(j, Real(0));
                if (fl + j < f1) {
                    if (k == 0) head_m |= 1u << j;
                    if (k < nr) {
                        real_m |= 1u << j;
                        const float rho = s_rho[skew(idx)], td = s_t[skew(idx)];
                        bad |= !(rho >= 0.0f && rho <= FLT_MAX) || (td != td);
                        D.set(j, column(rho, td, k));
                        if (td <= p.t_sub && D.get(j) == Real(0)) zero_m |= 1u << j;
                        ++idx;
                    } else {
                        virt_m |= 1u << j;
                    }
                }
                if (++k > nr) k = 0;
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(p.bad_input, p.seq);

        // segmented exclusive scan of D along each ray
        Sum agg;
        agg.zero();
        bool hh = false;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if ((head_m >> j) & 1u) { agg.zero(); hh = true; }
            agg.add(D.get(j));
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Sum o = agg.shfl_up(d);
            const bool oh = __shfl_up_sync(0xffffffffu, hh, d);
            if (lane >= d) {
                if (!hh) agg.add(o);
                hh = hh || oh;
            }
        }
        Sum excl = agg.shfl_up(1);
        bool exh = __shfl_up_sync(0xffffffffu, hh, 1);
        if (lane == 0) { excl.zero(); exh = false; }
        if (lane == 31) { s_wsum[warp] = agg; s_whead[warp] = hh; }
        __syncthreads();
        Sum pre;
        if (t == t_begin) {
            double c0 = 0.0;
            for (int w = 0; w < W; ++w) c0 += s_cpart[w];
            pre.set(c0);
        } else {
            pre.set(s_carry[buf]);
        }
        for (int w = 0; w < warp; ++w) {
            if (s_whead[w]) pre = s_wsum[w];
            else pre.add(s_wsum[w]);
        }
        if (exh) pre = excl;
        else pre.add(excl);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if ((head_m >> j) & 1u) pre.zero();
            N.set(j, pre.value());
            pre.add(D.get(j));
        }
        // the column at the end of this tile continues into the next one
        if (tid == W * 32 - 1) s_carry[buf ^ 1] = to_double(pre);

        // frequency loop (escape cells carry D = 0 and absorb nothing here)
        Cells<Real, C> acc;
#pragma unroll
        for (int j = 0; j < C; ++j) acc.set(j, Real(0));
        if constexpr (MODE == RT_FP64) {
#pragma unroll 1
            for (int i = 0; i < p.nnu_pad; ++i) {
                const double2 e = s_nu64[i];  // (kappa_i, F_i / F_max)
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const double g = e.y * exp(-e.x * N.get(j));
                    acc.set(j, fma(g, -expm1(-e.x * D.get(j)), acc.get(j)));
                }
            }
        } else {
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
            const int na = p.n_active;
            const BinClasses bc = classify_bins(s_nu, na, lane, dmax, dmin);
            moment_range<1, C>(0, bc.b1, s_nu, s_mom, 0.0f, N.v, D.v, acc.v);
            moment_range<2, C>(bc.b1, bc.b2, s_nu, s_mom, 0.0f, N.v, D.v, acc.v);
            bin_range<3, C>(bc.b2, bc.b3, s_nu, 0.0f, N.v, D.v, acc.v);
            bin_range<5, C>(bc.b3, bc.b5, s_nu, 0.0f, N.v, D.v, acc.v);
            bin_range<6, C>(bc.b5, bc.bb, s_nu, 0.0f, N.v, D.v, acc.v);
            bin_range<7, C>(bc.bb, na, s_nu, 0.0f, N.v, D.v, acc.v);
        }

        // rho == 0 cells with dust: the force limit sum_i kappa_i g_i (rare; per
        // slot, only in warps that hold such a cell). Reuses D (0 there).
        if (__any_sync(0xffffffffu, zero_m != 0u)) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (__any_sync(0xffffffffu, (zero_m >> j) & 1u)) {
                Real s = Real(0);
                for (int i = 0; i < p.nnu_pad; ++i) {
                    if constexpr (MODE == RT_FP64) s = fma((double)s_kap[i] * s_nu64[i].y, exp(-s_nu64[i].x * N.get(j)), s);
                    else s = fmaf(s_kap[i], ex2_approx(fmaf(s_nu[i].x, N.get(j), s_nu[i].z)), s);
                }
                if ((zero_m >> j) & 1u) D.set(j, s);
            }
        }
        }

        // escaping power of every ray whose escape cell is in this warp: the
        // warp's lanes share the bins of sum_i F_i/F_max e^{-kappa_i N_total}
#pragma unroll
        for (int j = 0; j < C; ++j) {
            unsigned vb = __ballot_sync(0xffffffffu, (virt_m >> j) & 1u);
            while (vb) {
                const int src = __ffs(vb) - 1;
                vb &= vb - 1;
                const Real ntot = __shfl_sync(0xffffffffu, N.get(j), src);
                const unsigned fsrc = __shfl_sync(0xffffffffu, fl, src) + (unsigned)j;
                Real s = Real(0);
                for (int i = lane; i < p.nnu_pad; i += 32) {
                    if constexpr (MODE == RT_FP64) s += s_nu64[i].y * exp(-s_nu64[i].x * ntot);
                    else s += ex2_approx(fmaf(s_nu[i].x, ntot, s_nu[i].z));
                }
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) eesc.add(s * solid_angle<MODE>(p, p.r1div.div(fsrc)));
            }
        }

        // q_abs, a_rad (= q/(rho c) = Ga0 acc / dN) into the warp's slice of the
        // output staging; the lane's absorbed power, summed per ray and weighted by
        // the ray's solid angle, into the CTA's energy; then the warp stores its
        // contiguous run of cells
        {
            int k = kl, idx = idx0;
            unsigned ray = rayl;
            ESum part;
            part.zero();
            bool pend = false;
            unsigned pray = 0;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if ((real_m >> j) & 1u) {
                    if (pend && pray != ray) {
                        add_weighted(eabs, part, solid_angle<MODE>(p, pray));
                        part.zero();
                    }
                    part.add(acc.get(j));
                    pray = ray;
                    pend = true;
                    const bool zc = (zero_m >> j) & 1u;
                    const Real dj = D.get(j);
                    Real q, a;
                    if constexpr (MODE == RT_FP64) {
                        const RadRow64 g = p.rtab64[k];
                        q = zc ? 0.0 : g.y * acc.get(j);
                        a = g.z * (zc ? dj : (dj > 0.0 ? acc.get(j) / dj : 0.0));
                    } else {
                        q = (dj > 0.0f && !zc) ? rad_gq(k) * acc.get(j) : 0.0f;
                        a = rad_ga(k) * (zc ? dj : (dj > 0.0f ? __fdividef(acc.get(j), dj) : 0.0f));
                    }
                    s_out[skew(idx)] = (float)q;
                    s_out[TS + skew(idx)] = (float)a;
                    ++idx;
                }
                if (++k > nr) { k = 0; ++ray; }
            }
            if (pend) add_weighted(eabs, part, solid_angle<MODE>(p, pray));
            // the warp's real cells are the tile indices [lane 0's idx0, lane 31's
            // end); lanes past the end of a partial tile point beyond nreal
            const int wend_lane = idx;
            const int wbeg = min(__shfl_sync(0xffffffffu, idx0, 0), nreal);
            const int wend = min(__shfl_sync(0xffffffffu, wend_lane, 31), nreal);
            __syncwarp();
            for (int i = wbeg + lane; i < wend; i += 32) {
                p.q[m0 + i] = s_out[skew(i)];
                p.a[m0 + i] = s_out[TS + skew(i)];
            }
        }
    }
    cp_async_commit();  // no copies remain in flight at exit
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Block-wide sum of the per-lane energy sums; the result is valid in thread 0.
template <int W, typename ESum>
__device__ __forceinline__ void block_energy(ESum &eabs, ESum &eesc)
{
    __shared__ ESum s_red[W][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        eabs.add(eabs.shfl_xor(o));
        eesc.add(eesc.shfl_xor(o));
    }
    __syncthreads();  // s_red may still be read by a previous call
    if (lane == 0) { s_red[warp][0] = eabs; s_red[warp][1] = eesc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < W; ++w) { eabs.add(s_red[w][0]); eesc.add(s_red[w][1]); }
    }
}


template <int C, int W, int MODE>
size_t trace_smem_bytes(const TraceArgs &a)
{
    constexpr int TS = skewed_len<32 * W * C>();
    const bool staged = (MODE != RT_FP64) && a.nr <= kRtabSmemMax;
    const size_t nrs = staged ? (size_t)((a.nr + a.nr / 32 + 1 + 3) & ~3) : 0;
    return (size_t)TS * 6 * sizeof(float) + 3 * nrs * sizeof(float) +
           (size_t)a.nnu_pad * sizeof(float) + (size_t)a.nnu_pad * (16 + 32) + 16;
}

}  // namespace
}  // namespace rt
