// Device helpers shared by the two tracer kernels (rt_trace.cu: flattened tiles;
// rt_ray.cu: one warp per ray): the hardware exp2, compensated FP32 sums, packed
// per-lane cell storage, and the per-bin absorbed-fraction classes.
//
// FP32 arithmetic per (cell, bin). The exponential g = F_i/F_max e^{-kappa_i N_in}
// runs on the MUFU unit (ex2.approx). The absorbed fraction 1 - 2^y,
// y = -kappa dN log2(e) (Eqs. 31-32), is taken from whichever form is exact to well
// below the accuracy target:
//   - the Taylor series of 1 - e^{-x} truncated after n terms (n = 1, 2, 3, 5),
//     where the largest x in the warp keeps the first omitted term x^n/(n+1)! below
//     5e-7 of the value (FMA pipe only, no cancellation);
//   - 1 - ex2(y) (MUFU), where every x in the warp is at least 1/8, so the hardware
//     exp2 error (measured below 1.5e-7) is amplified by at most 7.5;
//   - both, and the smaller of the two (the 5-term series bounds 1 - e^{-x} from
//     above), for the bins whose x straddles 1/8 in the warp.
// The bins are sorted by opacity at set-up, so each class is one contiguous range of
// bins per warp, found with a few ballots; the loops carry no per-bin branch. Two
// cells share every FMA-pipe instruction (packed f32x2).
#pragma once

#include <float.h>
#include <math.h>

#include <type_traits>

#include "rt_internal.cuh"

namespace rt {
namespace {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 ex2_approx2(float2 x)
{
    return make_float2(ex2_approx(x.x), ex2_approx(x.y));
}

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// the hardware reciprocal (relative error below 2^-22; 0 for +-Inf, flushes subnormals)
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Running sums of one ray's column density. KahanSum is a compensated FP32 pair:
// value = hi + lo; two pairs combine exactly with TwoSum.
struct KahanSum {
    float hi, lo;
    __device__ void zero() { hi = lo = 0.0f; }
    // one term: Kahan's compensated summation (lo carries the lost low-order part;
    // error below 2 eps of the sum of the terms, in any order)
    __device__ void add(float v)
    {
        const float y = v + lo;
        const float t = hi + y;
        lo = y - (t - hi);
        hi = t;
    }
    __device__ void add(const KahanSum &o)
    {
        float s, e;
        two_sum(o.hi, hi, s, e);
        hi = s;
        lo = lo + o.lo + e;
    }
    __device__ float value() const { return hi + lo; }
    // the pair nearest to an FP64 value: hi its float rounding, lo the rest
    __device__ void set(double d)
    {
        hi = (float)d;
        lo = (float)(d - (double)hi);
    }
    __device__ KahanSum shfl_up(int d, int width = 32) const
    {
        KahanSum r;
        r.hi = __shfl_up_sync(0xffffffffu, hi, d, width);
        r.lo = __shfl_up_sync(0xffffffffu, lo, d, width);
        return r;
    }
    __device__ KahanSum shfl_xor(int d) const
    {
        KahanSum r;
        r.hi = __shfl_xor_sync(0xffffffffu, hi, d);
        r.lo = __shfl_xor_sync(0xffffffffu, lo, d);
        return r;
    }
};

template <typename Real>
struct PlainSum {  // one accumulator, no compensation
    Real hi;
    __device__ void zero() { hi = Real(0); }
    __device__ void add(Real v) { hi += v; }
    __device__ void add(const PlainSum &o) { hi += o.hi; }
    __device__ Real value() const { return hi; }
    __device__ void set(double d) { hi = (Real)d; }
    __device__ PlainSum shfl_up(int d, int width = 32) const
    {
        PlainSum r;
        r.hi = __shfl_up_sync(0xffffffffu, hi, d, width);
        return r;
    }
    __device__ PlainSum shfl_xor(int d) const
    {
        PlainSum r;
        r.hi = __shfl_xor_sync(0xffffffffu, hi, d);
        return r;
    }
};

// the column-density sum of each precision mode
template <int MODE>
using ColSum = typename std::conditional<
    MODE == RT_FP32_KAHAN, KahanSum,
    typename std::conditional<MODE == RT_FP64, PlainSum<double>, PlainSum<float>>::type>::type;

// Per-lane cell values. In FP32 they are stored as packed pairs (the layout the
// f32x2 bin loop works on), so no second scalar copy stays alive in registers;
// get/set with a compile-time j resolve to one register.
template <typename Real, int C>
struct Cells {
    Real v[C];
    __device__ __forceinline__ Real get(int j) const { return v[j]; }
    __device__ __forceinline__ void set(int j, Real x) { v[j] = x; }
};
template <int C>
struct Cells<float, C> {
    float2 v[C / 2];
    __device__ __forceinline__ float get(int j) const { return (j & 1) ? v[j >> 1].y : v[j >> 1].x; }
    __device__ __forceinline__ void set(int j, float x)
    {
        if (j & 1) v[j >> 1].y = x;
        else v[j >> 1].x = x;
    }
};

// 1 - 2^y = -sum_{k>=1} (y ln2)^k / k!  =  y * sum_{k>=0} p_k y^k,
// p_k = -ln2^{k+1} / (k+1)!  (Taylor series of 1 - e^{-x} at x = -y ln2 >= 0).
__host__ __device__ constexpr double taylor_coeff(int k)
{
    double c = -kLn2;
    for (int i = 1; i <= k; ++i) c *= kLn2 / (i + 1);
    return c;
}

// 1 / k! (a compile-time constant for constant k)
__host__ __device__ constexpr double inv_factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return 1.0 / f;
}

// Largest x = kappa dN for which n terms keep the first omitted term x^n/(n+1)!
// below 5e-7 of the value; the last class ends where the MUFU form takes over.
constexpr double kTrunc = 5e-7;
constexpr double kXSplit = 0.125;
__host__ __device__ constexpr double taylor_xmax(int n)
{
    // solve x^n / (n+1)! = kTrunc by bisection at compile time
    double fact = 1.0;
    for (int i = 2; i <= n + 1; ++i) fact *= i;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        double p = 1.0;
        for (int i = 0; i < n; ++i) p *= mid;
        if (p / fact < kTrunc) lo = mid;
        else hi = mid;
    }
    return lo < kXSplit ? lo : kXSplit;
}

// |y| thresholds (log2 units) of the classes n = 1..3, and the MUFU split
constexpr float kYT1 = (float)(taylor_xmax(1) * kLog2e);
constexpr float kYT2 = (float)(taylor_xmax(2) * kLog2e);
constexpr float kYT3 = (float)(taylor_xmax(3) * kLog2e);
constexpr float kYSplit = (float)(kXSplit * kLog2e);

// y * sum_{k<n} p_k y^k for a pair of cells (Horner, packed)
template <int N>
__device__ __forceinline__ float2 taylor_fraction(float2 y)
{
    float2 p = f2((float)taylor_coeff(N - 1));
#pragma unroll
    for (int k = N - 2; k >= 0; --k) p = __ffma2_rn(p, y, f2((float)taylor_coeff(k)));
    return __fmul2_rn(y, p);
}

// Moment form of the truncated series for the classes with 1-3 terms. With
// c_k = p_k nk^{k+1} per bin,
//   sum_i g_i (1 - 2^{nk_i dN}) = sum_k dN^{k+1} M_k,   M_k = sum_i g_i c_{k,i},
// so each (cell, bin) costs one FMA per term (every term of one M_k has the sign of
// p_k: no cancellation), and dN enters once per cell and range (Horner).
// s_mom[2 i] = (c0, c0, c1, c1), s_mom[2 i + 1] = (c2, c2, c3, c3).
__device__ __forceinline__ void fill_moments(float4 *s_mom, int i, float nk)
{
    const float c0 = (float)taylor_coeff(0) * nk;
    const float c1 = (float)taylor_coeff(1) * nk * nk;
    const float c2 = (float)taylor_coeff(2) * nk * nk * nk;
    const float c3 = (float)taylor_coeff(3) * nk * nk * nk * nk;
    s_mom[2 * i] = make_float4(c0, c0, c1, c1);
    s_mom[2 * i + 1] = make_float4(c2, c2, c3, c3);
}

// n0: a column the cells' n2 are counted from (the exponent is nk (n0 + n2) + lf,
// taken as nk n2 + (nk n0 + lf)); 0 where n2 is the whole column.
template <int NT, int C>
__device__ __forceinline__ void moment_range(int i0, int i1, const float4 *s_nu, const float4 *s_mom, float n0,
                                             const float2 (&n2)[C / 2], const float2 (&d2)[C / 2],
                                             float2 (&a2)[C / 2])
{
    static_assert(NT >= 1 && NT <= 3, "moment form for 1-3 terms");
    if (i0 >= i1) return;  // warp-uniform
    float2 M[NT][C / 2];
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
        for (int m = 0; m < C / 2; ++m) M[k][m] = f2(0.0f);
#pragma unroll(NT <= 2 ? 2 : 1)
    for (int i = i0; i < i1; ++i) {
        const float4 e = s_nu[i];
        const float2 nk = make_float2(e.x, e.y), lf = f2(fmaf(e.x, n0, e.z));
        const float4 m01 = s_mom[2 * i];
        const float2 c0 = make_float2(m01.x, m01.y), c1 = make_float2(m01.z, m01.w);
        float2 c2 = f2(0.0f);
        if constexpr (NT >= 3) {
            const float4 m23 = s_mom[2 * i + 1];
            c2 = make_float2(m23.x, m23.y);
        }
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float2 g = ex2_approx2(__ffma2_rn(nk, n2[m], lf));
            M[0][m] = __ffma2_rn(g, c0, M[0][m]);
            if constexpr (NT >= 2) M[1][m] = __ffma2_rn(g, c1, M[1][m]);
            if constexpr (NT >= 3) M[2][m] = __ffma2_rn(g, c2, M[2][m]);
        }
    }
#pragma unroll
    for (int m = 0; m < C / 2; ++m) {
        float2 t = M[NT - 1][m];
#pragma unroll
        for (int k = NT - 2; k >= 0; --k) t = __ffma2_rn(t, d2[m], M[k][m]);
        a2[m] = __ffma2_rn(t, d2[m], a2[m]);
    }
}

// Bin classes per warp: 1, 2, 3, 5 = Taylor with that many terms, 6 = mixed,
// 7 = MUFU. Classes 1-3 run in the moment form above; bin_range serves 5-7.
template <int CLASS, int C>
__device__ __forceinline__ void bin_range(int i0, int i1, const float4 *s_nu, float n0, const float2 (&n2)[C / 2],
                                          const float2 (&d2)[C / 2], float2 (&a2)[C / 2])
{
#pragma unroll(CLASS <= 2 ? 2 : 1)
    for (int i = i0; i < i1; ++i) {
        const float4 e = s_nu[i];
        const float2 nk = make_float2(e.x, e.y), lf = f2(fmaf(e.x, n0, e.z));
        const float2 nk1 = __fmul2_rn(nk, f2((float)taylor_coeff(0)));  // class 1
#pragma unroll
        for (int m = 0; m < C / 2; ++m) {
            const float2 g = ex2_approx2(__ffma2_rn(nk, n2[m], lf));
            float2 om;
            if constexpr (CLASS == 1) {
                om = __fmul2_rn(nk1, d2[m]);
            } else {
                const float2 y = __fmul2_rn(nk, d2[m]);
                if constexpr (CLASS <= 5) {
                    om = taylor_fraction<CLASS>(y);
                } else if constexpr (CLASS == 7) {
                    om = __ffma2_rn(ex2_approx2(y), f2(-1.0f), f2(1.0f));
                } else {
                    // The 5-term series is an upper bound of 1 - e^{-x} for every x > 0
                    // (its derivative, the 4-term series of e^{-x}, bounds e^{-x} from
                    // above) and exact to 5e-9 of the value below x = 1/8; 1 - ex2(y) is
                    // within 2.1e-7 of it (ex2 error and rounding). The smaller of the
                    // series and 1 - ex2(y) + 2^-22 is therefore the series wherever the
                    // series is the accurate form, and within 1.6e-6 of the value
                    // elsewhere: no compare, no select.
                    const float2 big = __ffma2_rn(ex2_approx2(y), f2(-1.0f), f2(1.0f + 0x1p-22f));
                    const float2 small = taylor_fraction<5>(y);
                    om = make_float2(fminf(small.x, big.x), fminf(small.y, big.y));
                }
            }
            a2[m] = __ffma2_rn(g, om, a2[m]);
        }
    }
}

// Class boundaries of one warp: with the bins sorted by |nk| ascending, b1, b2,
// b3 and b5 count the bins whose largest |y| = |nk| dmax in the warp stays below
// the thresholds of 1, 2, 3 and 5 Taylor terms, and bb those whose smallest non-zero
// |y| = |nk| dmin stays below the MUFU split (bins from bb on are MUFU-only).
// Warp-uniform results; one pass over the bins, 32 at a time.
struct BinClasses {
    int b1, b2, b3, b5, bb;
};
// from > 0: only bins from the 32-bin chunk holding `from` on are looked at, and the
// bins before that chunk count as inside every class (exact for every boundary at or
// above `from`, which is how the thin-series caller uses them).
__device__ __forceinline__ BinClasses classify_bins(const float4 *s_nu, int n_active, int lane,
                                                     float dmax, float dmin, int from = 0)
{
    const int start = from & ~31;
    // dmax >= 0 and dmin >= 0 at every caller, so padding lanes (ak = inf) never count
    BinClasses c{start, start, start, start, start};
    for (int c0 = start; c0 < n_active; c0 += 32) {
        const int i = c0 + lane;
        const float ak = (i < n_active) ? -s_nu[i].x : INFINITY;
        const float ym = ak * dmax, yn = ak * dmin;
        c.b1 += __popc(__ballot_sync(0xffffffffu, ym < kYT1));
        c.b2 += __popc(__ballot_sync(0xffffffffu, ym < kYT2));
        c.b3 += __popc(__ballot_sync(0xffffffffu, ym < kYT3));
        c.b5 += __popc(__ballot_sync(0xffffffffu, ym < kYSplit));
        c.bb += __popc(__ballot_sync(0xffffffffu, yn < kYSplit));
    }
    c.bb = c.bb > c.b5 ? c.bb : c.b5;
    return c;
}

// Bins optically thin along every ray a warp holds: kappa_i N_max <= kThinX, N_max the
// largest total column of those rays. With the bins sorted by kappa ascending they
// are a prefix; the count is warp-uniform.
constexpr float kThinY = (float)(kThinX * kLog2e);  // the bound in the units of -nk
__device__ __forceinline__ int thin_count(const float4 *s_nu, int n_active, int lane, float nmax)
{
    // Padding lanes carry ak = inf and must never count: with a column of at least 0,
    // inf * n is inf or NaN. A negative or NaN column (invalid input, flagged) is taken
    // as 0 so that the count stays within n_active.
    nmax = fmaxf(nmax, 0.0f);
    int bt = 0;
    for (int c0 = 0; c0 < n_active; c0 += 32) {
        const int i = c0 + lane;
        const float ak = (i < n_active) ? -s_nu[i].x : INFINITY;
        bt += __popc(__ballot_sync(0xffffffffu, ak * nmax <= kThinY));
    }
    return bt;
}

// thin_count for two columns at once (one pass over the bins)
__device__ __forceinline__ void thin_counts(const float4 *s_nu, int n_active, int lane, float n1, float n2, int &b1,
                                            int &b2)
{
    n1 = fmaxf(n1, 0.0f);  // as in thin_count
    n2 = fmaxf(n2, 0.0f);
    b1 = b2 = 0;
    for (int c0 = 0; c0 < n_active; c0 += 32) {
        const int i = c0 + lane;
        const float ak = (i < n_active) ? -s_nu[i].x : INFINITY;
        b1 += __popc(__ballot_sync(0xffffffffu, ak * n1 <= kThinY));
        b2 += __popc(__ballot_sync(0xffffffffu, ak * n2 <= kThinY));
    }
}

// the larger of a and b, NaN if either is NaN (PTX max.NaN)
__device__ __forceinline__ float max_nan(float a, float b)
{
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// The bins i < b of a thin prefix (Eqs. 17, 19 and 31-32 summed over them) as one
// series. With Phi(u) = sum_{i<b} w_i e^{-kappa_i u}, a cell with column N in front of
// it and dN in it absorbs Phi(N) - Phi(N + dN). Expanding e^{-kappa u} in powers of
// kappa u and writing a = s (N + dN), c = s N (s = kappa_{b-1}, so a, c <= kThinX):
//   Phi(N) - Phi(N + dN) = dN s sum_{k>=1} C_k h_{k-1}(a, c),
//   h_{k-1}(a, c) = sum_{j<k} a^j c^{k-1-j} = (a^k - c^k) / (a - c),
// with C_k the row's coefficients. The sum over k is the divided difference of
// P(u) = sum_k C_k u^k between a and c, evaluated by the paired Horner recurrence
// (no a - c cancellation); all terms of one power carry one sign and |a|, |c| <=
// kThinX, so the alternating sum loses at most a factor e^{2 kThinX} of precision.
// row: the table row b (s, C_1 .. C_kThinTerms).
template <int C>
__device__ __forceinline__ void thin_series(const float *row, const float2 (&n2)[C / 2],
                                            const float2 (&d2)[C / 2], float2 (&a2)[C / 2])
{
    static_assert(kThinTerms >= 2, "paired Horner form needs two terms");
    const float s = __ldg(row);
    float c[kThinTerms + 1];
#pragma unroll
    for (int k = 1; k <= kThinTerms; ++k) c[k] = __ldg(row + k);
    const float2 s2 = f2(s);
#pragma unroll
    for (int m = 0; m < C / 2; ++m) {
        const float2 cc = __fmul2_rn(s2, n2[m]);
        const float2 aa = __ffma2_rn(s2, d2[m], cc);
        float2 dd = f2(c[kThinTerms]);
        float2 pc = __ffma2_rn(dd, cc, f2(c[kThinTerms - 1]));
#pragma unroll
        for (int k = kThinTerms - 2; k >= 1; --k) {
            dd = __ffma2_rn(dd, aa, pc);
            pc = __ffma2_rn(pc, cc, f2(c[k]));
        }
        dd = __ffma2_rn(dd, aa, pc);
        a2[m] = __ffma2_rn(__fmul2_rn(d2[m], dd), s2, a2[m]);
    }
}

// Escaping part of the thin bins of a row for a ray of total column n:
// sum_{i<b} w_i e^{-kappa_i n} = S_0 - sum_{k>=1} C_k (s n)^k with S_0 = sum_{i<b} w_i
// (the row's last entry); s n <= kThinX keeps the result above e^{-kThinX} S_0.
__device__ __forceinline__ float thin_escape(const float *row, float n)
{
    const float u = __ldg(row) * n;
    float p = __ldg(row + kThinTerms);
#pragma unroll
    for (int k = kThinTerms - 1; k >= 1; --k) p = fmaf(p, u, __ldg(row + k));
    return fmaf(-p, u, __ldg(row + kThinTerms + 1));
}

// solid angle of ray r of this launch, in the mode's precision
template <int MODE>
__device__ __forceinline__ auto solid_angle(const TraceArgs &p, unsigned r)
{
    if constexpr (MODE == RT_FP64) return __ldg(p.domega + r);
    else return __ldg(p.domega32 + r);
}

__device__ __forceinline__ double to_double(const KahanSum &s) { return (double)s.hi + (double)s.lo; }
__device__ __forceinline__ double to_double(const PlainSum<double> &s) { return s.hi; }
__device__ __forceinline__ double to_double(const PlainSum<float> &s) { return (double)s.hi; }

// acc += part * w for a compensated (hi, lo) part, or a plain FP64 one
__device__ __forceinline__ void add_weighted(KahanSum &acc, const KahanSum &part, float w)
{
    acc.add(part.hi * w);
    acc.add(part.lo * w);
}
__device__ __forceinline__ void add_weighted(PlainSum<double> &acc, const PlainSum<double> &part, double w)
{
    acc.add(part.hi * w);
}


}  // namespace
}  // namespace rt
