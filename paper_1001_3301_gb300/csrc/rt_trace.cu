// Fused frequency-dependent ray tracer (Kuiper et al. 2010, Sect. 2.2-2.3, 3.3.4).
//
// Work decomposition
//   The rays of a grid are laid out one after another, each followed by one
//   virtual "escape" cell (flattened index f = ray * (nr + 1) + k, k = nr is the
//   escape cell). A CTA owns a contiguous tile of T = 32 * W * C flattened cells;
//   every lane owns C consecutive ones. Rays therefore straddle lanes, warps and
//   tiles freely and no lane idles on a ragged nr.
//
// Per tile
//   1. stage the tile's rho and T_dust (one contiguous run of memory) and the bin
//      table in shared memory;
//   2. column density of every cell's dust, dN = [T <= t_sub] rho dr, and an
//      exclusive segmented prefix sum N_in of it along each ray (Eq. 19; the
//      opacity depends on frequency only, so tau_nu,in = kappa_nu N_in and one scan
//      serves every bin). Lane-serial, then warp shuffles, then across warps; in
//      compensated double-float FP32 (or FP64). The part of a ray that lies in
//      earlier tiles is re-summed from global memory (at most nr cells), so no tile
//      waits for another;
//   3. for every bin: g = F_i/F_max e^{-kappa_i N_in} (Eq. 17 without the dilution,
//      which Eq. 36 removes) and the absorbed fraction 1 - e^{-kappa_i dN} (Eqs.
//      31-32) accumulated into one register per cell; the escape cell takes
//      fraction 1 and so collects the escaping power (Eqs. 33-35);
//   4. q_abs = Gq(r) * sum, a_rad = q_abs / (rho c) (Sect. 5; its rho -> 0 limit
//      where rho == 0), and per-tile FP64 energy partials.
//
// FP32 arithmetic per (cell, bin): exponentials on the MUFU unit (ex2.approx);
// 1 - 2^y for small |y| from its Taylor series on the FMA pipe, where 1 - ex2(y)
// would cancel.
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

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Running sums of one ray's column density. KahanSum is double-float: value = hi + lo.
struct KahanSum {
    float hi, lo;
    __device__ void zero() { hi = lo = 0.0f; }
    __device__ void add(float v)
    {
        float s, e;
        two_sum(hi, v, s, e);
        hi = s;
        lo += e;
    }
    __device__ void add(const KahanSum &o)
    {
        float s, e;
        two_sum(o.hi, hi, s, e);
        hi = s;
        lo = lo + o.lo + e;
    }
    __device__ float value() const { return hi + lo; }
    __device__ KahanSum shfl_up(int d) const
    {
        KahanSum r;
        r.hi = __shfl_up_sync(0xffffffffu, hi, d);
        r.lo = __shfl_up_sync(0xffffffffu, lo, d);
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
    __device__ PlainSum shfl_up(int d) const
    {
        PlainSum r;
        r.hi = __shfl_up_sync(0xffffffffu, hi, d);
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

// 1 - 2^y = -sum_{n>=1} (y ln2)^n / n!  =  y * P(y),  P(y) = sum_{n=0}^{4} p_n y^n,
// p_n = -ln2^{n+1} / (n+1)!. Used for -Y0 < y <= 0 (dtau < 1/8): the first omitted
// term is below 4.2e-8 of the value there.
constexpr double kDtauSplit = 0.125;
constexpr float kY0 = (float)(kDtauSplit * kLog2e);
constexpr float kP0 = (float)(-kLn2);
constexpr float kP1 = (float)(-kLn2 * kLn2 / 2.0);
constexpr float kP2 = (float)(-kLn2 * kLn2 * kLn2 / 6.0);
constexpr float kP3 = (float)(-kLn2 * kLn2 * kLn2 * kLn2 / 24.0);
constexpr float kP4 = (float)(-kLn2 * kLn2 * kLn2 * kLn2 * kLn2 / 120.0);

// absorbed fraction 1 - 2^y of one cell in one bin, y = -kappa dN log2(e) <= 0
__device__ __forceinline__ float absorbed_fraction(float y)
{
    const float big = 1.0f - ex2_approx(y);
    const float p = fmaf(fmaf(fmaf(fmaf(kP4, y, kP3), y, kP2), y, kP1), y, kP0);
    return (y > -kY0) ? y * p : big;
}

template <int MODE>
__device__ __forceinline__ auto cell_column(float rho, float td, int k, const TraceArgs &p)
{
    if constexpr (MODE == RT_FP64) {
        const double dr = __ldg(&p.rtab64[k].x);
        return (td <= p.t_sub) ? (double)rho * dr : 0.0;
    } else {
        const float dr = __ldg(&p.rtab[k].x);
        return (td <= p.t_sub) ? rho * dr : 0.0f;
    }
}

template <int C, int W, int MODE>
__global__ void __launch_bounds__(W * 32) k_trace(const TraceArgs p)
{
    using Real = typename std::conditional<MODE == RT_FP64, double, float>::type;
    using Sum = ColSum<MODE>;
    constexpr int T = 32 * W * C;

    extern __shared__ __align__(16) unsigned char smem[];
    float *s_rho = reinterpret_cast<float *>(smem);
    float *s_t = s_rho + T;
    float *s_kap = s_t + T;  // [nnu_pad]
    NuEntry *s_nu = reinterpret_cast<NuEntry *>(s_kap + p.nnu_pad);
    double2 *s_nu64 = reinterpret_cast<double2 *>(s_kap + p.nnu_pad);

    __shared__ Sum s_wsum[W];
    __shared__ int s_whead[W];
    __shared__ Sum s_carry;
    __shared__ double s_red[W][2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nr = p.nr, R1 = nr + 1;
    const long long f0 = (long long)blockIdx.x * T;
    const long long f1 = (f0 + T < p.L) ? f0 + T : p.L;
    const long long ray0 = f0 / R1;
    const int k0 = (int)(f0 - ray0 * R1);
    const long long m0 = ray0 * nr + (k0 < nr ? k0 : nr);
    const long long rayE = f1 / R1;
    const int kE = (int)(f1 - rayE * R1);
    const long long m1 = rayE * nr + (kE < nr ? kE : nr);
    const int nreal = (int)(m1 - m0);

    // 1. bin table and the tile's fields -> shared memory
    for (int i = tid; i < p.nnu_pad; i += W * 32) {
        s_kap[i] = p.kap[i];
        if constexpr (MODE == RT_FP64) s_nu64[i] = p.nu64[i];
        else s_nu[i] = p.nu[i];
    }
    for (int i = tid; i < nreal; i += W * 32) {
        s_rho[i] = __ldg(p.rho + m0 + i);
        s_t[i] = __ldg(p.tdust + m0 + i);
    }

    // 2a. column density of the part of ray0 that precedes this tile
    if (warp == 0) {
        Sum c;
        c.zero();
        const int kc = k0 < nr ? k0 : nr;
        const float *rr = p.rho + ray0 * nr;
        const float *tt = p.tdust + ray0 * nr;
        for (int k = lane; k < kc; k += 32) c.add(cell_column<MODE>(__ldg(rr + k), __ldg(tt + k), k, p));
        for (int o = 16; o > 0; o >>= 1) c.add(c.shfl_xor(o));
        if (lane == 0) s_carry = c;
    }
    __syncthreads();

    // 2b. this lane's cells
    const long long fl = f0 + (long long)(warp * 32 + lane) * C;
    const long long rayl = fl / R1;
    const int kl = (int)(fl - rayl * R1);
    Real D[C], N[C];
    unsigned real_m = 0, virt_m = 0, head_m = 0, zero_m = 0;
    bool bad = false;
    {
        long long ray = rayl;
        int k = kl;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            D[j] = Real(0);
            if (fl + j < f1) {
                if (k == 0) head_m |= 1u << j;
                if (k < nr) {
                    real_m |= 1u << j;
                    const int idx = (int)(ray * nr + k - m0);
                    const float rho = s_rho[idx], td = s_t[idx];
                    bad |= !(rho >= 0.0f && rho <= FLT_MAX) || (td != td);
                    D[j] = cell_column<MODE>(rho, td, k, p);
                    if (td <= p.t_sub && D[j] == Real(0)) zero_m |= 1u << j;
                } else {
                    virt_m |= 1u << j;
                }
            }
            if (++k > nr) { k = 0; ++ray; }
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(p.bad_input, p.seq);

    // 2c. segmented exclusive scan of D along each ray
    Sum agg;
    agg.zero();
    bool hh = false;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        if ((head_m >> j) & 1u) { agg.zero(); hh = true; }
        agg.add(D[j]);
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
    Sum pre = s_carry;
    for (int w = 0; w < warp; ++w) {
        if (s_whead[w]) pre = s_wsum[w];
        else pre.add(s_wsum[w]);
    }
    if (exh) pre = excl;
    else pre.add(excl);
#pragma unroll
    for (int j = 0; j < C; ++j) {
        if ((head_m >> j) & 1u) pre.zero();
        N[j] = pre.value();
        pre.add(D[j]);
        if ((virt_m >> j) & 1u) D[j] = Real(INFINITY);  // escape cell absorbs all
    }

    // 3. frequency loop
    Real acc[C];
#pragma unroll
    for (int j = 0; j < C; ++j) acc[j] = Real(0);
    if constexpr (MODE == RT_FP64) {
#pragma unroll 1
        for (int i = 0; i < p.nnu_pad; ++i) {
            const double2 e = s_nu64[i];  // (kappa_i, F_i / F_max)
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const double g = e.y * exp(-e.x * N[j]);
                acc[j] = fma(g, -expm1(-e.x * D[j]), acc[j]);
            }
        }
    } else {
#pragma unroll 1
        for (int i = 0; i < p.nnu_pad; i += kNuPad) {
#pragma unroll
            for (int u = 0; u < kNuPad; ++u) {
                const NuEntry e = s_nu[i + u];
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const float g = ex2_approx(fmaf(e.nk, N[j], e.lf));
                    acc[j] = fmaf(g, absorbed_fraction(e.nk * D[j]), acc[j]);
                }
            }
        }
    }

    // rho == 0 cells with dust: the force limit sum_i kappa_i g_i (rare; per slot,
    // only in warps that hold such a cell). Reuses D (0 there).
#pragma unroll
    for (int j = 0; j < C; ++j) {
        if (__any_sync(0xffffffffu, (zero_m >> j) & 1u)) {
            Real s = Real(0);
            for (int i = 0; i < p.nnu_pad; ++i) {
                if constexpr (MODE == RT_FP64) s = fma((double)s_kap[i] * s_nu64[i].y, exp(-s_nu64[i].x * N[j]), s);
                else s = fmaf(s_kap[i], ex2_approx(fmaf(s_nu[i].nk, N[j], s_nu[i].lf)), s);
            }
            if ((zero_m >> j) & 1u) D[j] = s;
        }
    }

    // 4a. energy partials: per ray, compensated FP32 (or FP64) sum of the lane's
    // absorbed cells, weighted by the ray's solid angle in FP64
    double e_abs = 0.0, e_esc = 0.0;
    {
        long long ray = rayl;
        int k = kl;
        Sum part;
        part.zero();
        long long pray = -1;  // ray of the cells summed in `part`, -1 if none
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if ((real_m >> j) & 1u) { part.add(acc[j]); pray = ray; }
            if ((virt_m >> j) & 1u) {
                const double w = __ldg(p.domega + ray);
                if (pray >= 0) e_abs += (double)part.value() * w;
                e_esc += (double)acc[j] * w;
                part.zero();
                pray = -1;
            }
            if (++k > nr) { k = 0; ++ray; }
        }
        if (pray >= 0) e_abs += (double)part.value() * __ldg(p.domega + pray);
    }

    // 4b. q_abs and a_rad into registers (reusing acc and N)
    {
        long long ray = rayl;
        int k = kl;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if ((real_m >> j) & 1u) {
                const int idx = (int)(ray * nr + k - m0);
                const float rho = s_rho[idx];
                Real q, a;
                if constexpr (MODE == RT_FP64) {
                    const double4 g = p.rtab64[k];
                    q = g.y * acc[j];
                    a = ((zero_m >> j) & 1u) ? g.z * D[j]
                        : (D[j] > 0.0 ? q / ((double)rho * kC) : 0.0);
                } else {
                    const float4 g = __ldg(&p.rtab[k]);
                    q = g.y * acc[j];
                    a = ((zero_m >> j) & 1u) ? g.z * D[j]
                        : (D[j] > 0.0f ? q / (rho * (float)kC) : 0.0f);
                }
                acc[j] = q;
                N[j] = a;
            }
            if (++k > nr) { k = 0; ++ray; }
        }
    }
    __syncthreads();  // every lane has read s_rho

    // 4c. outputs through shared memory, then coalesced stores
    {
        long long ray = rayl;
        int k = kl;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if ((real_m >> j) & 1u) {
                const int idx = (int)(ray * nr + k - m0);
                s_rho[idx] = (float)acc[j];
                s_t[idx] = (float)N[j];
            }
            if (++k > nr) { k = 0; ++ray; }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        e_abs += __shfl_xor_sync(0xffffffffu, e_abs, o);
        e_esc += __shfl_xor_sync(0xffffffffu, e_esc, o);
    }
    if (lane == 0) { s_red[warp][0] = e_abs; s_red[warp][1] = e_esc; }
    __syncthreads();
    for (int i = tid; i < nreal; i += W * 32) {
        p.q[m0 + i] = s_rho[i];
        p.a[m0 + i] = s_t[i];
    }
    if (tid == 0) {
        double sa = 0.0, se = 0.0;
        for (int w = 0; w < W; ++w) { sa += s_red[w][0]; se += s_red[w][1]; }
        p.partials[blockIdx.x] = make_double2(sa, se);
    }
}

template <int C, int W, int MODE>
cudaError_t launch_shape(const TraceArgs &a, long long ntiles, cudaStream_t stream)
{
    constexpr int T = 32 * W * C;
    const size_t smem = (size_t)T * 2 * sizeof(float) + (size_t)a.nnu_pad * sizeof(float) +
                        (size_t)a.nnu_pad * (MODE == RT_FP64 ? sizeof(double2) : sizeof(NuEntry)) + 16;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_trace<C, W, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_trace<C, W, MODE><<<(unsigned)ntiles, W * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

using LaunchFn = cudaError_t (*)(const TraceArgs &, long long, cudaStream_t);
struct ShapeEntry {
    int precision, c, w;
    LaunchFn fn;
};

#define RT_SHAPE(P, C, W) {P, C, W, &launch_shape<C, W, P>}
const ShapeEntry kShapes[] = {
    RT_SHAPE(RT_FP32_KAHAN, 2, 4),  RT_SHAPE(RT_FP32_KAHAN, 4, 4),  RT_SHAPE(RT_FP32_KAHAN, 8, 4),
    RT_SHAPE(RT_FP32_KAHAN, 16, 4), RT_SHAPE(RT_FP32_KAHAN, 4, 8),  RT_SHAPE(RT_FP32_KAHAN, 8, 8),
    RT_SHAPE(RT_FP32_KAHAN, 16, 8), RT_SHAPE(RT_FP32_PLAIN, 2, 4),  RT_SHAPE(RT_FP32_PLAIN, 4, 4),
    RT_SHAPE(RT_FP32_PLAIN, 8, 4),  RT_SHAPE(RT_FP32_PLAIN, 16, 4), RT_SHAPE(RT_FP32_PLAIN, 8, 8),
    RT_SHAPE(RT_FP32_PLAIN, 16, 8), RT_SHAPE(RT_FP64, 2, 4),        RT_SHAPE(RT_FP64, 4, 4),
    RT_SHAPE(RT_FP64, 8, 4),
};
#undef RT_SHAPE

const ShapeEntry *find_shape(int precision, int c, int w)
{
    for (const ShapeEntry &s : kShapes)
        if (s.precision == precision && s.c == c && s.w == w) return &s;
    return nullptr;
}

}  // namespace

bool trace_shape_supported(int precision, int cells_per_lane, int warps)
{
    return find_shape(precision, cells_per_lane, warps) != nullptr;
}

int trace_shapes(int precision, Shape *out, int max_out)
{
    int n = 0;
    for (const ShapeEntry &s : kShapes)
        if (s.precision == precision && n < max_out) out[n++] = Shape{s.c, s.w};
    return n;
}

long long trace_tile_cells(Shape s) { return 32LL * s.warps * s.cells_per_lane; }

cudaError_t launch_trace(int precision, Shape s, const TraceArgs &args, long long ntiles,
                         cudaStream_t stream)
{
    const ShapeEntry *e = find_shape(precision, s.cells_per_lane, s.warps);
    if (!e) return cudaErrorInvalidValue;
    return e->fn(args, ntiles, stream);
}

}  // namespace rt
