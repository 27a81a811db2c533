// Internal declarations shared by the translation units of the CUDA library.
// Nothing here is part of the public C ABI (include/rt_irradiation.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "rt_irradiation.h"

namespace rt {

// physical constants (cgs; CODATA 2018 exact SI values)
constexpr double kC = 2.99792458e10;      // speed of light, cm/s
constexpr double kH = 6.62607015e-27;     // Planck constant, erg s
constexpr double kKB = 1.380649e-16;      // Boltzmann constant, erg/K
constexpr double kPi = 3.14159265358979323846;
constexpr double kLog2e = 1.44269504088896340736;
constexpr double kLn2 = 0.69314718055994530942;

// padded bin count is a multiple of this (the bin loop is unrolled by it)
constexpr int kNuPad = 4;

// Per-bin table consumed by the FP32 tracer: nk = -kappa_i log2(e) and
// lf = log2(F_i / F_max), so F_i/F_max * exp(-kappa_i N) = 2^(nk N + lf).
// Only bins with kappa_i > 0 are listed, sorted by kappa ascending; padding bins
// after them have nk = -1, lf = -inf and contribute exactly zero.
struct alignas(8) NuEntry {
    float nk;
    float lf;
};

// Bins optically thin along every ray a warp holds (kappa_i N_total <= kThinX) are
// summed as one power series in the column instead of bin by bin (thin_series in
// rt_device.cuh). Its coefficients live in the buffer of the kappa table, after
// it: row b = 1..n_active holds s_b = kappa_{b-1} (column units) and then
// C_k(b) = (-1)^{k+1} / k! sum_{i<b} w_i (kappa_i / s_b)^k for k = 1..kThinTerms,
// then S_0(b) = sum_{i<b} w_i; w_i = F_i / F_max, bins in the kappa-sorted order.
// With x = kThinX the first omitted term is below x^kThinTerms / kThinTerms! =
// 2.8e-7 of the leading one; the alternating sum loses at most a factor
// e^{2 kThinX} = 7.4 of FP32 precision.
constexpr int kThinTerms = 10;
constexpr int kThinStride = 12;                                       // floats per row (>= kThinTerms + 2)
constexpr int kKapTable = RT_MAX_NU + kNuPad;                         // floats of the kappa table
constexpr int kKapBuffer = kKapTable + (RT_MAX_NU + 1) * kThinStride;  // with the series rows
constexpr float kThinX = 1.0f;
static_assert(kThinStride >= kThinTerms + 2, "a series row holds s, C_1..C_K and S_0");

// Scalars of one configured grid, resident in device memory.
struct DevScalars {
    double f_max;          // largest bin flux F_i (erg s^-1 cm^-2)
    double f_transparent;  // sum of F_i over bins with kappa_i == 0 (always escape)
    double sum_domega;     // sum over rays of dOmega_j (sr)
    double r2;             // R*^2
    double l_grid;         // R*^2 sigma T*^4 sum_j dOmega_j
    int n_active;          // bins with kappa_i > 0
    int nnu_pad;           // n_active rounded up to kNuPad (>= kNuPad)
};

// Division by an invariant 32-bit divisor d >= 1 with one multiply-high, two
// shifts and an add (Granlund & Montgomery 1994, unsigned case), exact for all
// 32-bit numerators.
struct FastDiv {
    unsigned m;
    int s1, s2;
    __host__ static FastDiv make(unsigned d)
    {
        int l = 0;
        while ((1ull << l) < d) ++l;  // ceil(log2 d)
        const unsigned long long m = (((1ull << l) - d) << 32) / d + 1;
        return FastDiv{(unsigned)m, l > 0 ? 1 : 0, l > 0 ? l - 1 : 0};
    }
    __device__ __forceinline__ unsigned div(unsigned n) const
    {
        const unsigned t = __umulhi(n, m);
        return (t + ((n - t) >> s1)) >> s2;
    }
};

// Radial constants of one cell in FP64: dr, Gq, Ga0 (and padding), 32-byte aligned.
struct alignas(32) RadRow64 {
    double x, y, z, w;
};

// Most temperature points of a temperature-dependent opacity table
constexpr int kMaxTdepPoints = 32;

// The lookup-table comparator's grid: s = log2(kappa_ref N_in + 2^-20) in [-20, 8],
// d = log2(kappa_ref dN + 2^-30) in [-30, 8], both in steps of 1/32 (rt_lut.cu).
constexpr int kLutNs = 897;
constexpr int kLutNd = 1217;
constexpr float kLutS0 = -20.0f;
constexpr float kLutD0 = -30.0f;
constexpr float kLutInvH = 32.0f;

// Largest flattened length one launch of the tracer covers; longer grids are
// split into ray chunks by the host.
constexpr long long kMaxLaunchCells = (1LL << 31) - (1LL << 16);

// Arguments of the fused tracer kernel (passed by value). Field, solid-angle and
// partials pointers are offset by the host to the launch's first ray / tile.
struct TraceArgs {
    const float *rho;
    const float *tdust;
    float *q;
    float *a;
    const NuEntry *nu;        // [nnu_pad]
    const float *kap;         // [nnu_pad] kappa_i (rho -> 0 force limit)
    const double2 *nu64;      // [nnu_pad] (kappa_i, F_i/F_max), FP64 mode
    const float4 *rtab;       // [nr] (dr, Gq, Ga0, 0)
    const RadRow64 *rtab64;    // [nr] same in FP64
    const double *domega;     // [nrays]
    const float *domega32;    // [nrays] the same in FP32
    double2 *partials;        // [CTAs] (sum of absorbed, sum of escaped) / (R*^2 F_max)
    unsigned *bad_input;      // set to `seq` when an input value is invalid
    unsigned seq;
    unsigned L;               // flattened length of this launch, nrays * (nr + 1)
    unsigned nrays;           // rays of this launch
    FastDiv r1div;            // division by nr + 1
    int nr;
    int nnu_pad;
    int n_active;             // bins with kappa > 0, sorted by kappa ascending
    float t_sub;
    // A temperature-dependent table that separates, kappa_i(T) = kappa_i b(T) (kappa_i
    // the bin's largest tabulated value): the column of a cell is weighted by b(T),
    // linear between the points of the temperature grid and held beyond its ends.
    // n_tw = 0: no weight (a table of kappa(nu) only).
    // Lookup-table comparator (rt_lut.cu): when lut is set, log2 G of every cell comes
    // from the bilinear table instead of the per-bin sum; a warp-slot holding a cell in
    // a flagged square (or off the table) takes the per-bin sum (one count per such
    // slot into lut_fallback, if set).
    const float2 *lut;        // [kLutNd][kLutNs] (log2 G at (s_i, d_j), at (s_{i+1}, d_j)); the lowest
                              // mantissa bit of .x: square (i, j) flagged
    float lut_kref;           // the reference opacity of the table's optical depths
    unsigned *lut_fallback;
    const float *tw_t;        // [kMaxTdepPoints] grid (K), padded with +Inf
    const float4 *tw_b;       // [kMaxTdepPoints] (T_j, T_{j+1}, b_j / dT, b_{j+1} / dT) per interval;
                              // (T_last, T_last + 1, b_last, b_last) from the last point on
    int n_tw;
};

// Launch shapes of the fused tracer that are compiled in.
constexpr int kKindTile = RT_KERNEL_TILE;  // flattened tiles, any nr (rt_trace.cu)
constexpr int kKindRay = RT_KERNEL_RAY;    // one warp per ray, nr <= 32 C (rt_ray.cu)
constexpr int kKindRayChunked = RT_KERNEL_RAY_CHUNKED;  // 8 lanes per ray, chunks of 8 C cells (rt_ray.cu)
constexpr int kMaxChunkedNr = 4096;                     // longest ray of the chunked form
struct Shape {
    int kind;
    int cells_per_lane;
    int warps;
    int min_blocks;  // minimum resident CTAs per SM the registers are capped for
};

// Lanes per ray of the warp-per-ray kernel with C cells per lane: the fewest of 8,
// 16 and 32 that hold the ray (a warp then traces 32 / G rays at a time).
inline int ray_lanes(int c, int nr) { return 8 * c >= nr ? 8 : (16 * c >= nr ? 16 : 32); }
// Warps per ray of the warp-per-ray kernel: 1 where 32 C cells hold the ray, 2 where
// 64 C do (for C <= 8: two warps of a CTA share a ray, exchanging their column sums
// in shared memory), 0 where the kernel does not apply.
inline int ray_warps_per_ray(int c, int nr) { return 32 * c >= nr ? 1 : ((c <= 8 && 64 * c >= nr) ? 2 : 0); }
// Cells of one ray that the lanes tracing it hold (G C, or 32 P C with P warps).
inline int ray_cells_held(int c, int nr)
{
    const int p = ray_warps_per_ray(c, nr);
    return p > 1 ? 32 * p * c : ray_lanes(c, nr) * c;
}

// Host-side launchers (rt_trace.cu, rt_ray.cu)
int trace_shapes(int precision, Shape *out, int max_out);      // tile kernel
int ray_shapes(int precision, int nr, Shape *out, int max_out);  // ray kernel, 32 C >= nr
// ray-kernel shapes compiled with the column weight of a separable kappa(nu, T) table
int ray_shapes_tw(int precision, int nr, Shape *out, int max_out);
// ray-kernel shapes compiled with the lookup-table comparator
int ray_shapes_lut(int precision, int nr, Shape *out, int max_out);
// shapes of the chunked ray kernel (8 C < nr <= kMaxChunkedNr), rt_ray_mc.cu
int ray_shapes_mc(int precision, int nr, Shape *out, int max_out);
cudaError_t launch_ray_mc_shape(int precision, Shape s, const TraceArgs &args, cudaStream_t stream,
                                unsigned *grid_out, unsigned max_grid);
long long trace_tile_cells(Shape s);
cudaError_t launch_ray_shape(int precision, Shape s, const TraceArgs &args, cudaStream_t stream,
                             unsigned *grid_out, unsigned max_grid = 0);
// Launches the persistent tracer over `ntiles` tiles; *grid_out receives the
// number of CTAs (= energy partials written). max_grid > 0 caps that number before
// the launch (the kernels are persistent: any grid of >= 1 CTA covers the work).
cudaError_t launch_trace(int precision, Shape s, const TraceArgs &args, unsigned ntiles,
                         cudaStream_t stream, unsigned *grid_out, unsigned max_grid = 0);

// Lookup-table comparator (rt_lut.cu): builds the [kLutNd][kLutNs] table of log2 G
// pairs with square flags for the tolerance tol (raw: kLutNs * kLutNd floats of scratch)
cudaError_t launch_build_lut(const NuEntry *nu, const DevScalars *sc, double kref, float *raw, float2 *tab, double tol,
                             cudaStream_t st);

// Tracer with temperature-dependent opacity tables (rt_tdep.cu)
int tdep_shapes(int nr, Shape *out, int max_out);
cudaError_t launch_tdep(Shape s, const TraceArgs &args, const float2 *kt2, const float *tg, int n_t,
                        cudaStream_t stream, unsigned *grid_out);
cudaError_t launch_build_tdep(int n_active, int nnu_pad, int n_t, const double *kappa_t, const int *order,
                              float2 *kt2, cudaStream_t stream);
// Tracer for kappa(nu, T) tables of rank 2-4: that many columns per ray (rt_tdep2.cu)
int tdep2_shapes(int rank, int nr, Shape *out, int max_out);
cudaError_t launch_tdep2(int rank, Shape s, const TraceArgs &args, const float4 *kr, const float4 *bw, const float *tg,
                         int n_t, cudaStream_t stream, unsigned *grid_out);
cudaError_t launch_build_rank2(int n_active, int nnu_pad, const double *fac_a, const int *order, float4 *kr,
                               cudaStream_t stream);

// A configured context's device tables, for the batch launcher (rt_api.cu).
struct CtxView {
    TraceArgs args;        // tables and sizes; field pointers, partials, validity word unset
    DevScalars *sc;        // device scalars of the grid
    int precision;
    int dev;
    long long flat_cells;  // nrays * (nr + 1)
    long long ncells;
    bool tdep;             // temperature-dependent opacity table (not batched)
};
}  // namespace rt
struct rt_ctx;
namespace rt {
bool ctx_view(const rt_ctx *c, CtxView *v);
void set_thread_error(const std::string &msg);  // text for rt_last_error(NULL)

// What the learned surrogate (rt_surrogate.cu) reads of a context (rt_api.cu).
struct CtxInfo {
    int dev;
    cudaStream_t stream;
    bool configured;
    int nr, ntheta, nphi;
    const double *r_if_h, *theta_if_h, *phi_if_h;  // host copies of the cell interfaces
    long long nrays, ncells;
    double t_sub, t_star, r_star;
    int n_nu;
    const double *nu_h;        // host copies of the table the tracer uses (kappa
    const double *kappa_h;     // after the optional BF16 rounding)
    unsigned long long table_fingerprint;  // of (n_nu, nu, kappa, t_sub, t_star)
    int n_t;                   // > 0: temperature-dependent table on t_grid_h [n_t],
    const double *t_grid_h;    // kappa_t_h [n_nu][n_t] (then kappa_h holds each bin's
    const double *kappa_t_h;   // largest value)
    const float4 *rtab;        // [nr] (dr, Gq, Ga0, 0)
    const float *domega32;     // [nrays]
    const NuEntry *nu_tab;     // [nnu_pad], kappa-sorted active bins
    const float *kap;          // [nnu_pad]
    DevScalars sc;             // host copy of the grid's scalars
};
struct SurState;
bool ctx_info(const rt_ctx *c, CtxInfo *out);
SurState *&ctx_surrogate(rt_ctx *c);   // owned by the context, freed by rt_destroy
// the context's Planck-mean table of the temperature update (device, freed by
// rt_destroy) and the table fingerprint it was built for
float *&ctx_temp_table(rt_ctx *c);
unsigned long long &ctx_temp_fingerprint(rt_ctx *c);
void sur_free(SurState *s);
// workspace of the flux-limited-diffusion step (rt_fld.cu), owned by the context
struct FldState;
FldState *&ctx_fld(rt_ctx *c);
void fld_free(FldState *s);
int ctx_fail(rt_ctx *c, int status, const std::string &msg);

// Set-up kernels (rt_setup.cu)
// order_dev (may be null) receives the original index of every kappa-sorted bin
cudaError_t launch_setup_bins(int n_nu, const double *nu_mid_dev, const double *kappa_dev,
                              double t_star, double r_star, int kappa_bf16,
                              double *f_bin_dev, NuEntry *nu_dev, float *kap_dev,
                              double2 *nu64_dev, DevScalars *sc_dev, cudaStream_t stream,
                              int *order_dev = nullptr);
cudaError_t launch_setup_geometry(int nr, int ntheta, int nphi, const double *r_if_dev,
                                  const double *theta_if_dev, const double *phi_if_dev,
                                  double t_star, float4 *rtab, RadRow64 *rtab64,
                                  double *domega, float *domega32, DevScalars *sc_dev,
                                  cudaStream_t stream);
cudaError_t launch_energy_reduce(const double2 *partials, long long ntiles,
                                 const DevScalars *sc_dev, rt_energy *out_dev,
                                 cudaStream_t stream);

}  // namespace rt
