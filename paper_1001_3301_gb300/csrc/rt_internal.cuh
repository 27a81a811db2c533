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
// Padding bins have nk = -1, lf = -inf and contribute exactly zero.
struct alignas(8) NuEntry {
    float nk;
    float lf;
};

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

// Arguments of the fused tracer kernel (passed by value).
struct TraceArgs {
    const float *rho;
    const float *tdust;
    float *q;
    float *a;
    const NuEntry *nu;        // [nnu_pad]
    const float *kap;         // [nnu_pad] kappa_i (rho -> 0 force limit)
    const double2 *nu64;      // [nnu_pad] (kappa_i, F_i/F_max), FP64 mode
    const float4 *rtab;       // [nr] (dr, Gq, Ga0, 0)
    const double4 *rtab64;    // [nr] same in FP64
    const double *domega;     // [nrays]
    double2 *partials;        // [ntiles] (sum of absorbed, sum of escaped) / (R*^2 F_max)
    unsigned *bad_input;      // set to `seq` when an input value is invalid
    unsigned seq;
    long long L;              // flattened length nrays * (nr + 1)
    int nr;
    int nnu_pad;
    float t_sub;
};

// Launch shapes of the fused tracer that are compiled in.
struct Shape {
    int cells_per_lane;
    int warps;
};

// Host-side launchers (rt_trace.cu)
bool trace_shape_supported(int precision, int cells_per_lane, int warps);
int trace_shapes(int precision, Shape *out, int max_out);
long long trace_tile_cells(Shape s);
cudaError_t launch_trace(int precision, Shape s, const TraceArgs &args, long long ntiles,
                         cudaStream_t stream);

// Set-up kernels (rt_setup.cu)
cudaError_t launch_setup_bins(int n_nu, const double *nu_mid_dev, const double *kappa_dev,
                              double t_star, double r_star, int kappa_bf16,
                              double *f_bin_dev, NuEntry *nu_dev, float *kap_dev,
                              double2 *nu64_dev, DevScalars *sc_dev, cudaStream_t stream);
cudaError_t launch_setup_geometry(int nr, int ntheta, int nphi, const double *r_if_dev,
                                  const double *theta_if_dev, const double *phi_if_dev,
                                  double t_star, float4 *rtab, double4 *rtab64,
                                  double *domega, DevScalars *sc_dev, cudaStream_t stream);
cudaError_t launch_energy_reduce(const double2 *partials, long long ntiles,
                                 const DevScalars *sc_dev, rt_energy *out_dev,
                                 cudaStream_t stream);

}  // namespace rt
