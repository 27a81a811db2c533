// Allocation-free form of the tracer: rt_irradiate_static.
//
// Some callers cannot allocate device memory at the moment they need the
// irradiation: a host code whose own pool allocator has already reserved the GPU
// memory, or a time-stepping loop where cudaMalloc/cudaFree (which synchronise
// the device) would stall other work. rt_irradiate_static serves them: it takes
// the whole problem by argument and keeps every intermediate (copied grid and bin
// arrays, per-bin and per-radius tables, per-ray solid angles, per-CTA energy
// partials, the input-validity word and the energy result) in one file-scope
// device array of fixed size. It calls no cudaMalloc, cudaFree or allocating
// library routine; the set-up, tracer and reduction kernels are the same ones
// rt_irradiate launches, only pointed at this array.
#include <stddef.h>

#include <mutex>
#include <string>

#include "rt_internal.cuh"

namespace rt {
void set_thread_error(const std::string &msg);  // rt_api.cu: text for rt_last_error(NULL)
}

namespace {

// Limits of the static scratch (see include/rt_irradiation.h).
constexpr int kStaticMaxNr = RT_STATIC_MAX_NR;
constexpr int kStaticMaxTheta = RT_STATIC_MAX_NTHETA;
constexpr int kStaticMaxPhi = RT_STATIC_MAX_NPHI;
constexpr long long kStaticMaxRays = RT_STATIC_MAX_RAYS;
constexpr int kStaticMaxCtas = 8192;  // energy partials; the launch is capped at this many CTAs

struct StaticScratch {
    double r_if[kStaticMaxNr + 1];
    double theta_if[kStaticMaxTheta + 1];
    double phi_if[kStaticMaxPhi + 1];
    double nu_mid[RT_MAX_NU];
    double kappa[RT_MAX_NU];
    double f_bin[RT_MAX_NU];
    rt::NuEntry nu_tab[RT_MAX_NU + rt::kNuPad];
    float kap[rt::kKapBuffer];  // kappa table, then the thin-ray series rows
    double2 nu64[RT_MAX_NU + rt::kNuPad];
    float4 rtab[kStaticMaxNr];
    rt::RadRow64 rtab64[kStaticMaxNr];
    double domega[kStaticMaxRays];
    float domega32[kStaticMaxRays];
    double2 partials[kStaticMaxCtas];
    rt::DevScalars sc;
    rt_energy energy;
    unsigned bad;
};

// The scratch itself. In host code this name is only a stand-in for the symbol;
// its device address comes from cudaGetSymbolAddress (once per device, below).
static __device__ __align__(256) unsigned char g_rt_static_scratch[sizeof(StaticScratch)];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
StaticScratch *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, resolved on first use.
int scratch_address(StaticScratch **out, std::string &err)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return RT_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device ordinal beyond the static-scratch table";
        return RT_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rt_static_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return RT_ERR_CUDA;
        }
        g_static_ptr[dev] = static_cast<StaticScratch *>(p);
    }
    *out = g_static_ptr[dev];
    return RT_OK;
}

bool increasing_finite(const double *a, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(a[i]) || (i > 0 && !(a[i] > a[i - 1]))) return false;
    return true;
}

int fail(int status, const std::string &msg)
{
    rt::set_thread_error(msg);
    return status;
}

// Warp-per-ray kernel when the rays fill 3/4 of the cells its lanes hold, else an 8-cell tile.
rt::Shape pick_shape(int precision, int nr)
{
    rt::Shape s[32];
    if (precision != RT_FP64) {
        const int n = rt::ray_shapes(precision, nr, s, 32);
        int bi = -1;
        for (int i = 0; i < n; ++i)
            if (4 * nr >= 3 * rt::ray_cells_held(s[i].cells_per_lane, nr) &&
                (bi < 0 || s[i].cells_per_lane < s[bi].cells_per_lane))
                bi = i;
        if (bi >= 0) return s[bi];
    }
    const int n = rt::trace_shapes(precision, s, 32);
    for (int i = 0; i < n; ++i)
        if (s[i].cells_per_lane == 8 && s[i].warps == 4) return s[i];
    return s[0];
}

}  // namespace

extern "C" int rt_irradiate_static(const rt_grid_desc *g, double t_star, double r_star, int n_nu,
                                   const double *nu_mid, const double *kappa, double t_sub,
                                   int kappa_bf16, const float *rho, const float *t_dust,
                                   float *q_abs, float *a_rad, rt_energy *energy, void *cuda_stream)
{
    // arguments: the same rules as rt_create / rt_set_opacity_table / rt_set_star
    if (!g || !g->r_if || !g->theta_if || !g->phi_if || g->nr < 1 || g->ntheta < 1 || g->nphi < 1)
        return fail(RT_ERR_INVALID_ARG, "grid sizes must be >= 1 and interface arrays non-NULL");
    if (g->precision != RT_FP32_KAHAN && g->precision != RT_FP32_PLAIN && g->precision != RT_FP64)
        return fail(RT_ERR_INVALID_ARG, "unknown precision");
    const long long nrays = (long long)g->ntheta * g->nphi;
    if (g->nr > kStaticMaxNr || g->ntheta > kStaticMaxTheta || g->nphi > kStaticMaxPhi || nrays > kStaticMaxRays)
        return fail(RT_ERR_INVALID_ARG,
                    "grid exceeds the static scratch: nr <= " + std::to_string(kStaticMaxNr) +
                        ", ntheta <= " + std::to_string(kStaticMaxTheta) + ", nphi <= " +
                        std::to_string(kStaticMaxPhi) + ", ntheta*nphi <= " + std::to_string(kStaticMaxRays) +
                        " (use rt_create/rt_irradiate for larger grids)");
    if (!increasing_finite(g->r_if, g->nr + 1) || !(g->r_if[0] > 0.0))
        return fail(RT_ERR_INVALID_ARG, "r_if must be finite, > 0 and strictly increasing");
    if (!increasing_finite(g->theta_if, g->ntheta + 1) || g->theta_if[0] < 0.0 ||
        g->theta_if[g->ntheta] > 3.14159265358979323846 * (1 + 1e-15))
        return fail(RT_ERR_INVALID_ARG, "theta_if must be strictly increasing within [0, pi]");
    if (!increasing_finite(g->phi_if, g->nphi + 1))
        return fail(RT_ERR_INVALID_ARG, "phi_if must be strictly increasing");
    if (n_nu < 1 || n_nu > RT_MAX_NU || !nu_mid || !kappa)
        return fail(RT_ERR_INVALID_ARG, "n_nu must be in 1..128 with non-NULL arrays");
    if (!increasing_finite(nu_mid, n_nu) || !(nu_mid[0] > 0.0))
        return fail(RT_ERR_INVALID_ARG, "nu_mid must be finite, > 0 and strictly increasing");
    for (int i = 0; i < n_nu; ++i)
        if (!(kappa[i] >= 0.0) || !isfinite(kappa[i])) return fail(RT_ERR_INVALID_ARG, "kappa must be finite and >= 0");
    if (isnan(t_sub)) return fail(RT_ERR_INVALID_ARG, "t_sub is NaN");
    if (!(t_star > 0.0) || !(r_star > 0.0) || !isfinite(t_star) || !isfinite(r_star))
        return fail(RT_ERR_INVALID_ARG, "t_star and r_star must be finite and > 0");
    if (!rho || !t_dust || !q_abs || !a_rad) return fail(RT_ERR_INVALID_ARG, "NULL field pointer");

    std::string err;
    StaticScratch *s = nullptr;
    int st = scratch_address(&s, err);
    if (st != RT_OK) return fail(st, err);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm > 256)
        return fail(RT_ERR_CUDA, "device not supported by the static scratch (more than 256 SMs)");

    cudaStream_t stream = (cudaStream_t)cuda_stream;
#define RT_SCK(call)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return fail(RT_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

    // problem description into the scratch; the validity word starts at zero
    RT_SCK(cudaMemcpyAsync(s->r_if, g->r_if, sizeof(double) * (g->nr + 1), cudaMemcpyHostToDevice, stream));
    RT_SCK(cudaMemcpyAsync(s->theta_if, g->theta_if, sizeof(double) * (g->ntheta + 1), cudaMemcpyHostToDevice, stream));
    RT_SCK(cudaMemcpyAsync(s->phi_if, g->phi_if, sizeof(double) * (g->nphi + 1), cudaMemcpyHostToDevice, stream));
    RT_SCK(cudaMemcpyAsync(s->nu_mid, nu_mid, sizeof(double) * n_nu, cudaMemcpyHostToDevice, stream));
    RT_SCK(cudaMemcpyAsync(s->kappa, kappa, sizeof(double) * n_nu, cudaMemcpyHostToDevice, stream));
    RT_SCK(cudaMemsetAsync(&s->bad, 0, sizeof(unsigned), stream));

    // bin fluxes (Eq. 20) and geometry tables, as rt_set_star / rt_set_opacity_table do
    RT_SCK(rt::launch_setup_bins(n_nu, s->nu_mid, s->kappa, t_star, r_star, kappa_bf16 ? 1 : 0, s->f_bin,
                                 s->nu_tab, s->kap, s->nu64, &s->sc, stream));
    RT_SCK(rt::launch_setup_geometry(g->nr, g->ntheta, g->nphi, s->r_if, s->theta_if, s->phi_if, t_star, s->rtab,
                                     s->rtab64, s->domega, s->domega32, &s->sc, stream));
    rt::DevScalars sc;
    RT_SCK(cudaMemcpyAsync(&sc, &s->sc, sizeof(sc), cudaMemcpyDeviceToHost, stream));
    RT_SCK(cudaStreamSynchronize(stream));

    // the tracer (one launch: the limits keep nrays (nr + 1) below the 31-bit range)
    const rt::Shape shape = pick_shape(g->precision, g->nr);
    rt::TraceArgs args;
    args.rho = rho;
    args.tdust = t_dust;
    args.q = q_abs;
    args.a = a_rad;
    args.nu = s->nu_tab;
    args.kap = s->kap;
    args.nu64 = s->nu64;
    args.rtab = s->rtab;
    args.rtab64 = s->rtab64;
    args.domega = s->domega;
    args.domega32 = s->domega32;
    args.partials = s->partials;
    args.bad_input = &s->bad;
    args.seq = 1u;
    args.L = (unsigned)(nrays * (g->nr + 1));
    args.nrays = (unsigned)nrays;
    args.r1div = rt::FastDiv::make((unsigned)g->nr + 1u);
    args.nr = g->nr;
    args.nnu_pad = sc.nnu_pad;
    args.n_active = sc.n_active;
    args.t_sub = (float)t_sub;
    args.lut = nullptr;
    args.lut_kref = 0.0f;
    args.lut_fallback = nullptr;
    args.tw_t = nullptr;
    args.tw_b = nullptr;
    args.n_tw = 0;
    const long long T = rt::trace_tile_cells(shape);
    const unsigned ntiles = (unsigned)((nrays * (g->nr + 1) + T - 1) / T);
    unsigned grid = 0;
    // the grid is capped before the launch: one energy partial per CTA, kStaticMaxCtas of them
    RT_SCK(rt::launch_trace(g->precision, shape, args, ntiles, stream, &grid, (unsigned)kStaticMaxCtas));

    if (energy) {
        unsigned bad = 0;
        RT_SCK(rt::launch_energy_reduce(s->partials, grid, &s->sc, &s->energy, stream));
        RT_SCK(cudaMemcpyAsync(energy, &s->energy, sizeof(rt_energy), cudaMemcpyDeviceToHost, stream));
        RT_SCK(cudaMemcpyAsync(&bad, &s->bad, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
        RT_SCK(cudaStreamSynchronize(stream));
        if (bad == 1u)
            return fail(RT_ERR_NONFINITE_INPUT, "input field holds NaN/Inf/negative density or NaN temperature");
    }
#undef RT_SCK
    return RT_OK;
}
