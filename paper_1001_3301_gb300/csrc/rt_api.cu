// C ABI of the irradiation ray tracer: contexts, configuration, launches.
// Host code here validates arguments, owns device memory and enqueues kernels;
// every step of the computation runs in the kernels of rt_setup.cu / rt_trace.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "rt_internal.cuh"

using rt::DevScalars;
using rt::RadRow64;
using rt::NuEntry;
using rt::Shape;

struct rt_ctx {
    int dev = 0;
    int nr = 0, ntheta = 0, nphi = 0, precision = RT_FP32_KAHAN;
    long long nrays = 0, ncells = 0, L = 0;
    cudaStream_t stream = nullptr;

    // geometry (device, and host copies of the axes)
    double *r_if = nullptr, *theta_if = nullptr, *phi_if = nullptr;
    std::vector<double> r_if_h, theta_if_h, phi_if_h;
    float4 *rtab = nullptr;
    RadRow64 *rtab64 = nullptr;
    double *domega = nullptr;
    float *domega32 = nullptr;
    // bins (device)
    double *nu_mid = nullptr, *kappa = nullptr, *f_bin = nullptr;
    NuEntry *nu_tab = nullptr;
    float *kap = nullptr;
    double2 *nu64 = nullptr;
    DevScalars *sc = nullptr;
    // per-call scratch (device)
    double2 *partials = nullptr;
    long long partials_cap = 0;
    unsigned *bad = nullptr;
    rt_energy *energy_d = nullptr;
    // pinned host mirrors
    rt_energy *energy_h = nullptr;
    unsigned *bad_h = nullptr;
    // device staging for the host-buffer entry point, and its copy pipeline
    float *h_rho = nullptr, *h_t = nullptr, *h_q = nullptr, *h_a = nullptr;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[8] = {}, ev_done[8] = {}, ev_start = nullptr;  // kHostChunks entries
    cudaEvent_t ev_out = nullptr;  // the last host call's copies out are done
    bool host_pending = false;     // an asynchronous host call has not been waited for

    // host copies of the table as the tracer uses it, and its fingerprint
    std::vector<double> nu_h, kappa_h;
    // temperature-dependent table (rt_set_opacity_table_t): grid, rows, sorted pairs
    int n_t = 0;
    std::vector<double> tgrid_h, kappa_t_h;
    double *kappa_t_d = nullptr;
    float *tg32 = nullptr;
    float2 *kt2 = nullptr;
    // a table that separates, kappa_i(T) = kappa_i b(T): the one-column tracer with the
    // column weight b(T) (grid padded with +Inf; (b_j, slope to the next point))
    bool tw_sep = false;
    float *tw_t_d = nullptr;
    float4 *tw_b_d = nullptr;
    // a table of low rank rk (2-4), kappa_i(T_j) = sum_r A_ir B_rj: the rk-column kernel
    // of rt_tdep2.cu (A in FP64 per bin, 4 wide; the sorted -A log2 e per bin; B per
    // grid point); 0: none found
    int rk = 0;
    double *fac_a_d = nullptr;
    float4 *r2_ab = nullptr, *r2_bw = nullptr;
    // lookup-table comparator (rt_lut.cu): table, reference opacity, tolerance and the
    // table fingerprint it was built for; per-call count of warp-slots that fell back
    float2 *lut = nullptr;
    unsigned *lut_count = nullptr;
    double lut_kref = 0.0;
    float lut_tol = -1.0f;
    unsigned long long lut_fp = 0;
    bool lut_on = false;  // rt_irradiate_lut is tracing
    int *order_d = nullptr;
    unsigned long long fingerprint = 0;
    // learned surrogate (rt_surrogate.cu), created by rt_surrogate_train / _load
    rt::SurState *sur = nullptr;
    // Planck-mean table of the dust-temperature update (rt_temperature.cu)
    float *temp_lkp = nullptr;
    unsigned long long temp_fp = 0;
    // workspace of the flux-limited-diffusion step (rt_fld.cu)
    rt::FldState *fld = nullptr;

    // configuration state
    int n_nu = 0, kappa_bf16 = 0;
    bool have_table = false, have_star = false, configured = false;
    double t_sub = 0.0, t_star = 0.0, r_star = 0.0;
    DevScalars sc_h{};
    Shape shape{0, 0, 0, 0};
    bool shape_forced = false;
    unsigned seq = 0;
    long long last_ntiles = 0;
    bool traced = false;
    std::string err;
};

namespace {

thread_local std::string g_create_err;

constexpr int kHostChunks = 8;  // most ray chunks of the host-buffer pipeline
static_assert(sizeof(rt_ctx::ev_in) / sizeof(cudaEvent_t) == kHostChunks, "one event pair per chunk");

int fail(rt_ctx *ctx, int status, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    else g_create_err = msg;
    return status;
}

int cuda_fail(rt_ctx *ctx, const char *what, cudaError_t e)
{
    return fail(ctx, RT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RT_CK(ctx, call)                                      \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, #call, e_); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1));
}

bool increasing(const double *a, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(a[i]) || (i > 0 && !(a[i] > a[i - 1]))) return false;
    return true;
}

// shape choice cache across contexts: (precision, nr, nrays, nnu_pad, table kind) -> shape
std::mutex g_tune_mu;
std::map<std::tuple<int, int, long long, int, int>, Shape> g_tune_cache;

long long total_tiles(const rt_ctx *c, Shape s);

// A separable kappa(nu, T) table goes through the one-column ray kernel with the
// column weight b(T) where that kernel holds the rays (FP32 modes); other
// temperature-dependent tables through the per-bin kernel of rt_tdep.cu.
bool use_tw(const rt_ctx *c)
{
    if (c->n_t <= 0 || !c->tw_sep || c->precision == RT_FP64) return false;
    Shape s[16];
    return rt::ray_shapes_tw(c->precision, c->nr, s, 16) > 0;
}

// A table of low rank goes through the rk-column kernel of rt_tdep2.cu (FP32 modes).
bool use_r2(const rt_ctx *c)
{
    if (c->n_t <= 0 || c->rk < 2 || use_tw(c) || c->precision == RT_FP64) return false;
    Shape s[16];
    return rt::tdep2_shapes(c->rk, c->nr, s, 16) > 0;
}

int table_kind(const rt_ctx *c)
{
    if (c->n_t <= 0) return RT_TABLE_NU;
    if (use_tw(c)) return RT_TABLE_NU_T_SEPARABLE;
    if (!use_r2(c)) return RT_TABLE_NU_T;
    return c->rk == 2 ? RT_TABLE_NU_T_RANK2 : RT_TABLE_NU_T_LOW_RANK;
}

// every compiled shape that applies to this context: tile shapes, then ray shapes
int all_shapes(const rt_ctx *c, Shape *out, int max_out)
{
    if (c->n_t > 0) return use_tw(c) ? rt::ray_shapes_tw(c->precision, c->nr, out, max_out)
                                     : use_r2(c) ? rt::tdep2_shapes(c->rk, c->nr, out, max_out)
                                                 : rt::tdep_shapes(c->nr, out, max_out);
    int n = rt::trace_shapes(c->precision, out, max_out);
    if (c->precision != RT_FP64) {
        n += rt::ray_shapes(c->precision, c->nr, out + n, max_out - n);
        n += rt::ray_shapes_mc(c->precision, c->nr, out + n, max_out - n);
    }
    return n;
}

Shape default_shape(const rt_ctx *c)
{
    const bool tw = use_tw(c);
    if (c->n_t > 0 && !tw) {  // temperature-dependent table: the fewest cells per lane that hold a ray
        Shape ts[16];
        const int n = use_r2(c) ? rt::tdep2_shapes(c->rk, c->nr, ts, 16) : rt::tdep_shapes(c->nr, ts, 16);
        int bi = -1;
        for (int i = 0; i < n; ++i)
            if (bi < 0 || ts[i].cells_per_lane < ts[bi].cells_per_lane ||
                (ts[i].cells_per_lane == ts[bi].cells_per_lane && ts[i].min_blocks > ts[bi].min_blocks))
                bi = i;
        return bi >= 0 ? ts[bi] : Shape{rt::kKindRay, 0, 0, 0};
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(std::make_tuple(c->precision, c->nr, c->nrays, c->sc_h.nnu_pad, table_kind(c)));
        if (it != g_tune_cache.end()) return it->second;
    }
    // Prefer the warp-per-ray kernel with the fewest cells per lane when the rays
    // fill at least 3/4 of the G C cells of their lane segment; else the widest tile
    // that still gives every SM several tiles.
    if (c->precision != RT_FP64) {
        Shape rs[32];
        const int nrs = tw ? rt::ray_shapes_tw(c->precision, c->nr, rs, 32) : rt::ray_shapes(c->precision, c->nr, rs, 32);
        int bi = -1;
        for (int i = 0; i < nrs; ++i)
            if (4 * c->nr >= 3 * rt::ray_cells_held(rs[i].cells_per_lane, c->nr) &&
                (bi < 0 || rs[i].cells_per_lane < rs[bi].cells_per_lane))
                bi = i;
        if (bi >= 0) return rs[bi];
    }
    Shape cand[32];
    const int n = rt::trace_shapes(c->precision, cand, 32);
    Shape best = cand[0];
    long long best_t = 0;
    for (int i = 0; i < n; ++i) {
        const long long tiles = total_tiles(c, cand[i]);
        const long long tc = rt::trace_tile_cells(cand[i]);
        if (tiles >= 8LL * 152) {
            if (tc > best_t) { best = cand[i]; best_t = tc; }
        }
    }
    if (best_t == 0) {  // small grid: most tiles wins, then the smaller tile
        long long most = -1;
        for (int i = 0; i < n; ++i) {
            const long long tiles = total_tiles(c, cand[i]);
            if (tiles > most) { most = tiles; best = cand[i]; }
        }
    }
    return best;
}

int finalize(rt_ctx *c)
{
    c->configured = false;
    if (!(c->have_table && c->have_star)) return RT_OK;
    cudaError_t e = rt::launch_setup_bins(c->n_nu, c->nu_mid, c->kappa, c->t_star, c->r_star,
                                          c->kappa_bf16, c->f_bin, c->nu_tab, c->kap, c->nu64,
                                          c->sc, c->stream, c->order_d);
    if (e != cudaSuccess) return cuda_fail(c, "setup_bins", e);
    e = rt::launch_setup_geometry(c->nr, c->ntheta, c->nphi, c->r_if, c->theta_if, c->phi_if,
                                  c->t_star, c->rtab, c->rtab64, c->domega, c->domega32, c->sc,
                                  c->stream);
    if (e != cudaSuccess) return cuda_fail(c, "setup_geometry", e);
    RT_CK(c, cudaMemcpyAsync(&c->sc_h, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    RT_CK(c, cudaStreamSynchronize(c->stream));
    if (c->n_t > 0) {
        e = rt::launch_build_tdep(c->sc_h.n_active, c->sc_h.nnu_pad, c->n_t, c->kappa_t_d, c->order_d, c->kt2,
                                  c->stream);
        if (e != cudaSuccess) return cuda_fail(c, "build temperature table", e);
        if (c->rk >= 2) {
            e = rt::launch_build_rank2(c->sc_h.n_active, c->sc_h.nnu_pad, c->fac_a_d, c->order_d, c->r2_ab,
                                       c->stream);
            if (e != cudaSuccess) return cuda_fail(c, "build rank-two table", e);
        }
        RT_CK(c, cudaStreamSynchronize(c->stream));
    }
    if (!c->shape_forced) c->shape = default_shape(c);
    // FNV-1a over what fixes the per-cell absorption function of (N_in, dN)
    unsigned long long h = 1469598103934665603ULL;
    auto mix = [&h](const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ULL;
    };
    mix(&c->n_nu, sizeof(int));
    mix(c->nu_h.data(), sizeof(double) * c->nu_h.size());
    mix(c->kappa_h.data(), sizeof(double) * c->kappa_h.size());
    mix(&c->t_sub, sizeof(double));
    mix(&c->t_star, sizeof(double));
    mix(&c->n_t, sizeof(int));
    mix(c->tgrid_h.data(), sizeof(double) * c->tgrid_h.size());
    mix(c->kappa_t_h.data(), sizeof(double) * c->kappa_t_h.size());
    c->fingerprint = h;
    c->configured = true;
    return RT_OK;
}

int ensure_partials(rt_ctx *c, long long ntiles)
{
    if (ntiles <= c->partials_cap) return RT_OK;
    if (c->partials) cudaFree(c->partials);
    c->partials = nullptr;
    c->partials_cap = 0;
    if (dalloc(&c->partials, (size_t)ntiles) != cudaSuccess)
        return fail(c, RT_ERR_NO_MEMORY, "cannot allocate energy partials");
    c->partials_cap = ntiles;
    return RT_OK;
}

// Number of tiles of one grid; rays are launched in chunks of at most
// kMaxLaunchCells flattened cells (32-bit indexing inside the kernel).
long long chunk_rays(const rt_ctx *c) { return rt::kMaxLaunchCells / (c->nr + 1); }

// an upper bound of the CTAs of one launch of shape s over nr_c rays
long long launch_ctas(const rt_ctx *c, Shape s, long long nr_c)
{
    if (s.kind == rt::kKindRay)
        return (nr_c * rt::ray_warps_per_ray(s.cells_per_lane, c->nr) + s.warps - 1) / s.warps;
    if (s.kind == rt::kKindRayChunked) return (nr_c + 4LL * s.warps - 1) / (4LL * s.warps);
    const long long T = rt::trace_tile_cells(s);
    return (nr_c * (c->nr + 1) + T - 1) / T;
}

long long total_tiles(const rt_ctx *c, Shape s)
{
    const long long cr = chunk_rays(c);
    long long tiles = 0;
    for (long long r0 = 0; r0 < c->nrays; r0 += cr) {
        const long long nr_c = (c->nrays - r0 < cr) ? c->nrays - r0 : cr;
        tiles += launch_ctas(c, s, nr_c);
    }
    return tiles;
}

// Launches the tracer on rays [r_begin, r_end) of the context's fields (pointers to
// the whole grid) on `stream`; the CTAs' energy partials go to c->partials from
// *npart on, which advances. The caller has sized c->partials and set c->seq.
int trace_range(rt_ctx *c, const float *rho, const float *td, float *q, float *a, Shape s, long long r_begin,
                long long r_end, cudaStream_t stream, long long *npart)
{
    rt::TraceArgs args;
    args.nu = c->nu_tab;
    args.kap = c->kap;
    args.nu64 = c->nu64;
    args.rtab = c->rtab;
    args.rtab64 = c->rtab64;
    args.bad_input = c->bad;
    args.seq = c->seq;
    args.r1div = rt::FastDiv::make((unsigned)c->nr + 1u);
    args.nr = c->nr;
    args.nnu_pad = c->sc_h.nnu_pad;
    args.n_active = c->sc_h.n_active;
    args.t_sub = (float)c->t_sub;
    const bool tw = use_tw(c);
    args.lut = c->lut_on ? c->lut : nullptr;
    args.lut_kref = (float)c->lut_kref;
    args.lut_fallback = c->lut_on ? c->lut_count : nullptr;
    args.tw_t = tw ? c->tw_t_d : nullptr;
    args.tw_b = tw ? c->tw_b_d : nullptr;
    args.n_tw = tw ? c->n_t : 0;
    const long long T = rt::trace_tile_cells(s), cr = chunk_rays(c);
    for (long long r0 = r_begin; r0 < r_end; r0 += cr) {
        const long long nr_c = (r_end - r0 < cr) ? r_end - r0 : cr;
        const size_t off = (size_t)r0 * c->nr;
        args.rho = rho + off;
        args.tdust = td + off;
        args.q = q + off;
        args.a = a + off;
        args.domega = c->domega + r0;
        args.domega32 = c->domega32 + r0;
        args.partials = c->partials + *npart;
        args.L = (unsigned)(nr_c * (c->nr + 1));
        args.nrays = (unsigned)nr_c;
        const long long nt = (nr_c * (c->nr + 1) + T - 1) / T;
        unsigned grid = 0;
        cudaError_t e;
        if (c->n_t > 0 && !tw)
            e = use_r2(c) ? rt::launch_tdep2(c->rk, s, args, c->r2_ab, c->r2_bw, c->tg32, c->n_t, stream, &grid)
                          : rt::launch_tdep(s, args, c->kt2, c->tg32, c->n_t, stream, &grid);
        else
            e = rt::launch_trace(c->precision, s, args, (unsigned)nt, stream, &grid);
        if (e != cudaSuccess) return cuda_fail(c, "trace kernel launch", e);
        *npart += grid;
    }
    return RT_OK;
}

// tiles (an upper bound of the CTAs) of the launches over rays [r_begin, r_end)
long long range_tiles(const rt_ctx *c, Shape s, long long r_begin, long long r_end)
{
    const long long cr = chunk_rays(c);
    long long tiles = 0;
    for (long long r0 = r_begin; r0 < r_end; r0 += cr) {
        const long long nr_c = (r_end - r0 < cr) ? r_end - r0 : cr;
        tiles += launch_ctas(c, s, nr_c);
    }
    return tiles;
}

int trace(rt_ctx *c, const float *rho, const float *td, float *q, float *a, Shape s)
{
    // at most one persistent CTA per tile per chunk
    int st = ensure_partials(c, total_tiles(c, s));
    if (st != RT_OK) return st;
    ++c->seq;
    long long npart = 0;
    st = trace_range(c, rho, td, q, a, s, 0, c->nrays, c->stream, &npart);
    if (st != RT_OK) return st;
    c->last_ntiles = npart;
    c->traced = true;
    return RT_OK;
}

int read_energy(rt_ctx *c, rt_energy *out)
{
    cudaError_t e = rt::launch_energy_reduce(c->partials, c->last_ntiles, c->sc, c->energy_d, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, "energy reduce", e);
    RT_CK(c, cudaMemcpyAsync(c->energy_h, c->energy_d, sizeof(rt_energy), cudaMemcpyDeviceToHost, c->stream));
    RT_CK(c, cudaMemcpyAsync(c->bad_h, c->bad, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    RT_CK(c, cudaStreamSynchronize(c->stream));
    *out = *c->energy_h;
    if (*c->bad_h == c->seq) return fail(c, RT_ERR_NONFINITE_INPUT, "input field holds NaN/Inf/negative density or NaN temperature");
    return RT_OK;
}

int check_call(rt_ctx *c, const void *rho, const void *td, const void *q, const void *a)
{
    if (!c) return RT_ERR_INVALID_ARG;
    if (!rho || !td || !q || !a) return fail(c, RT_ERR_INVALID_ARG, "NULL field pointer");
    if (!c->configured) return fail(c, RT_ERR_NOT_CONFIGURED, "call rt_set_star and rt_set_opacity_table first");
    if (c->n_t > 0 && c->shape.cells_per_lane == 0)
        return fail(c, RT_ERR_INVALID_ARG, "temperature-dependent opacity tables need nr <= 1024");
    cudaError_t e = cudaSetDevice(c->dev);
    if (e != cudaSuccess) return cuda_fail(c, "cudaSetDevice", e);
    return RT_OK;
}

void free_all(rt_ctx *c)
{
    void *ptrs[] = {c->r_if, c->theta_if, c->phi_if, c->rtab, c->rtab64, c->domega, c->domega32, c->nu_mid,
                    c->kappa, c->f_bin, c->nu_tab, c->kap, c->nu64, c->sc, c->partials, c->bad,
                    c->energy_d, c->h_rho, c->h_t, c->h_q, c->h_a, c->temp_lkp, c->kappa_t_d,
                    c->tg32, c->kt2, c->order_d, c->tw_t_d, c->tw_b_d, c->fac_a_d, c->r2_ab, c->r2_bw,
                    c->lut, c->lut_count};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->energy_h) cudaFreeHost(c->energy_h);
    if (c->bad_h) cudaFreeHost(c->bad_h);
}

}  // namespace

namespace rt {
// failure text of context-less calls, reported by rt_last_error(NULL)
void set_thread_error(const std::string &msg) { g_create_err = msg; }

// The device tables of a configured context, for the batch launcher (rt_batch.cu):
// a TraceArgs with every table pointer and size set (field pointers, partials and
// validity word left for the caller), its scalars, and identity.
bool ctx_view(const rt_ctx *c, CtxView *v)
{
    if (!c || !c->configured) return false;
    TraceArgs a{};
    a.nu = c->nu_tab;
    a.kap = c->kap;
    a.nu64 = c->nu64;
    a.rtab = c->rtab;
    a.rtab64 = c->rtab64;
    a.domega = c->domega;
    a.domega32 = c->domega32;
    a.L = (unsigned)((c->L < kMaxLaunchCells) ? c->L : 0);
    a.nrays = (unsigned)c->nrays;
    a.r1div = FastDiv::make((unsigned)c->nr + 1u);
    a.nr = c->nr;
    a.nnu_pad = c->sc_h.nnu_pad;
    a.n_active = c->sc_h.n_active;
    a.t_sub = (float)c->t_sub;
    v->args = a;
    v->sc = c->sc;
    v->precision = c->precision;
    v->dev = c->dev;
    v->flat_cells = c->L;
    v->ncells = c->ncells;
    v->tdep = c->n_t > 0;
    return true;
}

bool ctx_info(const rt_ctx *c, CtxInfo *o)
{
    if (!c) return false;
    o->dev = c->dev;
    o->stream = c->stream;
    o->configured = c->configured;
    o->nr = c->nr;
    o->ntheta = c->ntheta;
    o->nphi = c->nphi;
    o->r_if_h = c->r_if_h.data();
    o->theta_if_h = c->theta_if_h.data();
    o->phi_if_h = c->phi_if_h.data();
    o->nrays = c->nrays;
    o->ncells = c->ncells;
    o->t_sub = c->t_sub;
    o->t_star = c->t_star;
    o->r_star = c->r_star;
    o->n_nu = c->n_nu;
    o->nu_h = c->nu_h.data();
    o->kappa_h = c->kappa_h.data();
    o->table_fingerprint = c->fingerprint;
    o->n_t = c->n_t;
    o->t_grid_h = c->tgrid_h.data();
    o->kappa_t_h = c->kappa_t_h.data();
    o->rtab = c->rtab;
    o->domega32 = c->domega32;
    o->nu_tab = c->nu_tab;
    o->kap = c->kap;
    o->sc = c->sc_h;
    return true;
}

SurState *&ctx_surrogate(rt_ctx *c) { return c->sur; }
float *&ctx_temp_table(rt_ctx *c) { return c->temp_lkp; }
unsigned long long &ctx_temp_fingerprint(rt_ctx *c) { return c->temp_fp; }
FldState *&ctx_fld(rt_ctx *c) { return c->fld; }

int ctx_fail(rt_ctx *c, int status, const std::string &msg) { return fail(c, status, msg); }
}  // namespace rt

extern "C" {

int rt_create(const rt_grid_desc *g, void *cuda_stream, rt_ctx **out)
{
    if (!out) return fail(nullptr, RT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!g || g->nr < 1 || g->ntheta < 1 || g->nphi < 1 || !g->r_if || !g->theta_if || !g->phi_if)
        return fail(nullptr, RT_ERR_INVALID_ARG, "grid sizes must be >= 1 and interface arrays non-NULL");
    if (g->precision != RT_FP32_KAHAN && g->precision != RT_FP32_PLAIN && g->precision != RT_FP64)
        return fail(nullptr, RT_ERR_INVALID_ARG, "unknown precision");
    if (!increasing(g->r_if, g->nr + 1) || !(g->r_if[0] > 0.0))
        return fail(nullptr, RT_ERR_INVALID_ARG, "r_if must be finite, > 0 and strictly increasing");
    if (!increasing(g->theta_if, g->ntheta + 1) || g->theta_if[0] < 0.0 ||
        g->theta_if[g->ntheta] > 3.14159265358979323846 * (1 + 1e-15))
        return fail(nullptr, RT_ERR_INVALID_ARG, "theta_if must be strictly increasing within [0, pi]");
    if (!increasing(g->phi_if, g->nphi + 1))
        return fail(nullptr, RT_ERR_INVALID_ARG, "phi_if must be strictly increasing");
    const long long nrays = (long long)g->ntheta * g->nphi;
    const long long ncells = nrays * g->nr;
    if (ncells > (1LL << 40) || g->nr > (1 << 24))
        return fail(nullptr, RT_ERR_INVALID_ARG, "grid too large");

    rt_ctx *c = new (std::nothrow) rt_ctx();
    if (!c) return fail(nullptr, RT_ERR_NO_MEMORY, "out of host memory");
    c->nr = g->nr;
    c->ntheta = g->ntheta;
    c->nphi = g->nphi;
    c->r_if_h.assign(g->r_if, g->r_if + g->nr + 1);
    c->theta_if_h.assign(g->theta_if, g->theta_if + g->ntheta + 1);
    c->phi_if_h.assign(g->phi_if, g->phi_if + g->nphi + 1);
    c->precision = g->precision;
    c->nrays = nrays;
    c->ncells = ncells;
    c->L = nrays * (g->nr + 1);
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&c->dev);
    bool ok = e == cudaSuccess;
    ok = ok && dalloc(&c->r_if, g->nr + 1) == cudaSuccess;
    ok = ok && dalloc(&c->theta_if, g->ntheta + 1) == cudaSuccess;
    ok = ok && dalloc(&c->phi_if, g->nphi + 1) == cudaSuccess;
    ok = ok && dalloc(&c->rtab, g->nr) == cudaSuccess;
    ok = ok && dalloc(&c->rtab64, g->nr) == cudaSuccess;
    ok = ok && dalloc(&c->domega, (size_t)nrays) == cudaSuccess;
    ok = ok && dalloc(&c->domega32, (size_t)nrays) == cudaSuccess;
    ok = ok && dalloc(&c->nu_mid, RT_MAX_NU) == cudaSuccess;
    ok = ok && dalloc(&c->kappa, RT_MAX_NU) == cudaSuccess;
    ok = ok && dalloc(&c->f_bin, RT_MAX_NU) == cudaSuccess;
    ok = ok && dalloc(&c->nu_tab, RT_MAX_NU + rt::kNuPad) == cudaSuccess;
    ok = ok && dalloc(&c->kap, rt::kKapBuffer) == cudaSuccess;
    ok = ok && dalloc(&c->nu64, RT_MAX_NU + rt::kNuPad) == cudaSuccess;
    ok = ok && dalloc(&c->sc, 1) == cudaSuccess;
    ok = ok && dalloc(&c->order_d, RT_MAX_NU) == cudaSuccess;
    ok = ok && dalloc(&c->bad, 1) == cudaSuccess;
    ok = ok && dalloc(&c->energy_d, 1) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&c->energy_h, sizeof(rt_energy)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&c->bad_h, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        free_all(c);
        delete c;
        cudaGetLastError();
        return fail(nullptr, RT_ERR_CUDA, "device allocation failed in rt_create");
    }
    ok = cudaMemcpyAsync(c->r_if, g->r_if, sizeof(double) * (g->nr + 1), cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(c->theta_if, g->theta_if, sizeof(double) * (g->ntheta + 1), cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(c->phi_if, g->phi_if, sizeof(double) * (g->nphi + 1), cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->bad, 0, sizeof(unsigned), c->stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(c->stream) == cudaSuccess;
    if (!ok) {
        free_all(c);
        delete c;
        return fail(nullptr, RT_ERR_CUDA, std::string("copy in rt_create: ") + cudaGetErrorString(cudaGetLastError()));
    }
    *out = c;
    return RT_OK;
}

int rt_set_stream(rt_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return RT_OK;
}

int rt_set_opacity_table(rt_ctx *ctx, int n_nu, const double *nu_mid, const double *kappa,
                         double t_sub, int kappa_bf16)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (n_nu < 1 || n_nu > RT_MAX_NU || !nu_mid || !kappa)
        return fail(ctx, RT_ERR_INVALID_ARG, "n_nu must be in 1..128 with non-NULL arrays");
    if (!increasing(nu_mid, n_nu) || !(nu_mid[0] > 0.0))
        return fail(ctx, RT_ERR_INVALID_ARG, "nu_mid must be finite, > 0 and strictly increasing");
    for (int i = 0; i < n_nu; ++i)
        if (!(kappa[i] >= 0.0) || !isfinite(kappa[i]))
            return fail(ctx, RT_ERR_INVALID_ARG, "kappa must be finite and >= 0");
    if (isnan(t_sub)) return fail(ctx, RT_ERR_INVALID_ARG, "t_sub is NaN");
    RT_CK(ctx, cudaSetDevice(ctx->dev));
    RT_CK(ctx, cudaMemcpyAsync(ctx->nu_mid, nu_mid, sizeof(double) * n_nu, cudaMemcpyHostToDevice, ctx->stream));
    RT_CK(ctx, cudaMemcpyAsync(ctx->kappa, kappa, sizeof(double) * n_nu, cudaMemcpyHostToDevice, ctx->stream));
    ctx->n_nu = n_nu;
    ctx->t_sub = t_sub;
    ctx->kappa_bf16 = kappa_bf16 ? 1 : 0;
    ctx->n_t = 0;
    ctx->tw_sep = false;
    ctx->rk = 0;
    ctx->tgrid_h.clear();
    ctx->kappa_t_h.clear();
    ctx->nu_h.assign(nu_mid, nu_mid + n_nu);
    ctx->kappa_h.assign(kappa, kappa + n_nu);
    if (ctx->kappa_bf16)  // the tracer's table: kappa rounded to BF16 (nearest, ties to even)
        for (double &k : ctx->kappa_h) {
            float f = (float)k;
            unsigned u;
            memcpy(&u, &f, 4);
            u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
            memcpy(&f, &u, 4);
            k = f;
        }
    ctx->have_table = true;
    return finalize(ctx);
}

namespace {

// Is the table [n_nu][n_t] of rank two with non-negative factors? In the plane of its
// columns every column is a non-negative vector, so all of them lie in the cone of the
// two columns with the smallest and the largest angle, and each column is a
// non-negative combination of those two:
//   kappa[i][j] = a[i][0] b[0][j] + a[i][1] b[1][j],  a = the two columns.
// The plane: u along the longest column, v along the largest residual orthogonal to
// it. Accepted when every entry is reproduced to 1e-10 of itself (FP64).
bool rank_two(const double *kappa, int n_nu, int n_t, std::vector<double> &a, std::vector<double> &b)
{
    auto col = [&](int i, int j) { return kappa[(size_t)i * n_t + j]; };
    std::vector<double> nrm(n_t, 0.0);
    int j1 = 0;
    for (int j = 0; j < n_t; ++j) {
        for (int i = 0; i < n_nu; ++i) nrm[j] += col(i, j) * col(i, j);
        nrm[j] = std::sqrt(nrm[j]);
        if (nrm[j] > nrm[j1]) j1 = j;
    }
    if (!(nrm[j1] > 0.0)) return false;
    std::vector<double> u(n_nu), v(n_nu, 0.0);
    for (int i = 0; i < n_nu; ++i) u[i] = col(i, j1) / nrm[j1];
    auto dot = [&](const std::vector<double> &w, int j) {
        double d = 0.0;
        for (int i = 0; i < n_nu; ++i) d += w[i] * col(i, j);
        return d;
    };
    int j2 = -1;
    double rmax = 0.0;
    for (int j = 0; j < n_t; ++j) {
        const double pu = dot(u, j);
        double r = 0.0;
        for (int i = 0; i < n_nu; ++i) r += (col(i, j) - pu * u[i]) * (col(i, j) - pu * u[i]);
        if (r > rmax) { rmax = r; j2 = j; }
    }
    if (j2 < 0 || !(std::sqrt(rmax) > 1e-12 * nrm[j1])) return false;  // one direction: not rank two
    const double pu2 = dot(u, j2);
    double vn = 0.0;
    for (int i = 0; i < n_nu; ++i) {
        v[i] = col(i, j2) - pu2 * u[i];
        vn += v[i] * v[i];
    }
    vn = std::sqrt(vn);
    for (int i = 0; i < n_nu; ++i) v[i] /= vn;
    std::vector<double> pu(n_t), pv(n_t);
    int jlo = -1, jhi = -1;
    double tlo = 0.0, thi = 0.0;
    for (int j = 0; j < n_t; ++j) {
        pu[j] = dot(u, j);
        pv[j] = dot(v, j);
        if (!(nrm[j] > 0.0)) continue;
        const double th = std::atan2(pv[j], pu[j]);
        if (jlo < 0 || th < tlo) { jlo = j; tlo = th; }
        if (jhi < 0 || th > thi) { jhi = j; thi = th; }
    }
    const double det = pu[jlo] * pv[jhi] - pu[jhi] * pv[jlo];
    if (jlo == jhi || !(det != 0.0)) return false;
    a.assign((size_t)2 * n_nu, 0.0);
    b.assign((size_t)2 * n_t, 0.0);
    for (int i = 0; i < n_nu; ++i) {
        a[2 * i] = col(i, jlo);
        a[2 * i + 1] = col(i, jhi);
    }
    for (int j = 0; j < n_t; ++j) {
        // (pu, pv)_j = x (pu, pv)_lo + y (pu, pv)_hi; rounding may leave a tiny negative
        const double x = (pu[j] * pv[jhi] - pu[jhi] * pv[j]) / det;
        const double y = (pu[jlo] * pv[j] - pu[j] * pv[jlo]) / det;
        b[j] = std::max(x, 0.0);
        b[n_t + j] = std::max(y, 0.0);
    }
    for (int i = 0; i < n_nu; ++i)
        for (int j = 0; j < n_t; ++j) {
            const double have = col(i, j), want = a[2 * i] * b[j] + a[2 * i + 1] * b[n_t + j];
            if (std::fabs(have - want) > 1e-10 * std::max(std::fabs(have), std::fabs(want))) return false;
        }
    return true;
}

// Is the table [n_nu][n_t] of rank R (3 or 4)? Its leading R right singular vectors v_r
// (one-sided Jacobi on the columns of K, FP64, which keeps the small singular values'
// vectors accurate) give B = V^T and A = K V, so that
//   kappa[i][j] = sum_r a[i][r] b[r][j]  (a: [n_nu][4], b: [4][n_t], unused rows 0).
// The first vector of a non-negative table is non-negative; the others carry either
// sign. Accepted when every entry is reproduced to 1e-10 of its row's largest.
bool low_rank(const double *kappa, int n_nu, int n_t, int R, std::vector<double> &a, std::vector<double> &b)
{
    if (R > n_t) return false;
    std::vector<double> u(kappa, kappa + (size_t)n_nu * n_t), v((size_t)n_t * n_t, 0.0);
    for (int p = 0; p < n_t; ++p) v[(size_t)p * n_t + p] = 1.0;
    auto U = [&](int i, int p) -> double & { return u[(size_t)i * n_t + p]; };
    auto V = [&](int k, int p) -> double & { return v[(size_t)k * n_t + p]; };
    for (int sweep = 0; sweep < 60; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < n_t; ++p)
            for (int q = p + 1; q < n_t; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < n_nu; ++i) {
                    al += U(i, p) * U(i, p);
                    be += U(i, q) * U(i, q);
                    ga += U(i, p) * U(i, q);
                }
                if (!(std::fabs(ga) > 1e-15 * std::sqrt(al * be))) continue;
                rotated = true;
                const double ze = (be - al) / (2.0 * ga);
                const double t = (ze >= 0.0 ? 1.0 : -1.0) / (std::fabs(ze) + std::sqrt(1.0 + ze * ze));
                const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < n_nu; ++i) {
                    const double up = U(i, p), uq = U(i, q);
                    U(i, p) = c * up - sn * uq;
                    U(i, q) = sn * up + c * uq;
                }
                for (int k = 0; k < n_t; ++k) {
                    const double vp = V(k, p), vq = V(k, q);
                    V(k, p) = c * vp - sn * vq;
                    V(k, q) = sn * vp + c * vq;
                }
            }
        if (!rotated) break;
    }
    std::vector<double> sig(n_t, 0.0);
    for (int p = 0; p < n_t; ++p)
        for (int i = 0; i < n_nu; ++i) sig[p] += U(i, p) * U(i, p);
    std::vector<int> idx(n_t);
    for (int p = 0; p < n_t; ++p) idx[p] = p;
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return sig[x] > sig[y]; });
    a.assign((size_t)4 * n_nu, 0.0);
    b.assign((size_t)4 * n_t, 0.0);
    for (int r = 0; r < R; ++r) {
        const int e = idx[r];
        double sum = 0.0;
        for (int k = 0; k < n_t; ++k) sum += V(k, e);
        const double sg = sum < 0.0 ? -1.0 : 1.0;
        for (int k = 0; k < n_t; ++k) b[(size_t)r * n_t + k] = sg * V(k, e);
        for (int i = 0; i < n_nu; ++i) a[(size_t)4 * i + r] = sg * U(i, e);  // (K V)_ie
    }
    for (int i = 0; i < n_nu; ++i) {
        double rowmax = 0.0;
        for (int j = 0; j < n_t; ++j) rowmax = std::max(rowmax, std::fabs(kappa[(size_t)i * n_t + j]));
        for (int j = 0; j < n_t; ++j) {
            double want = 0.0;
            for (int r = 0; r < R; ++r) want += a[(size_t)4 * i + r] * b[(size_t)r * n_t + j];
            if (!(std::fabs(kappa[(size_t)i * n_t + j] - want) <= 1e-10 * rowmax)) return false;
        }
    }
    return true;
}

}  // namespace

int rt_set_opacity_table_t(rt_ctx *ctx, int n_nu, const double *nu_mid, int n_t, const double *t_grid,
                           const double *kappa_t, double t_sub)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (n_nu < 1 || n_nu > RT_MAX_NU || !nu_mid || !kappa_t || !t_grid)
        return fail(ctx, RT_ERR_INVALID_ARG, "n_nu must be in 1..128 with non-NULL arrays");
    if (n_t < 2 || n_t > rt::kMaxTdepPoints) return fail(ctx, RT_ERR_INVALID_ARG, "n_t must be in 2..32");
    if (!increasing(nu_mid, n_nu) || !(nu_mid[0] > 0.0))
        return fail(ctx, RT_ERR_INVALID_ARG, "nu_mid must be finite, > 0 and strictly increasing");
    if (!increasing(t_grid, n_t) || !(t_grid[0] > 0.0))
        return fail(ctx, RT_ERR_INVALID_ARG, "t_grid must be finite, > 0 and strictly increasing");
    for (int i = 0; i < n_nu * n_t; ++i)
        if (!(kappa_t[i] >= 0.0) || !isfinite(kappa_t[i]))
            return fail(ctx, RT_ERR_INVALID_ARG, "kappa_t must be finite and >= 0");
    if (isnan(t_sub)) return fail(ctx, RT_ERR_INVALID_ARG, "t_sub is NaN");
    RT_CK(ctx, cudaSetDevice(ctx->dev));
    if (!ctx->kappa_t_d) {
        bool ok = dalloc(&ctx->kappa_t_d, (size_t)RT_MAX_NU * rt::kMaxTdepPoints) == cudaSuccess &&
                  dalloc(&ctx->tg32, rt::kMaxTdepPoints) == cudaSuccess &&
                  dalloc(&ctx->kt2, (size_t)(RT_MAX_NU + rt::kNuPad) * rt::kMaxTdepPoints) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return fail(ctx, RT_ERR_NO_MEMORY, "cannot allocate the temperature-dependent table");
        }
    }
    // each bin's largest value orders the bins and bounds the absorbed-fraction classes
    std::vector<double> kmax(n_nu, 0.0);
    for (int i = 0; i < n_nu; ++i)
        for (int j = 0; j < n_t; ++j) kmax[i] = std::max(kmax[i], kappa_t[(size_t)i * n_t + j]);
    std::vector<float> tg(t_grid, t_grid + n_t);
    // Does the table separate, kappa_i(T_j) = kmax_i b_j for every entry (to 1e-12)? Then
    // every bin's optical depth is kmax_i times one column weighted by b(T), linear in T
    // between the grid points like the rows themselves.
    int iref = 0;
    for (int i = 1; i < n_nu; ++i)
        if (kmax[i] > kmax[iref]) iref = i;
    std::vector<double> bj(n_t, 0.0);
    if (kmax[iref] > 0.0)
        for (int j = 0; j < n_t; ++j) bj[j] = kappa_t[(size_t)iref * n_t + j] / kmax[iref];
    bool sep = true;
    for (int i = 0; i < n_nu && sep; ++i)
        for (int j = 0; j < n_t; ++j) {
            const double have = kappa_t[(size_t)i * n_t + j], want = kmax[i] * bj[j];
            if (std::fabs(have - want) > 1e-12 * std::max(std::fabs(have), std::fabs(want))) {
                sep = false;
                break;
            }
        }
    if (sep) {
        float tw_t[rt::kMaxTdepPoints];
        float4 tw_b[rt::kMaxTdepPoints];
        for (int j = 0; j < rt::kMaxTdepPoints; ++j) {
            tw_t[j] = j < n_t ? (float)t_grid[j] : INFINITY;
            if (j + 1 < n_t) {
                const double idt = 1.0 / ((double)(float)t_grid[j + 1] - (double)(float)t_grid[j]);
                tw_b[j] = make_float4((float)t_grid[j], (float)t_grid[j + 1], (float)(bj[j] * idt),
                                      (float)(bj[j + 1] * idt));
            } else {  // the last point holds: b_last (T_last + 1 - T) + b_last (T - T_last)
                const float tl = (float)t_grid[n_t - 1], bl = (float)bj[n_t - 1];
                tw_b[j] = make_float4(tl, tl + 1.0f, bl, bl);
            }
        }
        if (!ctx->tw_t_d) {
            bool ok = dalloc(&ctx->tw_t_d, rt::kMaxTdepPoints) == cudaSuccess &&
                      dalloc(&ctx->tw_b_d, rt::kMaxTdepPoints) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                return fail(ctx, RT_ERR_NO_MEMORY, "cannot allocate the column-weight table");
            }
        }
        RT_CK(ctx, cudaMemcpyAsync(ctx->tw_t_d, tw_t, sizeof(tw_t), cudaMemcpyHostToDevice, ctx->stream));
        RT_CK(ctx, cudaMemcpyAsync(ctx->tw_b_d, tw_b, sizeof(tw_b), cudaMemcpyHostToDevice, ctx->stream));
    }
    ctx->tw_sep = sep;
    // not separable: is it of rank two (with non-negative factors), else of rank 3 or 4?
    std::vector<double> fa, fb, f4(4 * (size_t)n_nu, 0.0), b4(4 * (size_t)n_t, 0.0);
    int rk = 0;
    if (!sep) {
        if (rank_two(kappa_t, n_nu, n_t, fa, fb)) {
            rk = 2;
            for (int i = 0; i < n_nu; ++i) {
                f4[4 * (size_t)i] = fa[2 * (size_t)i];
                f4[4 * (size_t)i + 1] = fa[2 * (size_t)i + 1];
            }
            for (int j = 0; j < n_t; ++j) {
                b4[j] = fb[j];
                b4[(size_t)n_t + j] = fb[(size_t)n_t + j];
            }
        } else {
            for (int R = 3; R <= 4 && rk == 0; ++R)
                if (low_rank(kappa_t, n_nu, n_t, R, f4, b4)) rk = R;
        }
    }
    if (rk >= 2) {
        float4 bw[rt::kMaxTdepPoints];
        for (int j = 0; j < rt::kMaxTdepPoints; ++j) {
            const int jj = j < n_t ? j : n_t - 1;
            bw[j] = make_float4((float)b4[jj], (float)b4[(size_t)n_t + jj], (float)b4[2 * (size_t)n_t + jj],
                                (float)b4[3 * (size_t)n_t + jj]);
        }
        if (!ctx->fac_a_d) {
            bool ok = dalloc(&ctx->fac_a_d, (size_t)4 * RT_MAX_NU) == cudaSuccess &&
                      dalloc(&ctx->r2_ab, (size_t)RT_MAX_NU + rt::kNuPad) == cudaSuccess &&
                      dalloc(&ctx->r2_bw, rt::kMaxTdepPoints) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                return fail(ctx, RT_ERR_NO_MEMORY, "cannot allocate the low-rank table");
            }
        }
        RT_CK(ctx, cudaMemcpyAsync(ctx->fac_a_d, f4.data(), sizeof(double) * 4 * n_nu, cudaMemcpyHostToDevice,
                                   ctx->stream));
        RT_CK(ctx, cudaMemcpyAsync(ctx->r2_bw, bw, sizeof(bw), cudaMemcpyHostToDevice, ctx->stream));
    }
    ctx->rk = rk;
    RT_CK(ctx, cudaMemcpyAsync(ctx->nu_mid, nu_mid, sizeof(double) * n_nu, cudaMemcpyHostToDevice, ctx->stream));
    RT_CK(ctx, cudaMemcpyAsync(ctx->kappa, kmax.data(), sizeof(double) * n_nu, cudaMemcpyHostToDevice, ctx->stream));
    RT_CK(ctx, cudaMemcpyAsync(ctx->kappa_t_d, kappa_t, sizeof(double) * n_nu * n_t, cudaMemcpyHostToDevice,
                               ctx->stream));
    RT_CK(ctx, cudaMemcpyAsync(ctx->tg32, tg.data(), sizeof(float) * n_t, cudaMemcpyHostToDevice, ctx->stream));
    RT_CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->n_nu = n_nu;
    ctx->t_sub = t_sub;
    ctx->kappa_bf16 = 0;
    ctx->n_t = n_t;
    ctx->tgrid_h.assign(t_grid, t_grid + n_t);
    ctx->kappa_t_h.assign(kappa_t, kappa_t + (size_t)n_nu * n_t);
    ctx->nu_h.assign(nu_mid, nu_mid + n_nu);
    ctx->kappa_h = kmax;
    ctx->have_table = true;
    return finalize(ctx);
}

int rt_set_star(rt_ctx *ctx, double t_star, double r_star)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!(t_star > 0.0) || !(r_star > 0.0) || !isfinite(t_star) || !isfinite(r_star))
        return fail(ctx, RT_ERR_INVALID_ARG, "t_star and r_star must be finite and > 0");
    RT_CK(ctx, cudaSetDevice(ctx->dev));
    ctx->t_star = t_star;
    ctx->r_star = r_star;
    ctx->have_star = true;
    return finalize(ctx);
}

int rt_irradiate(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs, float *a_rad,
                 rt_energy *energy)
{
    int st = check_call(ctx, rho, t_dust, q_abs, a_rad);
    if (st != RT_OK) return st;
    st = trace(ctx, rho, t_dust, q_abs, a_rad, ctx->shape);
    if (st != RT_OK || !energy) return st;
    return read_energy(ctx, energy);
}

namespace {
// Enqueue the host-buffer pipeline of one call (no synchronisation). With energy
// the validity word is left to read_energy; otherwise it is copied to bad_h ahead
// of the last copies out, and ev_out marks the end of the call's copies.
int host_enqueue(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs, float *a_rad, bool energy)
{
    int st = check_call(ctx, rho, t_dust, q_abs, a_rad);
    if (st != RT_OK) return st;
    if (!ctx->h_rho) {
        bool ok = dalloc(&ctx->h_rho, ctx->ncells) == cudaSuccess &&
                  dalloc(&ctx->h_t, ctx->ncells) == cudaSuccess &&
                  dalloc(&ctx->h_q, ctx->ncells) == cudaSuccess &&
                  dalloc(&ctx->h_a, ctx->ncells) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return fail(ctx, RT_ERR_NO_MEMORY, "cannot allocate device staging buffers");
        }
    }
    // Pipeline over ray chunks: the copies in of chunk k+1 (stream s_in) and out of
    // chunk k-1 (stream s_out, the other direction of the link) overlap the trace of
    // chunk k on the context's stream.
    if (!ctx->s_in) {
        bool ok = cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking) == cudaSuccess;
        for (int k = 0; ok && k < kHostChunks; ++k)
            ok = cudaEventCreateWithFlags(&ctx->ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ctx->ev_done[k], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return cuda_fail(ctx, "host pipeline streams", cudaGetLastError());
        RT_CK(ctx, cudaEventRecord(ctx->ev_out, ctx->s_out));
    }
    // at least ~2 M cells per chunk: copies of >= 8 MB per field, since the link moves
    // small copies in both directions at once less efficiently (4 MB: 253 GB/s in
    // total, 16 MB: 312 GB/s, one 256 MB copy each way: 340 GB/s)
    const long long cells_min = 1LL << 21;
    int nch = (int)std::min<long long>(kHostChunks, std::max<long long>(1, ctx->ncells / cells_min));
    if (nch > ctx->nrays) nch = (int)ctx->nrays;
    long long bound = 0;
    for (int k = 0; k < nch; ++k)
        bound += range_tiles(ctx, ctx->shape, ctx->nrays * k / nch, ctx->nrays * (k + 1) / nch);
    st = ensure_partials(ctx, bound);
    if (st != RT_OK) return st;
    ++ctx->seq;
    // the staging buffers are free once earlier traces (context stream) and the
    // previous call's copies out (ev_out) are done
    RT_CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0));
    RT_CK(ctx, cudaEventRecord(ctx->ev_start, ctx->stream));
    RT_CK(ctx, cudaStreamWaitEvent(ctx->s_in, ctx->ev_start, 0));
    long long npart = 0;
    for (int k = 0; k < nch; ++k) {
        const long long r0 = ctx->nrays * k / nch, r1 = ctx->nrays * (k + 1) / nch;
        const size_t off = (size_t)r0 * ctx->nr, n = (size_t)(r1 - r0) * ctx->nr * sizeof(float);
        RT_CK(ctx, cudaMemcpyAsync(ctx->h_rho + off, rho + off, n, cudaMemcpyHostToDevice, ctx->s_in));
        RT_CK(ctx, cudaMemcpyAsync(ctx->h_t + off, t_dust + off, n, cudaMemcpyHostToDevice, ctx->s_in));
        RT_CK(ctx, cudaEventRecord(ctx->ev_in[k], ctx->s_in));
        RT_CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_in[k], 0));
        st = trace_range(ctx, ctx->h_rho, ctx->h_t, ctx->h_q, ctx->h_a, ctx->shape, r0, r1, ctx->stream, &npart);
        if (st != RT_OK) return st;
        if (k == nch - 1 && !energy)  // the validity word, ahead of the last copies out
            RT_CK(ctx, cudaMemcpyAsync(ctx->bad_h, ctx->bad, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        RT_CK(ctx, cudaEventRecord(ctx->ev_done[k], ctx->stream));
        RT_CK(ctx, cudaStreamWaitEvent(ctx->s_out, ctx->ev_done[k], 0));
        RT_CK(ctx, cudaMemcpyAsync(q_abs + off, ctx->h_q + off, n, cudaMemcpyDeviceToHost, ctx->s_out));
        RT_CK(ctx, cudaMemcpyAsync(a_rad + off, ctx->h_a + off, n, cudaMemcpyDeviceToHost, ctx->s_out));
    }
    RT_CK(ctx, cudaEventRecord(ctx->ev_out, ctx->s_out));
    ctx->last_ntiles = npart;
    ctx->traced = true;
    return RT_OK;
}

// Wait for the copies out of the last host call; its validity word was copied ahead
// of them.
int host_wait(rt_ctx *ctx)
{
    RT_CK(ctx, cudaEventSynchronize(ctx->ev_out));
    ctx->host_pending = false;
    if (*ctx->bad_h == ctx->seq)
        return fail(ctx, RT_ERR_NONFINITE_INPUT, "input field holds NaN/Inf/negative density or NaN temperature");
    return RT_OK;
}
}  // namespace

int rt_irradiate_host(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs,
                      float *a_rad, rt_energy *energy)
{
    if (ctx && ctx->host_pending) {
        const int w = host_wait(ctx);
        if (w != RT_OK && w != RT_ERR_NONFINITE_INPUT) return w;
    }
    int st = host_enqueue(ctx, rho, t_dust, q_abs, a_rad, energy != nullptr);
    if (st != RT_OK) return st;
    if (energy) {
        st = read_energy(ctx, energy);
        if (st != RT_OK && st != RT_ERR_NONFINITE_INPUT) return st;
        RT_CK(ctx, cudaEventSynchronize(ctx->ev_out));
        return st;
    }
    return host_wait(ctx);
}

int rt_irradiate_host_async(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs, float *a_rad)
{
    if (ctx && ctx->host_pending) {  // one call in flight per context: the last one's validity word
        const int w = host_wait(ctx);
        if (w != RT_OK) return w;
    }
    const int st = host_enqueue(ctx, rho, t_dust, q_abs, a_rad, false);
    if (st == RT_OK) ctx->host_pending = true;
    return st;
}

int rt_host_wait(rt_ctx *ctx)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!ctx->host_pending) return RT_OK;
    RT_CK(ctx, cudaSetDevice(ctx->dev));
    return host_wait(ctx);
}

int rt_energy_last(rt_ctx *ctx, rt_energy *out)
{
    if (!ctx || !out) return RT_ERR_INVALID_ARG;
    if (!ctx->traced) return fail(ctx, RT_ERR_NOT_CONFIGURED, "nothing traced yet");
    RT_CK(ctx, cudaSetDevice(ctx->dev));
    return read_energy(ctx, out);
}

int rt_lut_build(rt_ctx *ctx, float err_tol)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!ctx->configured) return fail(ctx, RT_ERR_NOT_CONFIGURED, "call rt_set_star and rt_set_opacity_table first");
    if (ctx->n_t > 0) return fail(ctx, RT_ERR_INVALID_ARG, "the lookup table needs an opacity table kappa(nu)");
    if (ctx->precision == RT_FP64) return fail(ctx, RT_ERR_INVALID_ARG, "the lookup table is for the FP32 precisions");
    if (!(err_tol > 0.0f) || !(err_tol < 1.0f)) return fail(ctx, RT_ERR_INVALID_ARG, "err_tol must be in (0, 1)");
    RT_CK(ctx, cudaSetDevice(ctx->dev));
    const int na = ctx->sc_h.n_active;
    if (na < 1) return fail(ctx, RT_ERR_INVALID_ARG, "the table has no bin with kappa > 0");
    // kappa_ref = sum_i w_i kappa_i / sum_i w_i from the tracer's own bin table
    std::vector<NuEntry> nu(na);
    RT_CK(ctx, cudaMemcpyAsync(nu.data(), ctx->nu_tab, sizeof(NuEntry) * na, cudaMemcpyDeviceToHost, ctx->stream));
    RT_CK(ctx, cudaStreamSynchronize(ctx->stream));
    double sw = 0.0, swk = 0.0;
    for (const NuEntry &e : nu) {
        const double w = exp2((double)e.lf);
        sw += w;
        swk += w * -(double)e.nk * rt::kLn2;
    }
    if (!(sw > 0.0) || !(swk > 0.0)) return fail(ctx, RT_ERR_INVALID_ARG, "no stellar flux in the absorbing bins");
    const size_t n = (size_t)rt::kLutNs * rt::kLutNd;
    if (!ctx->lut) {
        bool ok = dalloc(&ctx->lut, n) == cudaSuccess && dalloc(&ctx->lut_count, 1) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return fail(ctx, RT_ERR_NO_MEMORY, "cannot allocate the lookup table");
        }
    }
    float *raw = nullptr;
    if (dalloc(&raw, n) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RT_ERR_NO_MEMORY, "cannot allocate the lookup table's scratch");
    }
    ctx->lut_kref = swk / sw;
    cudaError_t e = rt::launch_build_lut(ctx->nu_tab, ctx->sc, ctx->lut_kref, raw, ctx->lut, err_tol, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(raw);
    if (e != cudaSuccess) return cuda_fail(ctx, "lookup table", e);
    ctx->lut_tol = err_tol;
    ctx->lut_fp = ctx->fingerprint;
    return RT_OK;
}

int rt_irradiate_lut(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs, float *a_rad,
                     rt_energy *energy, unsigned *fallback_slots)
{
    int st = check_call(ctx, rho, t_dust, q_abs, a_rad);
    if (st != RT_OK) return st;
    if (!ctx->lut || ctx->lut_fp != ctx->fingerprint || ctx->n_t > 0)
        return fail(ctx, RT_ERR_NOT_CONFIGURED, "build the lookup table for this opacity table and star first");
    Shape cand[16];
    const int nc = rt::ray_shapes_lut(ctx->precision, ctx->nr, cand, 16);
    if (nc < 1) return fail(ctx, RT_ERR_INVALID_ARG, "the lookup table needs rays of at most 512 cells");
    Shape s = cand[0];
    for (int i = 0; i < nc; ++i)  // the context's own shape where it is compiled with the table
        if (cand[i].cells_per_lane == ctx->shape.cells_per_lane && cand[i].warps == ctx->shape.warps &&
            cand[i].min_blocks == ctx->shape.min_blocks && ctx->shape.kind == rt::kKindRay)
            s = cand[i];
    if (fallback_slots) RT_CK(ctx, cudaMemsetAsync(ctx->lut_count, 0, sizeof(unsigned), ctx->stream));
    ctx->lut_on = true;
    st = trace(ctx, rho, t_dust, q_abs, a_rad, s);
    ctx->lut_on = false;
    if (st != RT_OK) return st;
    if (fallback_slots) {
        RT_CK(ctx, cudaMemcpyAsync(fallback_slots, ctx->lut_count, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        RT_CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (!energy) return RT_OK;
    return read_energy(ctx, energy);
}

int rt_opacity_table_kind(const rt_ctx *ctx, int *kind)
{
    if (!ctx || !kind) return RT_ERR_INVALID_ARG;
    if (!ctx->configured) return RT_ERR_NOT_CONFIGURED;
    *kind = table_kind(ctx);
    return RT_OK;
}

int rt_energy_reduce(rt_ctx *ctx)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!ctx->traced) return fail(ctx, RT_ERR_NOT_CONFIGURED, "nothing traced yet");
    RT_CK(ctx, cudaSetDevice(ctx->dev));
    cudaError_t e = rt::launch_energy_reduce(ctx->partials, ctx->last_ntiles, ctx->sc, ctx->energy_d, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, "energy reduce", e);
    return RT_OK;
}

int rt_get_bins(rt_ctx *ctx, double *f_bin)
{
    if (!ctx || !f_bin) return RT_ERR_INVALID_ARG;
    if (!ctx->configured) return fail(ctx, RT_ERR_NOT_CONFIGURED, "star or table not set");
    RT_CK(ctx, cudaSetDevice(ctx->dev));
    RT_CK(ctx, cudaMemcpyAsync(f_bin, ctx->f_bin, sizeof(double) * ctx->n_nu, cudaMemcpyDeviceToHost, ctx->stream));
    RT_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return RT_OK;
}

int rt_set_tuning(rt_ctx *ctx, int kind, int cells_per_lane, int warps_per_block, int min_blocks_per_sm)
{
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (cells_per_lane == 0 && warps_per_block == 0) {
        ctx->shape_forced = false;
        if (ctx->configured) ctx->shape = default_shape(ctx);
        return RT_OK;
    }
    Shape all[64];
    const int n = all_shapes(ctx, all, 64);
    for (int i = 0; i < n; ++i) {
        if (all[i].kind == kind && all[i].cells_per_lane == cells_per_lane && all[i].warps == warps_per_block &&
            (min_blocks_per_sm == 0 || all[i].min_blocks == min_blocks_per_sm)) {
            ctx->shape = all[i];
            ctx->shape_forced = true;
            return RT_OK;
        }
    }
    return fail(ctx, RT_ERR_INVALID_ARG, "launch shape not compiled in, or not applicable to this grid");
}

int rt_get_tuning(const rt_ctx *ctx, int *kind, int *cells_per_lane, int *warps_per_block, int *min_blocks_per_sm)
{
    if (!ctx || !kind || !cells_per_lane || !warps_per_block || !min_blocks_per_sm) return RT_ERR_INVALID_ARG;
    *kind = ctx->shape.kind;
    *cells_per_lane = ctx->shape.cells_per_lane;
    *warps_per_block = ctx->shape.warps;
    *min_blocks_per_sm = ctx->shape.min_blocks;
    return RT_OK;
}

int rt_list_tunings(const rt_ctx *ctx, int *kinds, int *cells_per_lane, int *warps_per_block,
                    int *min_blocks_per_sm, int max)
{
    if (!ctx || max < 0 || (max > 0 && (!kinds || !cells_per_lane || !warps_per_block || !min_blocks_per_sm)))
        return RT_ERR_INVALID_ARG;
    Shape all[64];
    const int n = all_shapes(ctx, all, 64);
    for (int i = 0; i < n && i < max; ++i) {
        kinds[i] = all[i].kind;
        cells_per_lane[i] = all[i].cells_per_lane;
        warps_per_block[i] = all[i].warps;
        min_blocks_per_sm[i] = all[i].min_blocks;
    }
    return n;
}

int rt_autotune(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs, float *a_rad, int reps)
{
    int st = check_call(ctx, rho, t_dust, q_abs, a_rad);
    if (st != RT_OK) return st;
    if (reps < 1) return fail(ctx, RT_ERR_INVALID_ARG, "reps must be >= 1");
    Shape cand[64];
    const int n = all_shapes(ctx, cand, 64);
    cudaEvent_t e0, e1;
    RT_CK(ctx, cudaEventCreate(&e0));
    RT_CK(ctx, cudaEventCreate(&e1));
    float best_ms = 1e30f;
    Shape best = ctx->shape;
    for (int i = 0; i < n; ++i) {
        st = trace(ctx, rho, t_dust, q_abs, a_rad, cand[i]);  // warm-up
        if (st != RT_OK) break;
        cudaEventRecord(e0, ctx->stream);
        for (int r = 0; r < reps && st == RT_OK; ++r) st = trace(ctx, rho, t_dust, q_abs, a_rad, cand[i]);
        cudaEventRecord(e1, ctx->stream);
        if (st != RT_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = cuda_fail(ctx, "autotune sync", cudaGetLastError()); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = cand[i]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RT_OK) return st;
    ctx->shape = best;
    ctx->shape_forced = true;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[std::make_tuple(ctx->precision, ctx->nr, ctx->nrays, ctx->sc_h.nnu_pad, table_kind(ctx))] = best;
    }
    return RT_OK;
}

void rt_destroy(rt_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->dev);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->sur) rt::sur_free(ctx->sur);
    if (ctx->fld) rt::fld_free(ctx->fld);
    if (ctx->s_in) {
        cudaStreamSynchronize(ctx->s_in);
        cudaStreamSynchronize(ctx->s_out);
        cudaStreamDestroy(ctx->s_in);
        cudaStreamDestroy(ctx->s_out);
        for (int k = 0; k < kHostChunks; ++k) {
            if (ctx->ev_in[k]) cudaEventDestroy(ctx->ev_in[k]);
            if (ctx->ev_done[k]) cudaEventDestroy(ctx->ev_done[k]);
        }
        if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
        if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    }
    free_all(ctx);
    delete ctx;
}

const char *rt_last_error(const rt_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

const char *rt_status_string(int status)
{
    switch (status) {
    case RT_OK: return "RT_OK";
    case RT_ERR_INVALID_ARG: return "RT_ERR_INVALID_ARG";
    case RT_ERR_NOT_CONFIGURED: return "RT_ERR_NOT_CONFIGURED";
    case RT_ERR_CUDA: return "RT_ERR_CUDA";
    case RT_ERR_TIMEOUT: return "RT_ERR_TIMEOUT";
    case RT_ERR_NONFINITE_INPUT: return "RT_ERR_NONFINITE_INPUT";
    case RT_ERR_NO_MEMORY: return "RT_ERR_NO_MEMORY";
    default: return "RT_UNKNOWN_STATUS";
    }
}

}  // extern "C"
