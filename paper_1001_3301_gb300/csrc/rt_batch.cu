// Many grids of uneven size in one persistent launch, replayed from a CUDA graph.
//
// A batch is a set of configured contexts (any nr, ntheta, nphi and number of
// bins; one precision). Their flattened tiles are concatenated; each CTA of one
// persistent launch owns a contiguous range of that concatenation whose cost
// (tiles weighted by the grid's bin count) is 1/G of the total, and walks it grid
// segment by grid segment with the tile body of rt_tile.cuh, writing one energy
// partial per (grid, CTA). A second small kernel reduces the partials of every
// grid in FP64. Both kernels and the partials reset form a CUDA graph built once;
// each run only replaces the field pointers in the tracer node and replays it.
// Two kernel families: the tile body of rt_tile.cuh (any nr; work units are tiles,
// split statically as above), and the warp-per-ray body of rt_ray.cuh (every grid
// with nr <= 32 C; work units are warp-slots of 32 / G rays, G = 8, 16 or 32 lanes
// per ray chosen per grid, handed out in chunks at run time from one counter that
// a memset node of the graph zeroes).
// The shape comes from rt_batch_autotune (timed on the caller's buffers) or,
// before that, from a fixed default.
#include <string.h>

#include <string>
#include <vector>

#include "rt_ray.cuh"
#include "rt_tile.cuh"

namespace rt {
namespace {

struct BatchParams {
    const TraceArgs *grids;          // [n] tables and sizes of every grid
    const unsigned *grid_tile_begin; // [n+1] first global work unit (tile or warp-slot) of every grid
    const unsigned *cta_begin;       // [G+1] first global work unit of every CTA
    double2 *partials;               // [n * G] (absorbed, escaped) per grid and CTA
    unsigned *work;                  // warp-per-ray kind: next chunk to hand out (zeroed per run)
    const unsigned *chunk_begin;     // [n+1] first chunk of every grid (warp-per-ray kind)
    unsigned n_chunks;               // chunks of all grids
    unsigned chunk_slots;            // warp-slots per chunk
    unsigned seq;                    // call number, stored in the validity word on bad input
    int n;
    const float *rho[RT_BATCH_MAX];
    const float *tdust[RT_BATCH_MAX];
    float *q[RT_BATCH_MAX];
    float *a[RT_BATCH_MAX];
};

// warp-slots per warp in one chunk of the warp-per-ray batch
constexpr unsigned kBatchChunkWarpSlots = 8;

template <int C, int W, int MODE, int MINB>
__global__ void __launch_bounds__(W * 32, MINB) k_batch(const __grid_constant__ BatchParams bp)
{
    __shared__ TraceArgs s_p;
    const unsigned T0 = bp.cta_begin[blockIdx.x], T1 = bp.cta_begin[blockIdx.x + 1];
    if (T0 >= T1) return;
    // first grid whose tiles extend past T0
    int lo = 0, hi = bp.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (bp.grid_tile_begin[mid + 1] > T0) hi = mid;
        else lo = mid + 1;
    }
    unsigned t = T0;
    for (int g = lo; t < T1 && g < bp.n; ++g) {
        const unsigned gb = bp.grid_tile_begin[g], ge = bp.grid_tile_begin[g + 1];
        const unsigned seg_end = T1 < ge ? T1 : ge;
        if (seg_end <= t) continue;
        __syncthreads();  // everyone is done with the previous grid's s_p
        if (threadIdx.x == 0) {
            s_p = bp.grids[g];
            s_p.rho = bp.rho[g];
            s_p.tdust = bp.tdust[g];
            s_p.q = bp.q[g];
            s_p.a = bp.a[g];
            s_p.seq = bp.seq;
        }
        __syncthreads();
        typename TileTypes<MODE>::ESum eabs, eesc;
        eabs.zero();
        eesc.zero();
        trace_tile_range<C, W, MODE>(s_p, t - gb, seg_end - gb, eabs, eesc);
        block_energy<W>(eabs, eesc);
        if (threadIdx.x == 0)
            bp.partials[(size_t)g * gridDim.x + blockIdx.x] = make_double2(to_double(eabs), to_double(eesc));
        t = seg_end;
    }
}

// Lanes per ray of grid p for C cells per lane: the fewest of 8, 16, 32 that hold
// the ray (nr <= 32 C for every grid of a ray-kind batch).
__host__ __device__ __forceinline__ int ray_lanes_for(int nr, int C)
{
    return nr <= 8 * C ? 8 : (nr <= 16 * C ? 16 : 32);
}

// The warp-per-ray batch. The grids' warp-slots are cut into chunks of
// chunk_slots (a chunk never spans two grids), and the CTAs take chunks in order
// from one counter: the cost of a warp-slot depends on how many of its bins the
// thin series takes, which only the fields decide, so a static split by bins would
// leave CTAs idle. Chunk indices grow, so a CTA meets every grid at most once; it
// stages the grid's descriptor and tables in shared memory when the grid changes
// and writes one FP64 energy partial per (grid, CTA) when it leaves it. The next
// chunk's index is fetched while the current one is traced.
template <int C, int W, int MODE, int MINB>
__global__ void __launch_bounds__(W * 32, MINB) k_batch_ray(const __grid_constant__ BatchParams bp)
{
    __shared__ TraceArgs s_p;
    __shared__ RayShared<C> rs;
    __shared__ unsigned s_next;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    float *const s_kap = reinterpret_cast<float *>(smem);
    float4 *s_nu = nullptr, *s_mom = nullptr;
    if (threadIdx.x == 0) s_next = atomicAdd(bp.work, 1u);
    __syncthreads();
    unsigned c = s_next;
    int cur = -1, G = 32;
    KahanSum eabs, eesc;
    eabs.zero();
    eesc.zero();
    while (c < bp.n_chunks) {
        __syncthreads();  // every thread has read s_next
        if (threadIdx.x == 0) s_next = atomicAdd(bp.work, 1u);
        int lo = 0, hi = bp.n - 1;  // grid of chunk c
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (bp.chunk_begin[mid + 1] > c) hi = mid;
            else lo = mid + 1;
        }
        if (lo != cur) {
            if (cur >= 0) {
                block_energy<W>(eabs, eesc);
                if (threadIdx.x == 0)
                    bp.partials[(size_t)cur * gridDim.x + blockIdx.x] = make_double2(to_double(eabs), to_double(eesc));
            }
            __syncthreads();  // everyone is done with the previous grid's tables
            if (threadIdx.x == 0) {
                s_p = bp.grids[lo];
                s_p.rho = bp.rho[lo];
                s_p.tdust = bp.tdust[lo];
                s_p.q = bp.q[lo];
                s_p.a = bp.a[lo];
                s_p.seq = bp.seq;
            }
            __syncthreads();
            G = ray_lanes_for(s_p.nr, C);
            s_nu = reinterpret_cast<float4 *>(s_kap + s_p.nnu_pad);
            s_mom = s_nu + s_p.nnu_pad;
            ray_tables<C, W>(s_p, G, rs, s_kap, s_nu, s_mom);
            __syncthreads();
            cur = lo;
            eabs.zero();
            eesc.zero();
        }
        const unsigned units = bp.grid_tile_begin[cur + 1] - bp.grid_tile_begin[cur];
        const unsigned w0 = (c - bp.chunk_begin[cur]) * bp.chunk_slots;
        const unsigned w1 = w0 + bp.chunk_slots < units ? w0 + bp.chunk_slots : units;
        if (G == 8) ray_slots<C, W, MODE, 8>(s_p, w0 + warp, w1, W, rs, s_kap, s_nu, s_mom, eabs, eesc);
        else if (G == 16) ray_slots<C, W, MODE, 16>(s_p, w0 + warp, w1, W, rs, s_kap, s_nu, s_mom, eabs, eesc);
        else ray_slots<C, W, MODE, 32>(s_p, w0 + warp, w1, W, rs, s_kap, s_nu, s_mom, eabs, eesc);
        __syncthreads();  // s_next holds the next chunk
        c = s_next;
    }
    if (cur >= 0) {
        block_energy<W>(eabs, eesc);
        if (threadIdx.x == 0)
            bp.partials[(size_t)cur * gridDim.x + blockIdx.x] = make_double2(to_double(eabs), to_double(eesc));
    }
}

// One block per grid: FP64 sum of its partials and the energy bookkeeping of
// rt_energy (the same formulas as the single-grid reduction).
__global__ void k_batch_energy(const double2 *partials, unsigned G, const DevScalars *const *sc,
                               rt_energy *out)
{
    __shared__ double s_a[32], s_e[32];
    const int g = blockIdx.x;
    double sa = 0.0, se = 0.0;
    for (unsigned b = threadIdx.x; b < G; b += blockDim.x) {
        sa += partials[(size_t)g * G + b].x;
        se += partials[(size_t)g * G + b].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        se += __shfl_xor_sync(0xffffffffu, se, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { s_a[w] = sa; s_e[w] = se; }
    __syncthreads();
    if (threadIdx.x == 0) {
        sa = 0.0;
        se = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { sa += s_a[i]; se += s_e[i]; }
        const DevScalars *s = sc[g];
        const double scale = s->r2 * s->f_max;
        rt_energy e;
        e.e_abs = scale * sa;
        e.e_esc = scale * se + s->r2 * s->f_transparent * s->sum_domega;
        e.l_star = s->l_grid;
        e.rel_err = (e.e_abs + e.e_esc) / e.l_star - 1.0;
        out[g] = e;
    }
}

using BatchKernel = void (*)(BatchParams);

struct BatchShape {
    int kind;  // RT_KERNEL_TILE or RT_KERNEL_RAY
    int precision, c, w, minb;
    BatchKernel kern;
};

#define RT_BSHAPE(P, C, W, MB) {RT_KERNEL_TILE, P, C, W, MB, &k_batch<C, W, P, MB>}
#define RT_BRAY(P, C, W, MB) {RT_KERNEL_RAY, P, C, W, MB, &k_batch_ray<C, W, P, MB>}
const BatchShape kBatchShapes[] = {
    RT_BSHAPE(RT_FP32_KAHAN, 2, 4, 8), RT_BSHAPE(RT_FP32_KAHAN, 4, 4, 8), RT_BSHAPE(RT_FP32_KAHAN, 4, 8, 4),
    RT_BSHAPE(RT_FP32_KAHAN, 8, 4, 6), RT_BSHAPE(RT_FP32_KAHAN, 8, 4, 5), RT_BSHAPE(RT_FP32_KAHAN, 8, 8, 3),
    RT_BRAY(RT_FP32_KAHAN, 8, 4, 6),   RT_BRAY(RT_FP32_KAHAN, 16, 4, 3), RT_BRAY(RT_FP32_KAHAN, 16, 4, 4),
    RT_BSHAPE(RT_FP32_PLAIN, 4, 4, 8), RT_BSHAPE(RT_FP32_PLAIN, 8, 4, 6), RT_BRAY(RT_FP32_PLAIN, 16, 4, 4),
    RT_BSHAPE(RT_FP64, 2, 4, 8),       RT_BSHAPE(RT_FP64, 4, 4, 4),
};
#undef RT_BSHAPE
#undef RT_BRAY

}  // namespace
}  // namespace rt

using rt::BatchParams;
using rt::BatchShape;

struct rt_batch {
    int n = 0, dev = 0, precision = 0;
    cudaStream_t stream = nullptr;
    std::vector<rt::CtxView> views;
    std::vector<const rt_ctx *> ctxs;
    // device memory owned by the batch
    rt::TraceArgs *grids_d = nullptr;
    unsigned *grid_tile_begin_d = nullptr;
    unsigned *cta_begin_d = nullptr;
    unsigned *chunk_begin_d = nullptr;  // [n+1], warp-per-ray kind
    unsigned *work_d = nullptr;         // chunk counter of the warp-per-ray kind
    double2 *partials_d = nullptr;
    const rt::DevScalars **sc_d = nullptr;
    rt_energy *energies_d = nullptr;
    unsigned *bad_d = nullptr;
    rt_energy *energies_h = nullptr;  // pinned
    unsigned *bad_h = nullptr;        // pinned
    size_t partials_cap = 0, cta_cap = 0;
    // launch plan
    const BatchShape *shape = nullptr;
    unsigned G = 0;
    size_t smem = 0;
    BatchParams params{};
    unsigned seq = 0;
    bool ran = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t kern_node = nullptr;
    cudaKernelNodeParams kp{};
    void *kp_args[1] = {nullptr};
    std::string err;
};

namespace {

int bfail(rt_batch *b, int status, const std::string &msg)
{
    if (b) b->err = msg;
    else rt::set_thread_error(msg);
    return status;
}

#define RT_BCK(b, call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return bfail(b, RT_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

size_t tile_smem(const rt::TraceArgs &a, const BatchShape &s)
{
    // rt_tile.cuh layout: input double buffer and output staging (skewed), radial
    // table (skewed, FP32 modes with nr <= 1024), bin tables
    const long long T = 32LL * s.w * s.c;
    const long long TS = (T + T / 32 + 1 + 3) & ~3LL;
    const bool staged = (s.precision != RT_FP64) && a.nr <= 1024;
    const long long nrs = staged ? ((a.nr + a.nr / 32 + 1 + 3) & ~3) : 0;
    return (size_t)(TS * 6 * 4 + 3 * nrs * 4 + (long long)a.nnu_pad * 4 + (long long)a.nnu_pad * (16 + 32) + 16);
}

// whether every grid of the batch fits the warp-per-ray body of shape s
bool ray_fits(const rt_batch *b, const BatchShape &s)
{
    for (const rt::CtxView &v : b->views)
        if (v.args.nr > 32 * s.c) return false;
    return true;
}

// Shape-dependent plan: work-unit ranges per CTA balanced by cost (tile kind; a tile
// of 32 W C flattened cells costs about (bins + 6) per cell) or the chunk table (ray
// kind: warp-slots of 32 / G rays), partials, graph.
int plan(rt_batch *b, const BatchShape *s)
{
    const int n = b->n;
    const bool ray = s->kind == RT_KERNEL_RAY;
    const long long T = 32LL * s->w * s->c;
    size_t smem = 0;
    for (const rt::CtxView &v : b->views)
        smem = std::max(smem, ray ? rt::ray_bin_smem(v.args.nnu_pad) + 16 : tile_smem(v.args, *s));
    if (smem > 48 * 1024)
        RT_BCK(b, cudaFuncSetAttribute(s->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nsm = 0, per_sm = 0;
    RT_BCK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->dev));
    RT_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s->kern, s->w * 32, smem));
    if (per_sm < 1) per_sm = 1;
    // tiles per grid and the cost of one tile (bins plus the per-cell work outside
    // the bin loop, about six bins' worth)
    std::vector<unsigned> gtb(n + 1, 0);
    std::vector<double> cost_before(n + 1, 0.0);
    for (int g = 0; g < n; ++g) {
        long long nt;
        if (ray) {
            const int R = 32 / rt::ray_lanes_for(b->views[g].args.nr, s->c);
            nt = ((long long)b->views[g].args.nrays + R - 1) / R;
        } else {
            nt = (b->views[g].flat_cells + T - 1) / T;
        }
        gtb[g + 1] = gtb[g] + (unsigned)nt;
        cost_before[g + 1] = cost_before[g] + (double)nt * (b->views[g].args.nnu_pad + 6);
    }
    const unsigned total_tiles = gtb[n];
    unsigned G = (unsigned)nsm * (unsigned)per_sm;
    // warp-per-ray kind: chunks of kBatchChunkWarpSlots warp-slots per warp, handed out
    // in order at run time (so G only needs to fill the GPU)
    const unsigned chunk_slots = (unsigned)s->w * rt::kBatchChunkWarpSlots;
    std::vector<unsigned> chb(n + 1, 0);
    for (int gg = 0; gg < n; ++gg) chb[gg + 1] = chb[gg] + (gtb[gg + 1] - gtb[gg] + chunk_slots - 1) / chunk_slots;
    if (ray) {
        if (G > chb[n]) G = chb[n];
    } else if (G > total_tiles) {
        G = total_tiles;
    }
    if (G < 1) G = 1;
    std::vector<unsigned> cb(G + 1, 0);
    int g = 0;
    for (unsigned k = 1; k < G; ++k) {
        const double target = cost_before[n] * k / G;
        while (g < n - 1 && cost_before[g + 1] <= target) ++g;
        const double per_tile = b->views[g].args.nnu_pad + 6.0;
        unsigned t = gtb[g] + (unsigned)((target - cost_before[g]) / per_tile);
        if (t > gtb[g + 1]) t = gtb[g + 1];
        cb[k] = std::max(t, cb[k - 1]);
    }
    cb[G] = total_tiles;

    // device buffers that depend on G
    if ((size_t)n * G > b->partials_cap) {
        if (b->partials_d) cudaFree(b->partials_d);
        b->partials_d = nullptr;
        RT_BCK(b, cudaMalloc(&b->partials_d, sizeof(double2) * (size_t)n * G));
        b->partials_cap = (size_t)n * G;
    }
    if (G + 1 > b->cta_cap) {
        if (b->cta_begin_d) cudaFree(b->cta_begin_d);
        b->cta_begin_d = nullptr;
        RT_BCK(b, cudaMalloc(&b->cta_begin_d, sizeof(unsigned) * (G + 1)));
        b->cta_cap = G + 1;
    }
    RT_BCK(b, cudaMemcpy(b->cta_begin_d, cb.data(), sizeof(unsigned) * (G + 1), cudaMemcpyHostToDevice));
    RT_BCK(b, cudaMemcpy(b->grid_tile_begin_d, gtb.data(), sizeof(unsigned) * (n + 1), cudaMemcpyHostToDevice));
    RT_BCK(b, cudaMemcpy(b->chunk_begin_d, chb.data(), sizeof(unsigned) * (n + 1), cudaMemcpyHostToDevice));

    b->shape = s;
    b->G = G;
    b->smem = smem;
    b->params.grids = b->grids_d;
    b->params.grid_tile_begin = b->grid_tile_begin_d;
    b->params.cta_begin = b->cta_begin_d;
    b->params.partials = b->partials_d;
    b->params.work = b->work_d;
    b->params.chunk_begin = b->chunk_begin_d;
    b->params.n_chunks = chb[n];
    b->params.chunk_slots = chunk_slots;
    b->params.n = n;

    // graph: reset partials -> tracer -> per-grid energy
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    RT_BCK(b, cudaGraphCreate(&b->graph, 0));
    cudaMemsetParams mp{};
    mp.dst = b->partials_d;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = (size_t)n * G * sizeof(double2) / 4;
    mp.height = 1;
    mp.pitch = 0;
    cudaGraphNode_t n_reset[2], n_energy;
    RT_BCK(b, cudaGraphAddMemsetNode(&n_reset[0], b->graph, nullptr, 0, &mp));
    cudaMemsetParams mw{};
    mw.dst = b->work_d;
    mw.value = 0;
    mw.elementSize = 4;
    mw.width = 1;
    mw.height = 1;
    mw.pitch = 0;
    RT_BCK(b, cudaGraphAddMemsetNode(&n_reset[1], b->graph, nullptr, 0, &mw));
    b->kp_args[0] = &b->params;
    b->kp.func = (void *)s->kern;
    b->kp.gridDim = dim3(G);
    b->kp.blockDim = dim3(s->w * 32);
    b->kp.sharedMemBytes = (unsigned)smem;
    b->kp.kernelParams = b->kp_args;
    b->kp.extra = nullptr;
    RT_BCK(b, cudaGraphAddKernelNode(&b->kern_node, b->graph, n_reset, 2, &b->kp));
    cudaKernelNodeParams ep{};
    const double2 *e_part = b->partials_d;  // argument values are copied into the node
    unsigned e_g = G;
    const rt::DevScalars *const *e_sc = b->sc_d;
    rt_energy *e_out = b->energies_d;
    void *eargs[4] = {&e_part, &e_g, &e_sc, &e_out};
    ep.func = (void *)rt::k_batch_energy;
    ep.gridDim = dim3(n);
    ep.blockDim = dim3(256);
    ep.sharedMemBytes = 0;
    ep.kernelParams = eargs;
    ep.extra = nullptr;
    RT_BCK(b, cudaGraphAddKernelNode(&n_energy, b->graph, &b->kern_node, 1, &ep));
    RT_BCK(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
    return RT_OK;
}

int set_pointers(rt_batch *b, const float *const *rho, const float *const *td, float *const *q,
                 float *const *a)
{
    if (!rho || !td || !q || !a) return bfail(b, RT_ERR_INVALID_ARG, "NULL pointer array");
    for (int g = 0; g < b->n; ++g) {
        if (!rho[g] || !td[g] || !q[g] || !a[g]) return bfail(b, RT_ERR_INVALID_ARG, "NULL field pointer");
        b->params.rho[g] = rho[g];
        b->params.tdust[g] = td[g];
        b->params.q[g] = q[g];
        b->params.a[g] = a[g];
    }
    b->params.seq = ++b->seq;
    return RT_OK;
}

void free_batch(rt_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    void *ptrs[] = {b->grids_d, b->grid_tile_begin_d, b->cta_begin_d, b->chunk_begin_d, b->work_d, b->partials_d,
                    (void *)b->sc_d, b->energies_d, b->bad_d};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->energies_h) cudaFreeHost(b->energies_h);
    if (b->bad_h) cudaFreeHost(b->bad_h);
}

}  // namespace

extern "C" {

int rt_batch_create(rt_ctx *const *ctxs, int n, void *cuda_stream, rt_batch **out)
{
    if (!out) return bfail(nullptr, RT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1 || n > RT_BATCH_MAX)
        return bfail(nullptr, RT_ERR_INVALID_ARG, "a batch holds 1.." + std::to_string(RT_BATCH_MAX) + " contexts");
    rt_batch *b = new (std::nothrow) rt_batch();
    if (!b) return bfail(nullptr, RT_ERR_NO_MEMORY, "out of host memory");
    b->n = n;
    b->stream = (cudaStream_t)cuda_stream;
    b->views.resize(n);
    for (int g = 0; g < n; ++g) {
        if (!rt::ctx_view(ctxs[g], &b->views[g])) {
            delete b;
            return bfail(nullptr, RT_ERR_NOT_CONFIGURED, "context " + std::to_string(g) + " is NULL or not configured");
        }
        const rt::CtxView &v = b->views[g];
        if (v.tdep) {
            delete b;
            return bfail(nullptr, RT_ERR_INVALID_ARG,
                         "context " + std::to_string(g) + " has a temperature-dependent table (not batched)");
        }
        if (g > 0 && (v.precision != b->views[0].precision || v.dev != b->views[0].dev)) {
            delete b;
            return bfail(nullptr, RT_ERR_INVALID_ARG, "all contexts of a batch need one precision and one device");
        }
        if (v.flat_cells >= rt::kMaxLaunchCells) {
            delete b;
            return bfail(nullptr, RT_ERR_INVALID_ARG, "context " + std::to_string(g) + " is too large for a batch");
        }
    }
    b->precision = b->views[0].precision;
    b->dev = b->views[0].dev;
    if (cudaSetDevice(b->dev) != cudaSuccess) {
        delete b;
        return bfail(nullptr, RT_ERR_CUDA, "cudaSetDevice failed");
    }
    bool ok = cudaMalloc(&b->grids_d, sizeof(rt::TraceArgs) * n) == cudaSuccess &&
              cudaMalloc(&b->grid_tile_begin_d, sizeof(unsigned) * (n + 1)) == cudaSuccess &&
              cudaMalloc(&b->chunk_begin_d, sizeof(unsigned) * (n + 1)) == cudaSuccess &&
              cudaMalloc(&b->work_d, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&b->sc_d, sizeof(void *) * n) == cudaSuccess &&
              cudaMalloc(&b->energies_d, sizeof(rt_energy) * n) == cudaSuccess &&
              cudaMalloc(&b->bad_d, sizeof(unsigned)) == cudaSuccess &&
              cudaMallocHost(&b->energies_h, sizeof(rt_energy) * n) == cudaSuccess &&
              cudaMallocHost(&b->bad_h, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(b);
        delete b;
        return bfail(nullptr, RT_ERR_CUDA, "device allocation failed in rt_batch_create");
    }
    std::vector<rt::TraceArgs> args(n);
    std::vector<const rt::DevScalars *> scs(n);
    for (int g = 0; g < n; ++g) {
        args[g] = b->views[g].args;
        args[g].L = (unsigned)b->views[g].flat_cells;
        args[g].bad_input = b->bad_d;
        scs[g] = b->views[g].sc;
    }
    ok = cudaMemcpy(b->grids_d, args.data(), sizeof(rt::TraceArgs) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->sc_d, scs.data(), sizeof(void *) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(b->bad_d, 0, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        free_batch(b);
        delete b;
        return bfail(nullptr, RT_ERR_CUDA, "copy failed in rt_batch_create");
    }
    // default shape: 8-cell tiles (4-cell for FP64)
    const BatchShape *def = nullptr;
    for (const BatchShape &s : rt::kBatchShapes)
        if (s.precision == b->precision && s.kind == RT_KERNEL_TILE && !def) def = &s;
    for (const BatchShape &s : rt::kBatchShapes)
        if (s.precision == b->precision && s.kind == RT_KERNEL_TILE && s.c == (b->precision == RT_FP64 ? 4 : 8) &&
            s.w == 4) {
            def = &s;
            break;
        }
    int st = plan(b, def);
    if (st != RT_OK) {
        rt::set_thread_error(b->err);
        free_batch(b);
        delete b;
        return st;
    }
    *out = b;
    return RT_OK;
}

int rt_batch_run(rt_batch *b, const float *const *rho, const float *const *t_dust, float *const *q_abs,
                 float *const *a_rad)
{
    if (!b) return RT_ERR_INVALID_ARG;
    RT_BCK(b, cudaSetDevice(b->dev));
    int st = set_pointers(b, rho, t_dust, q_abs, a_rad);
    if (st != RT_OK) return st;
    RT_BCK(b, cudaGraphExecKernelNodeSetParams(b->exec, b->kern_node, &b->kp));
    RT_BCK(b, cudaGraphLaunch(b->exec, b->stream));
    b->ran = true;
    return RT_OK;
}

int rt_batch_energy(rt_batch *b, rt_energy *energies)
{
    if (!b || !energies) return RT_ERR_INVALID_ARG;
    if (!b->ran) return bfail(b, RT_ERR_NOT_CONFIGURED, "the batch has not run yet");
    RT_BCK(b, cudaSetDevice(b->dev));
    RT_BCK(b, cudaMemcpyAsync(b->energies_h, b->energies_d, sizeof(rt_energy) * b->n, cudaMemcpyDeviceToHost, b->stream));
    RT_BCK(b, cudaMemcpyAsync(b->bad_h, b->bad_d, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    RT_BCK(b, cudaStreamSynchronize(b->stream));
    memcpy(energies, b->energies_h, sizeof(rt_energy) * b->n);
    if (*b->bad_h == b->seq)
        return bfail(b, RT_ERR_NONFINITE_INPUT, "an input field holds NaN/Inf/negative density or NaN temperature");
    return RT_OK;
}

int rt_batch_autotune(rt_batch *b, const float *const *rho, const float *const *t_dust, float *const *q_abs,
                      float *const *a_rad, int reps)
{
    if (!b || reps < 1) return RT_ERR_INVALID_ARG;
    RT_BCK(b, cudaSetDevice(b->dev));
    const BatchShape *best = b->shape;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    RT_BCK(b, cudaEventCreate(&e0));
    RT_BCK(b, cudaEventCreate(&e1));
    int st = RT_OK;
    for (const BatchShape &s : rt::kBatchShapes) {
        if (s.precision != b->precision) continue;
        if (s.kind == RT_KERNEL_RAY && !ray_fits(b, s)) continue;
        st = plan(b, &s);
        if (st != RT_OK) break;
        st = rt_batch_run(b, rho, t_dust, q_abs, a_rad);  // warm-up
        if (st != RT_OK) break;
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps && st == RT_OK; ++r) st = rt_batch_run(b, rho, t_dust, q_abs, a_rad);
        cudaEventRecord(e1, b->stream);
        if (st != RT_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = bfail(b, RT_ERR_CUDA, "autotune sync failed"); break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = &s; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RT_OK) return st;
    return plan(b, best);
}

int rt_batch_get_tuning(const rt_batch *b, int *kind, int *cells_per_lane, int *warps_per_block,
                        int *min_blocks_per_sm)
{
    if (!b || !kind || !cells_per_lane || !warps_per_block || !min_blocks_per_sm) return RT_ERR_INVALID_ARG;
    *kind = b->shape->kind;
    *cells_per_lane = b->shape->c;
    *warps_per_block = b->shape->w;
    *min_blocks_per_sm = b->shape->minb;
    return RT_OK;
}

int rt_batch_set_tuning(rt_batch *b, int kind, int cells_per_lane, int warps_per_block, int min_blocks_per_sm)
{
    if (!b) return RT_ERR_INVALID_ARG;
    RT_BCK(b, cudaSetDevice(b->dev));
    for (const BatchShape &s : rt::kBatchShapes) {
        if (s.precision != b->precision || s.kind != kind || s.c != cells_per_lane || s.w != warps_per_block ||
            (min_blocks_per_sm != 0 && s.minb != min_blocks_per_sm))
            continue;
        if (s.kind == RT_KERNEL_RAY && !ray_fits(b, s))
            return bfail(b, RT_ERR_INVALID_ARG, "a grid of the batch has more radial cells than 32 cells_per_lane");
        return plan(b, &s);
    }
    return bfail(b, RT_ERR_INVALID_ARG, "no such batch shape for this precision");
}

const char *rt_batch_last_error(const rt_batch *b) { return b ? b->err.c_str() : rt_last_error(nullptr); }

void rt_batch_destroy(rt_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->dev);
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
}

}  // extern "C"
