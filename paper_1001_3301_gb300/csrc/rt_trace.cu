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
//      which Eq. 36 removes) times the absorbed fraction 1 - e^{-kappa_i dN} (Eqs.
//      31-32), accumulated into one register per cell;
//   4. escaping power per ray (Eqs. 33-35) from the column at the ray's escape cell,
//      q_abs = Gq(r) * sum, a_rad = q_abs / (rho c) (Sect. 5; its rho -> 0 limit
//      where the column is 0), and per-tile FP64 energy partials.
//
//
// The per-(cell, bin) arithmetic is described in rt_device.cuh.
#include "rt_tile.cuh"

namespace rt {
namespace {

// Persistent single-grid tracer: CTA b traces the contiguous tiles
// [b n / G, (b+1) n / G) and writes its energy partial.
template <int C, int W, int MODE, int MINB>
__global__ void __launch_bounds__(W * 32, MINB) k_trace(const TraceArgs p)
{
    constexpr int T = 32 * W * C;
    const unsigned ntiles = (p.L + (unsigned)T - 1u) / (unsigned)T;
    const unsigned t_begin = (unsigned)((unsigned long long)blockIdx.x * ntiles / gridDim.x);
    const unsigned t_end = (unsigned)((unsigned long long)(blockIdx.x + 1) * ntiles / gridDim.x);
    typename TileTypes<MODE>::ESum eabs, eesc;
    eabs.zero();
    eesc.zero();
    trace_tile_range<C, W, MODE>(p, t_begin, t_end, eabs, eesc);
    block_energy<W>(eabs, eesc);
    if (threadIdx.x == 0) p.partials[blockIdx.x] = make_double2(to_double(eabs), to_double(eesc));
}

// Launch one chunk with a persistent grid of (SMs x resident CTAs) CTAs, or fewer
// when there are fewer tiles. Returns the grid size (energy partials written).
template <int C, int W, int MODE, int MINB>
cudaError_t launch_shape(const TraceArgs &a, unsigned ntiles, cudaStream_t stream, unsigned *grid_out,
                         unsigned max_grid)
{
    const size_t smem = trace_smem_bytes<C, W, MODE>(a);
    auto kern = k_trace<C, W, MODE, MINB>;
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
    if (grid > ntiles) grid = ntiles;
    if (max_grid > 0 && grid > max_grid) grid = max_grid;
    if (grid < 1) grid = 1;
    kern<<<grid, W * 32, smem, stream>>>(a);
    *grid_out = grid;
    return cudaGetLastError();
}

using LaunchFn = cudaError_t (*)(const TraceArgs &, unsigned, cudaStream_t, unsigned *, unsigned);
struct ShapeEntry {
    int precision, c, w, minb;
    LaunchFn fn;
};

// (cells per lane, warps per CTA, minimum resident CTAs per SM): the last one caps
// the registers per thread at 64K / (32 W MINB) and so trades ILP for occupancy.
#define RT_SHAPE(P, C, W, MB) {P, C, W, MB, &launch_shape<C, W, P, MB>}
const ShapeEntry kShapes[] = {
    RT_SHAPE(RT_FP32_KAHAN, 2, 4, 8),  RT_SHAPE(RT_FP32_KAHAN, 4, 4, 6),
    RT_SHAPE(RT_FP32_KAHAN, 4, 4, 8),  RT_SHAPE(RT_FP32_KAHAN, 8, 4, 4),
    RT_SHAPE(RT_FP32_KAHAN, 8, 4, 5),  RT_SHAPE(RT_FP32_KAHAN, 8, 4, 6),
    RT_SHAPE(RT_FP32_KAHAN, 16, 4, 2), RT_SHAPE(RT_FP32_KAHAN, 16, 4, 3),
    RT_SHAPE(RT_FP32_KAHAN, 4, 8, 4),  RT_SHAPE(RT_FP32_KAHAN, 8, 8, 2),
    RT_SHAPE(RT_FP32_KAHAN, 8, 8, 3),  RT_SHAPE(RT_FP32_PLAIN, 2, 4, 8),
    RT_SHAPE(RT_FP32_PLAIN, 4, 4, 6),  RT_SHAPE(RT_FP32_PLAIN, 8, 4, 4),
    RT_SHAPE(RT_FP32_PLAIN, 8, 8, 2),  RT_SHAPE(RT_FP64, 2, 4, 8),
    RT_SHAPE(RT_FP64, 4, 4, 4),        RT_SHAPE(RT_FP64, 8, 4, 2),
};
#undef RT_SHAPE

const ShapeEntry *find_shape(int precision, int c, int w, int mb)
{
    for (const ShapeEntry &s : kShapes)
        if (s.precision == precision && s.c == c && s.w == w && (mb == 0 || s.minb == mb)) return &s;
    return nullptr;
}

}  // namespace

int trace_shapes(int precision, Shape *out, int max_out)
{
    int n = 0;
    for (const ShapeEntry &s : kShapes)
        if (s.precision == precision && n < max_out) out[n++] = Shape{kKindTile, s.c, s.w, s.minb};
    return n;
}

long long trace_tile_cells(Shape s) { return 32LL * s.warps * s.cells_per_lane; }

cudaError_t launch_trace(int precision, Shape s, const TraceArgs &args, unsigned ntiles,
                         cudaStream_t stream, unsigned *grid_out, unsigned max_grid)
{
    if (s.kind == kKindRay || s.kind == kKindRayChunked)
        return launch_ray_shape(precision, s, args, stream, grid_out, max_grid);
    const ShapeEntry *e = find_shape(precision, s.cells_per_lane, s.warps, s.min_blocks);
    if (!e) return cudaErrorInvalidValue;
    return e->fn(args, ntiles, stream, grid_out, max_grid);
}

}  // namespace rt
