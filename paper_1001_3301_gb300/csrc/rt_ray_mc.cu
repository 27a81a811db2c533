// Chunked form of the warp-per-ray tracer (Kuiper et al. 2010, Sect. 2.2-2.3,
// 3.3.4; body in rt_ray.cuh): segments of 8 lanes (4 rays per warp) walk their rays
// outward in chunks of 8 C cells with the column carried, for rays longer than one
// chunk.
#include "rt_ray.cuh"

namespace rt {
namespace {

template <int C, int W, int MODE, int MINB>
cudaError_t launch_ray_mc(const TraceArgs &a, cudaStream_t stream, unsigned *grid_out, unsigned max_grid)
{
    if (a.n_tw > 0 || a.lut != nullptr || a.nr > kMaxChunkedNr) return cudaErrorInvalidValue;
    return launch_ray_g<C, W, MODE, MINB, 8, 1, false, false, true>(a, stream, grid_out, max_grid);
}

struct ChunkEntry {
    int precision, c, w, minb;
    cudaError_t (*fn)(const TraceArgs &, cudaStream_t, unsigned *, unsigned);
};

#define RT_RAYC(P, C, W, MB) {P, C, W, MB, &launch_ray_mc<C, W, P, MB>}
const ChunkEntry kRayShapesMC[] = {
    RT_RAYC(RT_FP32_KAHAN, 8, 4, 6),  RT_RAYC(RT_FP32_KAHAN, 16, 4, 3), RT_RAYC(RT_FP32_KAHAN, 16, 4, 4),
    RT_RAYC(RT_FP32_KAHAN, 16, 4, 5),
    RT_RAYC(RT_FP32_PLAIN, 8, 4, 6),  RT_RAYC(RT_FP32_PLAIN, 16, 4, 4),
};
#undef RT_RAYC

}  // namespace

// chunked shapes: rays longer than one chunk (8 C < nr), up to kMaxChunkedNr cells
int ray_shapes_mc(int precision, int nr, Shape *out, int max_out)
{
    int n = 0;
    for (const ChunkEntry &s : kRayShapesMC)
        if (s.precision == precision && 8 * s.c < nr && nr <= kMaxChunkedNr && n < max_out)
            out[n++] = Shape{kKindRayChunked, s.c, s.w, s.minb};
    return n;
}

cudaError_t launch_ray_mc_shape(int precision, Shape s, const TraceArgs &args, cudaStream_t stream,
                                unsigned *grid_out, unsigned max_grid)
{
    for (const ChunkEntry &e : kRayShapesMC)
        if (e.precision == precision && e.c == s.cells_per_lane && e.w == s.warps &&
            (s.min_blocks == 0 || e.minb == s.min_blocks) && 8 * e.c < args.nr)
            return e.fn(args, stream, grid_out, max_grid);
    return cudaErrorInvalidValue;
}

}  // namespace rt
