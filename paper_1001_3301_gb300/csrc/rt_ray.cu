// Warp-per-ray form of the frequency-dependent tracer (Kuiper et al. 2010,
// Sect. 2.2-2.3, 3.3.4), for grids whose rays fill most of 32 P C cells (P = 1 or 2
// warps per ray): the body of rt_ray.cuh over all rays of one grid, then the CTA's
// energy partial. Persistent: the grid holds (SMs x resident CTAs) CTAs that stride
// over the rays.
#include "rt_ray.cuh"

namespace rt {
namespace {

// The fewest lanes per ray that still hold the ray: 8, 16 or 32 (G C >= nr), else two
// warps per ray (ray_warps_per_ray).
template <int C, int W, int MODE, int MINB, bool TW = false, bool LUT = false>
cudaError_t launch_ray(const TraceArgs &a, unsigned, cudaStream_t stream, unsigned *grid_out, unsigned max_grid)
{
    if ((a.n_tw > 0) != TW || (a.lut != nullptr) != LUT) return cudaErrorInvalidValue;
    if (8 * C >= a.nr) return launch_ray_g<C, W, MODE, MINB, 8, 1, TW, LUT>(a, stream, grid_out, max_grid);
    if (16 * C >= a.nr) return launch_ray_g<C, W, MODE, MINB, 16, 1, TW, LUT>(a, stream, grid_out, max_grid);
    if (32 * C >= a.nr) return launch_ray_g<C, W, MODE, MINB, 32, 1, TW, LUT>(a, stream, grid_out, max_grid);
    if constexpr (C <= 8) {
        if (64 * C >= a.nr) return launch_ray_g<C, W, MODE, MINB, 32, 2, TW, LUT>(a, stream, grid_out, max_grid);
    }
    return cudaErrorInvalidValue;
}

struct RayEntry {
    int precision, c, w, minb;
    cudaError_t (*fn)(const TraceArgs &, unsigned, cudaStream_t, unsigned *, unsigned);
};

#define RT_RAY(P, C, W, MB) {P, C, W, MB, &launch_ray<C, W, P, MB>}
const RayEntry kRayShapes[] = {
    RT_RAY(RT_FP32_KAHAN, 2, 4, 8),  RT_RAY(RT_FP32_KAHAN, 4, 4, 8),  RT_RAY(RT_FP32_KAHAN, 6, 4, 8),
    RT_RAY(RT_FP32_KAHAN, 8, 4, 6),  RT_RAY(RT_FP32_KAHAN, 8, 4, 8),  RT_RAY(RT_FP32_KAHAN, 12, 4, 5),
    RT_RAY(RT_FP32_KAHAN, 16, 4, 3), RT_RAY(RT_FP32_KAHAN, 16, 4, 4), RT_RAY(RT_FP32_PLAIN, 4, 4, 8),
    RT_RAY(RT_FP32_PLAIN, 8, 4, 6),  RT_RAY(RT_FP32_PLAIN, 16, 4, 4),
};
// shapes compiled with the column weight of a separable kappa(nu, T) table
#define RT_RAYW(P, C, W, MB) {P, C, W, MB, &launch_ray<C, W, P, MB, true>}
const RayEntry kRayShapesTW[] = {
    RT_RAYW(RT_FP32_KAHAN, 4, 4, 8),  RT_RAYW(RT_FP32_KAHAN, 8, 4, 6), RT_RAYW(RT_FP32_KAHAN, 16, 4, 4),
    RT_RAYW(RT_FP32_PLAIN, 8, 4, 6),  RT_RAYW(RT_FP32_PLAIN, 16, 4, 4),
};
#undef RT_RAYW
// shapes compiled with the lookup-table comparator
#define RT_RAYL(P, C, W, MB) {P, C, W, MB, &launch_ray<C, W, P, MB, false, true>}
const RayEntry kRayShapesLUT[] = {
    RT_RAYL(RT_FP32_KAHAN, 4, 4, 8), RT_RAYL(RT_FP32_KAHAN, 8, 4, 6), RT_RAYL(RT_FP32_KAHAN, 16, 4, 4),
    RT_RAYL(RT_FP32_PLAIN, 8, 4, 6), RT_RAYL(RT_FP32_PLAIN, 16, 4, 4),
};
#undef RT_RAYL
#undef RT_RAY

}  // namespace

int ray_shapes(int precision, int nr, Shape *out, int max_out)
{
    int n = 0;
    for (const RayEntry &s : kRayShapes)
        if (s.precision == precision && ray_warps_per_ray(s.c, nr) > 0 && n < max_out)
            out[n++] = Shape{kKindRay, s.c, s.w, s.minb};
    return n;
}

int ray_shapes_tw(int precision, int nr, Shape *out, int max_out)
{
    int n = 0;
    for (const RayEntry &s : kRayShapesTW)
        if (s.precision == precision && ray_warps_per_ray(s.c, nr) > 0 && n < max_out)
            out[n++] = Shape{kKindRay, s.c, s.w, s.minb};
    return n;
}

int ray_shapes_lut(int precision, int nr, Shape *out, int max_out)
{
    int n = 0;
    for (const RayEntry &s : kRayShapesLUT)
        if (s.precision == precision && ray_warps_per_ray(s.c, nr) > 0 && n < max_out)
            out[n++] = Shape{kKindRay, s.c, s.w, s.minb};
    return n;
}

cudaError_t launch_ray_shape(int precision, Shape s, const TraceArgs &args, cudaStream_t stream,
                             unsigned *grid_out, unsigned max_grid)
{
    if (s.kind == kKindRayChunked) return launch_ray_mc_shape(precision, s, args, stream, grid_out, max_grid);
    const bool tw = args.n_tw > 0, lut = args.lut != nullptr;
    const RayEntry *tab = lut ? kRayShapesLUT : (tw ? kRayShapesTW : kRayShapes);
    const int ntab = lut  ? (int)(sizeof(kRayShapesLUT) / sizeof(RayEntry))
                     : tw ? (int)(sizeof(kRayShapesTW) / sizeof(RayEntry))
                          : (int)(sizeof(kRayShapes) / sizeof(RayEntry));
    for (int k = 0; k < ntab; ++k) {
        const RayEntry &e = tab[k];
        if (e.precision == precision && e.c == s.cells_per_lane && e.w == s.warps &&
            (s.min_blocks == 0 || e.minb == s.min_blocks) && ray_warps_per_ray(e.c, args.nr) > 0)
            return e.fn(args, 0, stream, grid_out, max_grid);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rt
