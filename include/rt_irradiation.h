/*
 * rt_irradiation.h -- C ABI of the GB300 (sm_103a) frequency-dependent
 * first-order stellar irradiation ray tracer.
 *
 * The library computes, for a central star irradiating a spherical (r, theta, phi)
 * grid along radial rays, the absorbed stellar power per unit volume q_abs and the
 * radial radiative acceleration a_rad of every cell, following Kuiper et al. (2010):
 *   Sect. 2.2, Eqs. 17-19   F(r) = F(R_s) (R_s/r)^2 exp(-tau(r)), tau = int kappa rho dr,
 *                           tau = 0 at the inner grid radius;
 *   Sect. 2.3, Eq. 20       a fixed set of frequency bins, each with its own opacity
 *                           kappa(nu_i) and its own Planck-band stellar flux;
 *   Sect. 3.3.4, Eqs. 27-36 cell-integrated absorption F_in (1 - exp(-dtau)) in the
 *                           cancellation-free expm1 form; the geometric dilution does
 *                           not contribute (Eq. 36);
 *   Sect. 5                 a_rad = -div(F_s) / (rho c), radial.
 * Dust above the sublimation temperature t_sub has no opacity (Sect. 2: evaporated
 * dust leaves an optically thin region).
 *
 * Conventions
 *  - Units are cgs: cm, g, s, K, Hz; q_abs in erg s^-1 cm^-3; a_rad in cm s^-2.
 *  - Fields are float32 arrays of nphi * ntheta * nr elements in the layout
 *    [nphi][ntheta][nr], r fastest (one radial ray is one contiguous run of nr).
 *  - "device" pointers are CUDA global-memory addresses on the current device
 *    (e.g. torch.Tensor.data_ptr()); "host" pointers are CPU addresses.
 *  - Every call returns RT_OK (0) or a negative RT_ERR_* status; no C++ exception
 *    crosses this interface. rt_last_error() gives the text of the last failure of
 *    a context, rt_status_string() the name of a status.
 *  - Work is enqueued asynchronously on the context's CUDA stream. A call that
 *    returns results to the host (energy, host-buffer variants) synchronises that
 *    stream before it returns.
 *  - The caller owns every field buffer; the library owns the context, the
 *    per-grid tables and every scratch buffer it allocates.
 *  - A context must not be used from two host threads at once.
 */
#ifndef RT_IRRADIATION_H
#define RT_IRRADIATION_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define RT_OK                   0
#define RT_ERR_INVALID_ARG     (-1)  /* bad size, pointer, non-monotone grid, ...    */
#define RT_ERR_NOT_CONFIGURED  (-2)  /* star or opacity table not set yet            */
#define RT_ERR_CUDA            (-3)  /* a CUDA runtime call failed (see last_error)  */
#define RT_ERR_TIMEOUT         (-4)  /* a bounded device wait gave up                */
#define RT_ERR_NONFINITE_INPUT (-5)  /* NaN/Inf/negative density or NaN temperature  */
#define RT_ERR_NO_MEMORY       (-6)  /* host or device allocation failed             */

/* ---- precision of the optical-depth scan and of the per-bin arithmetic --- */
#define RT_FP32_KAHAN 0  /* FP32 bins; column density scanned in compensated
                            (double-float) FP32 and carried across tiles in the
                            same form. The default. In both FP32 modes the
                            warp-per-ray kernel sums the bins optically thin along
                            all rays of a warp (kappa_i N_total <= 1/2) as one
                            power series in the column, truncated below 1e-7 of
                            the value, instead of bin by bin. */
#define RT_FP32_PLAIN 1  /* FP32 bins; plain FP32 running sum (precision study) */
#define RT_FP64       2  /* FP64 scan and FP64 per-bin arithmetic (libm-grade exp
                            and expm1); outputs still rounded to float32 */

#define RT_MAX_NU 128    /* largest number of frequency bins per table */

typedef struct rt_ctx rt_ctx;

/* Grid description. All arrays are copied by rt_create; the caller may free them. */
typedef struct rt_grid_desc {
    int nr, ntheta, nphi;   /* cells per direction, each >= 1                      */
    const double *r_if;     /* [nr+1] radial interfaces, strictly increasing, r_if[0] > 0 */
    const double *theta_if; /* [ntheta+1] polar interfaces in [0, pi], strictly increasing */
    const double *phi_if;   /* [nphi+1] azimuthal interfaces, strictly increasing;
                               with nphi == 1 the span may be 2 pi (axisymmetric)   */
    int precision;          /* RT_FP32_KAHAN, RT_FP32_PLAIN or RT_FP64              */
} rt_grid_desc;

/* Energy bookkeeping of one rt_irradiate call (Eqs. 33-35: the flux difference
 * telescopes along a ray, so absorbed + escaped = emitted). */
typedef struct rt_energy {
    double e_abs;   /* sum over cells of q_abs * V (erg/s), from the kernel's own sums */
    double e_esc;   /* power leaving the outer radial boundary (erg/s)                */
    double l_star;  /* R_s^2 sigma T_s^4 sum_j dOmega_j: the stellar luminosity into the
                       grid's solid angle (= 4 pi R_s^2 sigma T_s^4 on the full sphere)  */
    double rel_err; /* (e_abs + e_esc) / l_star - 1                                  */
} rt_energy;

/* rt_create -- allocate a context for one grid (geometry of Sect. 2.2: radial rays
 * along the r axis of a spherical grid; one ray per (theta, phi) column).
 *   g            grid description (copied).
 *   cuda_stream  cudaStream_t to enqueue work on; NULL = the legacy default stream.
 *   out          receives the new context; *out is NULL on failure.
 * Errors: RT_ERR_INVALID_ARG (sizes < 1, non-increasing or non-positive radii,
 * theta outside [0, pi], unknown precision), RT_ERR_CUDA, RT_ERR_NO_MEMORY. */
int rt_create(const rt_grid_desc *g, void *cuda_stream, rt_ctx **out);

/* rt_set_stream -- change the CUDA stream later calls enqueue on. */
int rt_set_stream(rt_ctx *ctx, void *cuda_stream);

/* rt_set_opacity_table -- the frequency bins of Sect. 2.3.
 *   n_nu        1..RT_MAX_NU bins.
 *   nu_mid      [n_nu] host, bin mid-frequencies (Hz), strictly increasing, > 0. Bin
 *               edges are the arithmetic midpoints (nu_{i-1}+nu_i)/2 of Eq. 20; the
 *               first bin starts at 0 Hz and the last ends at infinity.
 *   kappa       [n_nu] host, absorption opacity per bin (cm^2 g^-1), finite, >= 0.
 *   t_sub       dust sublimation temperature (K): a cell with t_dust > t_sub has
 *               zero opacity in every bin; t_dust == t_sub keeps its dust.
 *   kappa_bf16  non-zero: round each kappa to bfloat16 before use (precision study).
 * The Planck-band fluxes are (re)computed on the device once the star is also set.
 * Errors: RT_ERR_INVALID_ARG, RT_ERR_CUDA. */
int rt_set_opacity_table(rt_ctx *ctx, int n_nu, const double *nu_mid, const double *kappa,
                         double t_sub, int kappa_bf16);

/* rt_set_opacity_table_t -- temperature-dependent opacities (an extension the
 * paper's tabulated dust opacities allow): kappa_t [n_nu][n_t] (cm^2 g^-1, >= 0,
 * row-major, bin-major) on the strictly increasing temperature grid t_grid [n_t]
 * (K, 2 <= n_t <= 32); a cell's kappa of bin i is row i linear in T between the
 * bracketing grid points (the end values beyond the grid), zero where
 * T_dust > t_sub. The optical depth of every bin is then its own scan along the
 * ray (Eq. 19), traced by a separate warp-per-ray kernel (nr <= 1024). A table
 * whose rows are one spectral shape times one temperature factor,
 * kappa_i(T_j) = kappa_i b_j for every entry to 1e-12 (one dust species whose
 * abundance depends on T), keeps the single column of the temperature-independent
 * tracer instead, each cell's column weighted by b(T) (FP32 precisions, rays up to
 * 512 cells). A table of rank two with non-negative factors, every entry a
 * non-negative combination of two of the table's own columns to 1e-10 of itself
 * (two species whose abundances depend on T), is traced with two columns per ray
 * (kappa_i(T) = A_i1 b_1(T) + A_i2 b_2(T); FP32 precisions, nr <= 1024). A table of
 * rank three or four (three or four species), whose leading singular vectors reproduce
 * every entry to 1e-10 of its row's largest value, is traced the same way with that
 * many columns (factors of either sign).
 * rt_opacity_table_kind reports which kernel serves the table. The
 * temperature-independent entry rt_set_opacity_table switches back. Not
 * available to the multi-grid batch or the learned surrogate (their calls fail
 * with RT_ERR_INVALID_ARG); rt_planck_mean_opacity / rt_dust_temperature use
 * kappa_i(T). Host arrays, copied. */
int rt_set_opacity_table_t(rt_ctx *ctx, int n_nu, const double *nu_mid, int n_t, const double *t_grid,
                           const double *kappa_t, double t_sub);

/* rt_set_star -- the central black-body star (Eqs. 18 and 20).
 *   t_star  effective temperature (K), > 0;  r_star  radius (cm), > 0.
 * Bin fluxes F_i = pi * int B_nu(T_s) dnu over each bin (sum_i F_i = sigma T_s^4) are
 * computed on the device in FP64. Errors: RT_ERR_INVALID_ARG, RT_ERR_CUDA. */
int rt_set_star(rt_ctx *ctx, double t_star, double r_star);

/* rt_opacity_table_kind -- how the configured table is traced: RT_TABLE_NU (kappa per
 * bin, one column for every bin), RT_TABLE_NU_T_SEPARABLE (a temperature-dependent
 * table that separates: the same single column, weighted per cell by b(T)),
 * RT_TABLE_NU_T_RANK2 (a table of rank two: two columns per ray),
 * RT_TABLE_NU_T_LOW_RANK (rank three or four: that many columns per ray), RT_TABLE_NU_T
 * (one scan per bin). Errors: RT_ERR_INVALID_ARG, RT_ERR_NOT_CONFIGURED. */
#define RT_TABLE_NU             0
#define RT_TABLE_NU_T_SEPARABLE 1
#define RT_TABLE_NU_T           2
#define RT_TABLE_NU_T_RANK2     3
#define RT_TABLE_NU_T_LOW_RANK  4
int rt_opacity_table_kind(const rt_ctx *ctx, int *kind);

/* rt_irradiate -- trace every ray of the grid (Eqs. 17-20, 27-36).
 *   rho       device [nphi][ntheta][nr] gas density (g cm^-3), >= 0 and finite.
 *   t_dust    device, same layout, dust temperature (K).
 *   q_abs     device, same layout, caller-allocated: absorbed stellar power per
 *             volume (erg s^-1 cm^-3), i.e. -div(F_s), the source term of Eq. 15.
 *   a_rad     device, same layout, caller-allocated: radial radiative acceleration
 *             (cm s^-2) = q_abs / (rho c) for rho > 0, and its rho -> 0 limit
 *             sum_i kappa_i F_i,in / c (cell-averaged) where rho == 0; 0 where the
 *             dust is sublimated.
 *   energy    NULL, or a host struct to receive the call's energy sums; when given
 *             the call synchronises the stream.
 * q_abs and a_rad are fully overwritten; inputs are only read. Input and output
 * buffers must not overlap. Invalid input values (NaN/Inf/negative rho, NaN t_dust)
 * are flagged on the device, never trapped: the call that requests energy (or
 * rt_energy_last) returns RT_ERR_NONFINITE_INPUT if the traced fields held any.
 * Errors: RT_ERR_NOT_CONFIGURED, RT_ERR_INVALID_ARG (NULL field), RT_ERR_CUDA,
 * RT_ERR_NONFINITE_INPUT (only when energy != NULL). */
int rt_irradiate(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs,
                 float *a_rad, rt_energy *energy);

/* rt_irradiate_host -- as rt_irradiate, with HOST buffers of the same layout. The
 * library copies rho and t_dust to device buffers it owns (allocated on first use,
 * freed by rt_destroy), traces, and copies q_abs and a_rad back before it returns.
 * Page-locked host memory makes the copies asynchronous DMA; pageable memory works
 * but is slower. Errors: as rt_irradiate, plus RT_ERR_NO_MEMORY. */
int rt_irradiate_host(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs,
                      float *a_rad, rt_energy *energy);

/* rt_irradiate_host_async -- rt_irradiate_host without the wait: the copies in, the
 * trace and the copies out are enqueued and the call returns, so that the calls of
 * several contexts overlap on the link. The host buffers must stay untouched (rho,
 * t_dust) and unread (q_abs, a_rad) until rt_host_wait(ctx) returns. One call is in
 * flight per context: a new host call on the context first waits for the previous
 * one (and returns its RT_ERR_NONFINITE_INPUT, if any). Errors: as
 * rt_irradiate_host, except that invalid input is reported by rt_host_wait. */
int rt_irradiate_host_async(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs, float *a_rad);

/* rt_host_wait -- wait until the last rt_irradiate_host_async of the context has
 * copied its outputs back; RT_ERR_NONFINITE_INPUT if its input fields held invalid
 * values. RT_OK at once if no asynchronous call is pending. */
int rt_host_wait(rt_ctx *ctx);

/* rt_energy_last -- energy sums of the most recent trace on this context (runs the
 * FP64 reduction of its per-tile partial sums, synchronises the stream).
 * Errors: RT_ERR_NOT_CONFIGURED (nothing traced yet), RT_ERR_CUDA,
 * RT_ERR_NONFINITE_INPUT (that trace saw invalid input; *out is still filled). */
int rt_energy_last(rt_ctx *ctx, rt_energy *out);

/* rt_energy_reduce -- enqueue, on the context's stream, the FP64 reduction of the
 * most recent trace's per-tile partial sums into the energy sums E_abs, E_esc and
 * their balance against L* (Eqs. 33-35; Eq. 18 for L*), kept in device memory the
 * context owns; no synchronisation, nothing is returned to the host. A step that
 * needs the energy on the device every time and on the host only now and then
 * calls this after rt_irradiate and rt_energy_last when it reads them (which runs
 * the same reduction again). Errors: RT_ERR_NOT_CONFIGURED (nothing traced yet),
 * RT_ERR_CUDA. */
int rt_energy_reduce(rt_ctx *ctx);

/* rt_get_bins -- copy the per-bin stellar surface fluxes F_i (erg s^-1 cm^-2, FP64,
 * Eq. 20) that the device computed for the current star and table into host
 * f_bin[n_nu]. Synchronises. Errors: RT_ERR_NOT_CONFIGURED, RT_ERR_CUDA. */
int rt_get_bins(rt_ctx *ctx, double *f_bin);

/* Tracer kernels. RT_KERNEL_TILE: the flattened ray array in tiles of
 * 32 * warps * cells_per_lane cells, any nr (rays straddle threads and tiles).
 * RT_KERNEL_RAY: one warp per ray, each lane cells_per_lane consecutive cells of
 * it; only for nr <= 32 * cells_per_lane. RT_KERNEL_RAY_CHUNKED: 8 lanes per ray
 * (4 rays per warp) walk each ray outward in chunks of 8 * cells_per_lane cells,
 * the column carried from chunk to chunk; for 8 * cells_per_lane < nr <= 4096,
 * the plain (temperature-independent) table and the FP32 modes. The FP64 mode
 * always uses tiles. */
#define RT_KERNEL_TILE        0
#define RT_KERNEL_RAY         1
#define RT_KERNEL_RAY_CHUNKED 2

/* rt_set_tuning -- force the tracer kernel and its launch shape: kind
 * (RT_KERNEL_TILE, RT_KERNEL_RAY or RT_KERNEL_RAY_CHUNKED), cells_per_lane, warps_per_block and
 * min_blocks_per_sm (the resident CTAs per SM the registers are capped for; 0 =
 * the first compiled variant). cells_per_lane = warps_per_block = 0 restores
 * automatic choice. Shapes that are not compiled in or do not fit the grid return
 * RT_ERR_INVALID_ARG. rt_get_tuning reports the shape in use; rt_list_tunings
 * writes the shapes that apply to this context's grid and precision (up to max of
 * them) into the four arrays and returns their number (negative status on error). */
int rt_set_tuning(rt_ctx *ctx, int kind, int cells_per_lane, int warps_per_block,
                  int min_blocks_per_sm);
int rt_get_tuning(const rt_ctx *ctx, int *kind, int *cells_per_lane, int *warps_per_block,
                  int *min_blocks_per_sm);
int rt_list_tunings(const rt_ctx *ctx, int *kinds, int *cells_per_lane, int *warps_per_block,
                    int *min_blocks_per_sm, int max);

/* rt_autotune -- time every applicable kernel and launch shape on the given device buffers
 * (same meaning as rt_irradiate; q_abs and a_rad are overwritten), keep the fastest
 * for this context and remember it for grids of the same shape class in this
 * process. reps >= 1 timed calls per shape. Synchronises. Errors: as rt_irradiate. */
int rt_autotune(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs,
                float *a_rad, int reps);

/* rt_destroy -- free the context and everything it owns (NULL is ignored). Work
 * still queued on the stream is waited for first. */
void rt_destroy(rt_ctx *ctx);

/* rt_last_error -- text of the last failure on ctx (never NULL; "" if none). With
 * ctx == NULL: the last failure of rt_create in this thread. */
const char *rt_last_error(const rt_ctx *ctx);

/* rt_status_string -- constant name of a status code. */
const char *rt_status_string(int status);

/* ---- many grids in one launch --------------------------------------------- */

#define RT_BATCH_MAX 256  /* contexts per batch */

typedef struct rt_batch rt_batch;

/* rt_batch_create -- plan one persistent launch over several grids of any size
 * (each a configured context; all of one precision and one device; each below
 * 2^31 - 2^16 flattened cells). With tile shapes the grids' tiles are
 * concatenated and split over the CTAs by cost (tiles weighted by the grid's bin
 * count); with warp-per-ray shapes the CTAs take chunks of rays from a counter at
 * run time. The launch, a reset of the energy partials (and of the counter) and a
 * per-grid FP64 energy reduction are built into a CUDA graph once. The contexts must outlive the batch and must not be reconfigured
 * while it exists (re-create the batch after rt_set_star/rt_set_opacity_table).
 *   ctxs  [n] contexts, n in 1..RT_BATCH_MAX;  cuda_stream  the stream runs use.
 * Errors: RT_ERR_INVALID_ARG, RT_ERR_NOT_CONFIGURED, RT_ERR_CUDA, RT_ERR_NO_MEMORY;
 * failure text via rt_last_error(NULL). */
int rt_batch_create(rt_ctx *const *ctxs, int n, void *cuda_stream, rt_batch **out);

/* rt_batch_run -- trace every grid of the batch (the semantics of rt_irradiate
 * per grid). rho[g], t_dust[g], q_abs[g], a_rad[g]: device fields of grid g, layout
 * as in rt_irradiate. One graph replay on the batch's stream; does not
 * synchronise. Errors: RT_ERR_INVALID_ARG (NULL pointer), RT_ERR_CUDA. */
int rt_batch_run(rt_batch *b, const float *const *rho, const float *const *t_dust,
                 float *const *q_abs, float *const *a_rad);

/* rt_batch_energy -- the energy sums of every grid of the last run into host
 * energies[n]; synchronises. RT_ERR_NONFINITE_INPUT if any field held invalid
 * values (energies are still filled). */
int rt_batch_energy(rt_batch *b, rt_energy *energies);

/* rt_batch_autotune -- time every compiled shape of the batch's precision on the
 * given fields (overwriting q_abs and a_rad), keep the fastest and rebuild the
 * graph. reps >= 1. Synchronises. The shapes are tiles of the flattened grids
 * (RT_KERNEL_TILE, any nr) and, where every grid has nr <= 32 cells_per_lane,
 * warp-per-ray bodies (RT_KERNEL_RAY; 8, 16 or 32 lanes per ray chosen per grid).
 * rt_batch_get_tuning reports the shape in use; rt_batch_set_tuning selects one
 * (RT_ERR_INVALID_ARG if no such shape is compiled for the batch's precision or a
 * grid's rays do not fit it; min_blocks_per_sm 0 = any) and rebuilds the graph. */
int rt_batch_autotune(rt_batch *b, const float *const *rho, const float *const *t_dust,
                      float *const *q_abs, float *const *a_rad, int reps);
int rt_batch_get_tuning(const rt_batch *b, int *kind, int *cells_per_lane, int *warps_per_block,
                        int *min_blocks_per_sm);
int rt_batch_set_tuning(rt_batch *b, int kind, int cells_per_lane, int warps_per_block, int min_blocks_per_sm);

/* rt_batch_last_error -- text of the batch's last failure ("" if none). */
const char *rt_batch_last_error(const rt_batch *b);

/* rt_batch_destroy -- wait for the batch's stream, free the batch (NULL ignored). */
void rt_batch_destroy(rt_batch *b);

/* ---- lookup-table comparator (no counterpart in the paper) ----------------- */

/* rt_lut_build -- build the context's lookup table for the per-bin sum (a
 * non-learned comparator of the learned surrogate). With kappa depending on the
 * frequency only, the power a cell absorbs over all bins, sum_i F_i e^{-kappa_i N_in}
 * (1 - e^{-kappa_i dN}) (Eqs. 17, 28-32, 36 summed over the bins of Sect. 2.3), is a
 * function of the column in front of the cell and of its own column. The table holds
 * log2 of that sum per unit kappa_ref dN on a grid of s = log2(kappa_ref N_in +
 * 2^-20) in [-20, 8] and d = log2(kappa_ref dN + 2^-30) in [-30, 8], steps 1/32
 * (897 x 1217 pairs of floats, 8.7 MB of device memory the context owns), computed in FP64
 * from the tracer's bin table; kappa_ref is the flux-weighted mean opacity. Each grid
 * square whose bilinear interpolation is off by more than err_tol / 2 at its centre
 * or an edge midpoint is flagged. Rebuild after rt_set_star / rt_set_opacity_table.
 * Only for temperature-independent tables in the FP32 precisions. Synchronises.
 * Errors: RT_ERR_NOT_CONFIGURED, RT_ERR_INVALID_ARG, RT_ERR_NO_MEMORY, RT_ERR_CUDA. */
int rt_lut_build(rt_ctx *ctx, float err_tol);

/* rt_irradiate_lut -- rt_irradiate with the per-bin sum of every cell taken from the
 * lookup table (bilinear in log2; rays of at most 512 cells). A warp of rays that
 * holds a cell in a flagged square or off the table computes the per-bin sum
 * instead. The escaping power and the rho -> 0 force limit stay exact. The result is
 * within about err_tol of rt_irradiate per cell (not within the tracer's 1e-5), and
 * so is the energy. fallback_slots, if not NULL, receives the number of warp-slots
 * that took the per-bin sum (the call then synchronises). Arguments and errors as
 * rt_irradiate, plus RT_ERR_NOT_CONFIGURED (no table for the current configuration)
 * and RT_ERR_INVALID_ARG (rays longer than 512 cells). */
int rt_irradiate_lut(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs, float *a_rad,
                     rt_energy *energy, unsigned *fallback_slots);

/* ---- allocation-free form (no counterpart in the paper) -------------------- */

/* Limits of rt_irradiate_static: its scratch is one fixed device array of about
 * 1.9 MB that every GPU loading this library holds until the process exits. */
#define RT_STATIC_MAX_NR     1024
#define RT_STATIC_MAX_NTHETA 8192
#define RT_STATIC_MAX_NPHI   8192
#define RT_STATIC_MAX_RAYS   131072   /* ntheta * nphi */

/* rt_irradiate_static -- the whole trace in one call that allocates no memory.
 *
 * For callers that cannot allocate device memory when they need the irradiation:
 * host codes whose own pool allocator has already reserved the GPU, or time loops
 * in which cudaMalloc/cudaFree (both synchronise the device) would stall other
 * work. Instead of a context (rt_create allocates), everything is passed in and
 * every intermediate lives in one file-scope device array of fixed size.
 *   g, t_star, r_star, n_nu, nu_mid, kappa, t_sub, kappa_bf16
 *       as for rt_create, rt_set_star and rt_set_opacity_table (host memory);
 *       additionally nr <= RT_STATIC_MAX_NR, ntheta <= RT_STATIC_MAX_NTHETA,
 *       nphi <= RT_STATIC_MAX_NPHI and ntheta * nphi <= RT_STATIC_MAX_RAYS;
 *       larger grids are rejected with RT_ERR_INVALID_ARG (use rt_irradiate).
 *   rho, t_dust, q_abs, a_rad, energy
 *       as for rt_irradiate (device fields owned by the caller; energy may be NULL).
 *   cuda_stream
 *       the stream to work on (NULL = legacy default stream).
 * No cudaMalloc, cudaFree or allocating library call is made. The call copies the
 * grid and bin arrays into the array, runs the set-up kernels, reads back a few
 * scalars (so it synchronises the stream), then launches the tracer; with energy
 * it synchronises again. The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any stream
 * capture. Every call uses the same array and leaves its contents behind: calls
 * whose work overlaps on the GPU (other streams, other host threads) race with
 * each other; calls on one stream are ordered. Errors as rt_create and
 * rt_irradiate; the failure text is rt_last_error(NULL). */
int rt_irradiate_static(const rt_grid_desc *g, double t_star, double r_star, int n_nu,
                        const double *nu_mid, const double *kappa, double t_sub, int kappa_bf16,
                        const float *rho, const float *t_dust, float *q_abs, float *a_rad,
                        rt_energy *energy, void *cuda_stream);

/* ---- diagnostics (no counterpart in the paper) ---------------------------- */

/* ------------------------------------------------------------------------
 * Planck-mean opacity and the dust temperature (Sect. 2.2, Eq. 16).
 * ------------------------------------------------------------------------ */

/* rt_planck_mean_opacity -- kappa_P(T) = sum_i kappa_i B_i(T) / sum_i B_i(T) of the
 * context's table, B_i(T) the Planck integral over bin i (the bin edges of Eq. 20)
 * at temperature t (K, > 0), in FP64 on the device. kappa_P(T_star) is the gray
 * opacity of Eq. 19: a one-bin table with that kappa gives the gray irradiation.
 * Synchronises the context's stream. */
int rt_planck_mean_opacity(rt_ctx *ctx, double t, double *kappa_p);

/* rt_dust_temperature -- Eq. 16 with the frequency-dependent fluxes: per cell the
 * dust temperature T with
 *     a T^4 = E_R + sum_i kappa_i F_i / (c kappa_P(T))  =  E_R + a_rad / kappa_P(T),
 * since over a cell sum_i kappa_i F_i = q_abs / rho = c a_rad.
 *   a_rad   device, [nphi][ntheta][nr] FP32, the rt_irradiate output (cm s^-2);
 *   e_rad   device, same layout, the radiation energy density E_R of the diffuse
 *           field (erg cm^-3), or NULL for E_R = 0;
 *   t_dust  device, same layout, receives T (K); 0 where a_rad = E_R = 0.
 * kappa_P(T) is tabulated for the context's table on 1 K .. 1e5 K (1024 points of
 * ln T, cubic interpolation) and held constant outside; the root is found by
 * Newton's method on ln T in FP32. Asynchronous on the context's stream (the first
 * call per table builds the table and synchronises). */
int rt_dust_temperature(rt_ctx *ctx, const float *a_rad, const float *e_rad, float *t_dust);

/* ------------------------------------------------------------------------
 * Flux-limited diffusion of the re-emitted radiation (Sect. 2.1, Eqs. 7-15).
 * ------------------------------------------------------------------------ */

/* rt_rosseland_mean_opacity -- kappa_R(T) with 1/kappa_R = sum_i w_i / kappa_i /
 * sum_i w_i, w_i the integral of dB_nu/dT over bin i (the bin edges of Eq. 20), at
 * temperature t (K, > 0), in FP64 on the device; 0 if a bin with weight has
 * kappa_i = 0. The opacity of Eqs. 10-13. Synchronises the context's stream. */
int rt_rosseland_mean_opacity(rt_ctx *ctx, double t, double *kappa_r);

typedef struct rt_fld_stats {
    int iterations;      /* conjugate-gradient iterations taken, all passes */
    int passes;          /* refinement passes */
    double rel_change;   /* max over cells of |correction| / |E'| of the last pass */
    int levels;          /* multigrid levels of the preconditioner (1: Jacobi) */
} rt_fld_stats;

/* rt_fld_step -- one backward-Euler step of Eqs. 8-15,
 *     (E' - E) / dt = f_c (div(D grad E') + q_abs),
 *     f_c = 1 / (c_v rho / (4 a T^3) + 1),                                (Eq. 9)
 *     D = lambda c / (kappa_R rho), lambda = (2 + R) / (6 + 3 R + R^2),
 *     R = |grad E| / (kappa_R rho E),                                      (Eqs. 10-13)
 * with D, f_c and kappa_R(T) taken at the old state (kappa_R of the context's
 * table, on 1 K .. 1e5 K, held constant outside) and D = c (2 s + g) /
 * (6 s^2 + 3 s g + g^2), s = kappa_R rho, g = |grad E| / E, so that D stays finite
 * as rho -> 0 (D = 0 where s = g = 0).
 *   rho, t_gas  device [nphi][ntheta][nr] FP32: density (g cm^-3, >= 0) and gas =
 *               dust temperature (K, > 0);
 *   q_abs       device, same layout: the absorbed stellar power per volume
 *               (erg s^-1 cm^-3, >= 0; the rt_irradiate output), the source of Eq. 15;
 *   e_old       device, same layout: E_R at the start of the step (erg cm^-3, >= 0);
 *   e_new       device, same layout, caller-allocated, not aliasing e_old: E_R after it;
 *   dt (s) > 0 (1e300 gives the steady state), c_v (erg g^-1 K^-1) >= 0,
 *   t_bg (K) >= 0: E = a t_bg^4 half a cell beyond the outer radius;
 *   tol > 0, max_iter >= 1: mixed-precision iterative refinement (true residual in
 *   FP32, conjugate gradients for each correction, FP64 reductions) from
 *   E' = E_old until a pass changes no cell by more than tol relative, or max_iter
 *   conjugate-gradient iterations in total. Grids of more than 512 cells are
 *   preconditioned by an aggregation-multigrid V-cycle (Galerkin coarse levels
 *   halving every direction), smaller ones by Jacobi.
 *   stats       NULL or a host struct: iterations, refinement passes, the last
 *               pass's relative change and the number of multigrid levels.
 * Finite volumes: harmonic-mean face coefficients, no flux through the inner radius
 * or the theta ends, periodic in phi when nphi > 1 (the wrap distance measured
 * around the full circle). Runs on a private stream ordered after the context's
 * stream and synchronises it every 8 iterations; returns with e_new complete. Errors:
 * RT_ERR_NOT_CONFIGURED, RT_ERR_INVALID_ARG, RT_ERR_NONFINITE_INPUT (rho < 0,
 * T <= 0, E_old < 0, q_abs < 0 or NaN/Inf; e_new is then unchanged),
 * RT_ERR_TIMEOUT (tol not reached in max_iter; e_new holds the last iterate),
 * RT_ERR_NO_MEMORY, RT_ERR_CUDA. */
int rt_fld_step(rt_ctx *ctx, const float *rho, const float *t_gas, const float *q_abs, const float *e_old,
                float *e_new, double dt, double c_v, double t_bg, double tol, int max_iter, rt_fld_stats *stats);

/* ------------------------------------------------------------------------
 * Learned surrogate of the per-bin sum of one cell.
 *
 * Along a ray the tracer gives a cell with dust column N_in in front of it and
 * dust column dN of its own the absorbed share
 *     acc = sum_i (F_i / F_max) exp(-kappa_i N_in) (1 - exp(-kappa_i dN))
 * of the power R*^2 F_max dOmega entering the ray (Sect. 2.3, Eqs. 17, 28-32, 36).
 * The surrogate is an 8 -> 128 -> 128 -> 1 SiLU network whose inputs are
 *     x_m = log2(kappa_m N_in + 2^-20) / 16   (m = 0..5: the bins nearest 1e11,
 *                                              1e12, ..., 1e16 Hz in |ln nu|),
 *     x_6 = T_dust / 1000 - 0.8,
 *     x_7 = log2(kappa_550 dN + 2^-30) / 16   (the bin nearest 550 nm),
 * and whose output y gives g = acc / (kappa_550 dN) by ln g = mu + sigma y. Then
 * q_abs = Gq g kappa_550 dN and a_rad = q_abs / (rho c) = Gq (dr / c) g kappa_550.
 * BF16 weights with FP32 accumulation on the tensor cores: W1, b1 and W2 in BF16,
 * b2, w3 and b3 in FP32; inputs and first-layer activations reach the tensor core
 * as sums of BF16 parts, so they keep FP32-like precision.
 *
 * A surrogate belongs to one context and is valid for the opacity table,
 * sublimation temperature and stellar temperature it was made with (other grids
 * and stellar radii are fine: the inputs and output do not depend on them).
 * ------------------------------------------------------------------------ */
#define RT_SUR_NPARAMS 17793   /* W1 [8][128], b1 [128], W2 [128][128], b2 [128], w3 [128], b3 */

typedef struct {
    long long n_samples;  /* training cells drawn from the grids; <= 0: 20,000,000 */
    int batch;            /* minibatch rows, a multiple of 256; <= 0: 8192 */
    int steps;            /* Adam steps (warm-up, then cosine decay); <= 0: 30000 */
    float lr;             /* peak learning rate; <= 0: 2e-3 */
    unsigned long long seed;
} rt_train_cfg;

typedef struct {
    long long n_train, n_val;  /* cells collected for training / held out */
    double mu, sigma;          /* standardisation of ln g */
    double final_loss;         /* mean minibatch loss of the last 1 % of steps (standardised units) */
    double val_rms, val_max;   /* error of ln g on the held-out cells (to first order the
                                  relative error of q_abs), inference arithmetic */
    double train_ms;           /* device time of the optimisation loop */
} rt_train_stats;

typedef struct {
    long long n_dust;      /* cells with dust (T_dust <= t_sub) */
    long long n_fallback;  /* of those, answered by the exact per-bin sum */
    long long n_judged;    /* validate == 1: cells absorbing more than 1e-12 of L* */
    double max_rel_err;    /* validate == 1: largest |q_net / q_exact - 1| over judged cells (before fallback) */
    double mean_rel_err;   /* validate == 1: its mean */
    double e_abs, e_esc, rel_err;  /* energy of the returned fields, as in rt_energy */
} rt_surrogate_stats;

/* rt_surrogate_train -- train the context's surrogate on cells of `ngrids` density
 * and temperature fields of this context's grid (device pointers, the layout of
 * rt_irradiate). The exact tracer (rt_irradiate) traces every field; cells with
 * dust that absorb more than 1e-12 of L* are sampled (a counter hash of cfg->seed
 * and the cell; 2-5 % held out), and the network is trained on the GPU by the
 * library's forward, backward and Adam kernels. Deterministic for a given input.
 * Replaces any previous surrogate of the context. Synchronises the stream.
 * Errors: RT_ERR_INVALID_ARG (no opacity at 550 nm, fewer than 1024 usable cells,
 * bad cfg), RT_ERR_NOT_CONFIGURED, RT_ERR_NO_MEMORY, RT_ERR_CUDA. */
int rt_surrogate_train(rt_ctx *ctx, const rt_train_cfg *cfg, const float *const *rho,
                       const float *const *t_dust, int ngrids, rt_train_stats *stats_or_null);

/* rt_irradiate_surrogate -- rt_irradiate with the surrogate in place of the per-bin
 * loop. rho, t_dust, q_abs, a_rad as in rt_irradiate (fully overwritten).
 *   validate == 0  a trust map over (log2 tau_550 in front of the cell,
 *                  log2 dtau_550 of the cell), built on first use for `err_tol`
 *                  by judging 32 points per bin against the exact per-bin sum,
 *                  decides per cell; cells outside it take the exact sum.
 *   validate == 1  the exact tracer runs first and judges every cell; cells whose
 *                  q_abs differs by more than err_tol (relative) take the exact values.
 *   validate == 2  the network everywhere (no gate; for tests).
 * Cells without dust get q_abs = a_rad = 0 exactly. Asynchronous on the
 * context's stream unless stats is non-NULL (then filled after a synchronisation;
 * without stats an invalid input or a timeout is not reported). The first call
 * with validate == 0 for a new err_tol builds the trust map (synchronous). Errors as rt_irradiate, and
 * RT_ERR_NOT_CONFIGURED without a surrogate for this table, RT_ERR_TIMEOUT if a
 * tensor-core product did not complete within the kernel's bounded wait. */
int rt_irradiate_surrogate(rt_ctx *ctx, const float *rho, const float *t_dust, float *q_abs,
                           float *a_rad, float err_tol, int validate, rt_surrogate_stats *stats_or_null);

/* Parameters of the network, host buffers of RT_SUR_NPARAMS floats in the order of
 * RT_SUR_NPARAMS; set creates the surrogate for the context's current table. */
int rt_surrogate_set_params(rt_ctx *ctx, const float *params, double mu, double sigma);
int rt_surrogate_get_params(rt_ctx *ctx, float *params, double *mu_or_null, double *sigma_or_null);

/* rt_surrogate_grad -- one forward and backward pass of the training kernels on
 * n given rows (host buffers): x [n][8] features, t [n] standardised targets;
 * grad [RT_SUR_NPARAMS] receives d/dparams of mean((y - t)^2), loss that mean.
 * For checking the training kernels; the parameters are not changed. */
int rt_surrogate_grad(rt_ctx *ctx, const float *x, const float *t, int n, float *grad, double *loss);

/* rt_surrogate_eval -- network output y [n] (standardised) for feature rows
 * x [n][8] (host buffers), with the inference kernel's arithmetic. */
int rt_surrogate_eval(rt_ctx *ctx, const float *x, int n, float *y);

/* rt_surrogate_loss_history -- minibatch losses of the last training, one per step;
 * copies min(steps, max) values and returns the number of steps. */
int rt_surrogate_loss_history(rt_ctx *ctx, float *loss, int max);

/* rt_surrogate_trust_map -- build the trust map for err_tol and copy its 64 x 64
 * bits (bin iu * 64 + iv, 128 words) to `bits`; ranges (if non-NULL) receives
 * (u0, du, v0, dv): bin iu covers u0 + iu du .. u0 + (iu + 1) du, bin 0 also all
 * smaller values; likewise for v. */
int rt_surrogate_trust_map(rt_ctx *ctx, float err_tol, unsigned *bits, float *ranges_or_null);

/* Save / load the surrogate (parameters, standardisation, feature constants and
 * the fingerprint of the table it belongs to). Loading into a context whose table
 * differs fails with RT_ERR_NOT_CONFIGURED. */
int rt_surrogate_save(rt_ctx *ctx, const char *path);
int rt_surrogate_load(rt_ctx *ctx, const char *path);

/* rt_probe_ex2 -- y[i] = 2^x[i] with the hardware approximation the FP32 tracer
 * uses, for accuracy tests. x, y: device float32 arrays of n elements; runs on
 * stream (NULL = default) and synchronises it. */
int rt_probe_ex2(const float *x, float *y, long long n, void *cuda_stream);

/* rt_probe_alu_rates -- micro-benchmark of the current device: sustained MUFU
 * ex2.approx.f32 and FP32 FFMA throughput in operations per SM per clock, and the
 * SM clock (MHz) measured during the ex2 run. Synchronises the device. */
int rt_probe_alu_rates(double *ex2_per_sm_clk, double *ffma_per_sm_clk, double *sm_mhz);

/* rt_probe_tanh -- y[i] = tanh(x[i]) with the hardware approximation (tanh.approx)
 * the surrogate network's activations use: FP32 when packed_bf16 == 0, else the
 * packed BF16 form applied to x[i] rounded to BF16. x, y: device, n floats.
 * Synchronises `cuda_stream`. */
int rt_probe_tanh(const float *x, float *y, long long n, int packed_bf16, void *cuda_stream);

/* rt_probe_umma -- one fifth-generation tensor-core product D = A B^T with
 * M = N = 128 and K = k (a multiple of 16, at most 128), through the shared-memory
 * operand layout, matrix descriptors and TMEM read-back the surrogate's inference
 * kernel uses. a, b: device, [128][k] BF16 bit patterns, row-major (both K-major);
 * d: device, [128][128] FP32. Synchronises `cuda_stream`; RT_ERR_TIMEOUT if the
 * product did not complete within the kernel's bounded wait. */
int rt_probe_umma(const unsigned short *a, const unsigned short *b, int k, float *d, void *cuda_stream);

/* rt_probe_tensor_rates -- sustained rates per SM per clock on the current device:
 * multiply-adds of the warp-level BF16 MMA (mma.sync m16n8k16, 32 warps per SM)
 * and of tcgen05 BF16 products with M = 128, K = 16 and N = 128 or 256 (one CTA
 * per SM, one issuing thread); tanh.approx instructions in FP32 and packed BF16;
 * rcp.approx.f32 instructions (the reciprocal of the surrogate's SiLU). */
int rt_probe_tensor_rates(double *mma_sync_mac, double *umma_n128_mac, double *umma_n256_mac,
                          double *tanh_f32, double *tanh_bf16x2, double *rcp_f32);

#ifdef __cplusplus
}
#endif
#endif /* RT_IRRADIATION_H */
