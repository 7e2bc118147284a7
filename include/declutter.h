/*
 * declutter.h -- C ABI of the GB300 (sm_103a) implementation of one
 * de-cluttering iteration from Rave, Molchanov and Linsen, "De-cluttering
 * Scatterplots with Integral Images" (arXiv 2408.06513):
 *
 *   (a) splat the n samples into a 2^k x 2^k count grid and smooth it
 *       (Sec. 4.1, Sec. 4.3 step 1),
 *   (b) build the axis-aligned and 45-degree tilted integral images of the
 *       density (Sec. 3.1, Sec. 4.3 step 2),
 *   (c) evaluate the defect-corrected per-pixel displacement of eq. (map_res)
 *       built on eq. (map) (Sec. 3.2, Sec. 4.2),
 *   (d) move every sample by bilinear interpolation of that field
 *       (Sec. 4.2, Sec. 4.3 step 3),
 * repeated for a number of iterations (Sec. 4.3 step 4).
 *
 * Conventions used by every call.
 *   - Grid resolution N = 2^log2_res, 16 <= N <= 8192.  Pixel (i, j): i is
 *     the column (x), j the row (y, pointing down), origin top-left
 *     (Sec. 4.1).  Every grid is row-major: element (i, j) at j * N + i.
 *   - Samples are float32 pairs (x, y) in the unit square (Sec. 4.1),
 *     interleaved: pos_xy[2p] = x_p, pos_xy[2p + 1] = y_p.  A sample splats
 *     to pixel (floor(x N), floor(y N)) after clamping x and y to [0, 1]
 *     (NaN counts as 0); the index N is clamped to N - 1.
 *   - Pixel (i, j) sits at (i, j) / N (Sec. 3.2, text under eq. (map)), or at
 *     (i + 1/2, j + 1/2) / N when dc_params.pixel_center is set.
 *   - Displacements are in domain units (multiply by N for pixels).
 *
 * Memory and ownership.
 *   - Every pointer argument named *_out, pos_xy or grid is a DEVICE pointer
 *     owned by the caller (for instance the data pointer of a CUDA tensor),
 *     except where a comment says "host".  Device arrays of samples must be
 *     8-byte aligned; grids must be 16-byte aligned.
 *   - The context owns its internal grids (counts, density, displacement,
 *     band aggregates and carries), allocated once by declutter_create.
 *   - All calls are asynchronous on the context's stream unless stated.
 *
 * Errors.
 *   - Every call returns a dc_status; nothing throws or aborts across the
 *     ABI.  declutter_last_error() gives a message for the last failure of
 *     the calling thread.
 *   - Kernels report device-side problems in a sticky status word;
 *     declutter_sync() waits for the stream and returns it.
 *   - There is no CPU path: without a usable CUDA device every call that
 *     needs one fails with DC_ERR_CUDA.
 */
#ifndef DECLUTTER_H
#define DECLUTTER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dc_ctx dc_ctx;

typedef enum {
    DC_OK = 0,
    DC_ERR_INVALID_ARG = 1, /* null or misaligned pointer, bad size or parameter */
    DC_ERR_NOT_POW2 = 2,    /* resolution outside 2^4 .. 2^13 */
    DC_ERR_OOM = 3,         /* device allocation failed */
    DC_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed */
    DC_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired */
    DC_ERR_RANGE = 6,       /* a device-side range check failed */
    DC_ERR_STATE = 7        /* call order: e.g. displacement before any splat */
} dc_status;

/* Carry arithmetic of the float (smoothed-density) integral images. */
enum {
    DC_CARRY_COMPENSATED = 0, /* FP32 two-sum (compensated) cross-band carries */
    DC_CARRY_F64 = 1          /* FP64 cross-band carries, rounded once to FP32 */
};

typedef struct {
    uint32_t log2_res;       /* N = 1 << log2_res, 4..13 */
    int32_t kernel_r;        /* Gaussian taps |k| <= r (Sec. 4.1): 0 = no smoothing,
                                exact integer mode (any N); < 0 = N/128, at least 2;
                                max 64, < N.  r > 0 (float mode) needs N <= 2048:
                                there its displacement is within 1e-4 px of FP64;
                                above, the FP32 region sums alone err by about
                                2^-24 N / 2 px, and creation fails */
    float sigma;             /* Gaussian width; <= 0 = r / 3 */
    float d0;                /* regularising constant of eq. (d0); < 0 = n / N^2 */
    int32_t pixel_center;    /* 0: pixel at (i, j)/N; 1: at (i + 1/2, j + 1/2)/N */
    int32_t clamp_positions; /* 1: clamp each updated sample to [0, 1]^2 */
    int32_t carry_mode;      /* DC_CARRY_* (float mode only) */
    int32_t band_rows;       /* rows per band of the integral-image kernels,
                                1..64 (the last band may be shorter); 0 =
                                automatic: one band per SM of the device
                                from 1024 x 1024, N / 256 (at least 1) below */
    int32_t keep_order;      /* regularize(): 0 = iterate on an internal copy of the
                                samples sorted by pixel (faster; results identical),
                                1 = iterate in the caller's order */
    int32_t options;         /* OR of DC_OPT_* (0 = the default launch sequence) */
    int32_t wait_limit_us;   /* bound of the grid-barrier waits of the
                                DC_OPT_FUSED_BANDS launch, in microseconds,
                                1..10^7; 0 = one second */
    int32_t reserved[1];     /* must be zero */
} dc_params;

/* Launch-sequence options of dc_params.options.  Every option gives results
 * bit-identical to the default sequence; the defaults are the measured
 * fastest on a GB300. */
enum {
    /* float and exact mode below 2048 x 2048: the aggregate pass, the
     * carries and the final pass of the integral images as one cooperative
     * launch with two grid barriers (where all band CTAs fit on the GPU at
     * once), instead of three launches */
    DC_OPT_FUSED_BANDS = 1,
    /* float mode: the Gaussian smoothing as its own launch instead of inside
     * the aggregate pass (128^2 .. 1024^2) */
    DC_OPT_SEPARATE_SMOOTH = 2,
    /* regularize_host(): always stage pinned host samples through a device
     * copy instead of iterating on them over the host link */
    DC_OPT_STAGE_HOST = 4,
    /* declutter_batch_create(): one launch per step over all panels of a
     * resolution instead of per-panel graph branches */
    DC_OPT_BATCHED_LAUNCHES = 8,
    /* For testing the timeout path only: the grid barrier of the
     * DC_OPT_FUSED_BANDS launch waits for one CTA more than the grid holds,
     * so every wait runs to wait_limit_us, the call's results are undefined
     * and declutter_sync() returns DC_ERR_TIMEOUT. */
    DC_OPT_TEST_UNREACHED_BARRIER = 1 << 30
};

/* Read-back of the configuration a context settled on. */
typedef struct {
    int32_t N;               /* resolution */
    int32_t kernel_r;        /* effective radius (0 = exact integer mode) */
    float sigma;             /* effective Gaussian width */
    int32_t band_rows;       /* rows per band */
    int32_t n_bands;         /* ceil(N / band_rows) */
    int32_t band_threads;    /* threads per band CTA */
    int32_t kernels_per_iter;/* kernel launches per iteration of regularize */
    int32_t device;          /* CUDA device ordinal */
    int64_t scratch_bytes;   /* device bytes held by the context */
} dc_info;

/* Create a context for one resolution and parameter set.
 *   params : host pointer, read once.
 *   device : CUDA device ordinal; made current for the call.
 *   cuda_stream : a cudaStream_t to run on, or NULL for a stream the library
 *                 creates (ordered with the legacy default stream).
 *   out    : host pointer receiving the context.
 * Fails with DC_ERR_NOT_POW2 for a resolution outside 2^4..2^13 and with
 * DC_ERR_INVALID_ARG for any other bad parameter. */
dc_status declutter_create(const dc_params *params, int device, void *cuda_stream, dc_ctx **out);

/* Wait for outstanding work and free the context (NULL is accepted). */
dc_status declutter_destroy(dc_ctx *ctx);

/* Effective configuration (host pointer out). */
dc_status declutter_get_info(const dc_ctx *ctx, dc_info *out);

/* Step (a), Sec. 4.1 and Sec. 4.3 step 1: single-pixel accumulation of the n
 * samples into the context's uint32 count grid, then (kernel_r > 0) the
 * separable Gaussian smoothing with reflect border into its float density
 * d_r.  The regularising constant d0 of eq. (d0) is applied analytically by
 * the later steps and is not added to d_r.
 *   pos_xy     : device float[2n].
 *   n          : 0 <= n < 2^32.
 *   counts_out : device uint32[N*N] receiving a copy of the counts, or NULL.
 *   density_out: device float[N*N] receiving d_r (float mode), or NULL. */
dc_status splat_density(dc_ctx *ctx, const float *pos_xy, int64_t n, uint32_t *counts_out,
                        float *density_out);

/* Step (a) split at the count grid, for a plot whose samples are sharded
 * over several devices or processes (Sec. 4.3 step 1: the counts are integer
 * sums, so per-shard grids added together give exactly the grid of all
 * samples).  splat_counts: the single-pixel accumulation of this shard's n
 * samples into counts_out (device uint32[N*N], 16-byte aligned; zeroed
 * first); the context's own grids are not touched.  density_from_counts:
 * takes the summed grid (device uint32[N*N], 16-byte aligned) of all n
 * samples of the plot as the context's count grid and smooths it as
 * splat_density does; displacement_field() and advect_samples() (on this
 * shard's samples) follow.  Asynchronous.  Errors: DC_ERR_INVALID_ARG for a
 * null or misaligned pointer or n outside [0, 2^32). */
dc_status splat_counts(dc_ctx *ctx, const float *pos_xy, int64_t n, uint32_t *counts_out);
dc_status density_from_counts(dc_ctx *ctx, const uint32_t *counts, int64_t n);

/* Step (b), Sec. 3.1: alpha (sum over i' <= i, j' <= j) and alpha_t (sum over
 * i'+j' <= i+j, i'-j' >= i-j) of the density of the last splat_density call.
 * The other six images follow from these two and their marginals
 * (Sec. 3.1, Fig. 2 caption) and are not stored.
 *   exact mode (kernel_r = 0): alpha_out, alpha_t_out are device uint64[N*N],
 *       bit-exact sums of the counts;
 *   float mode: device float[N*N] sums of d_r (without d0).
 * Either output may be NULL. */
dc_status integral_images(dc_ctx *ctx, void *alpha_out, void *alpha_t_out);

/* Step (b) on an arbitrary grid: exact uint64 alpha and alpha_t of the
 * device uint32[N*N] array grid (N of the context).  Independent of the
 * context's splat state; uses the context's scratch.  Either output may be
 * NULL. */
dc_status integral_images_u32(dc_ctx *ctx, const uint32_t *grid, uint64_t *alpha_out,
                              uint64_t *alpha_t_out);

/* Step (c), eqs. (map), (d0), (map_res): per-pixel displacement
 * D = t(x, y; d_r + d0) - t(x, y; d0) of the density of the last
 * splat_density call, into the context's field and, if disp_xy_out is not
 * NULL, into device float[2*N*N] (interleaved x, y; domain units).
 * Exact mode evaluates the numerator in exact integer arithmetic and rounds
 * once, so an even count grid gives exactly zero. */
dc_status displacement_field(dc_ctx *ctx, float *disp_xy_out);

/* The virtual lens of Molchanov and Linsen (end of Sec. 3.2): the mapping of
 * eq. (map) itself, t(x, y; d), for a caller's density d >= 0 (for the lens,
 * constant inside and outside a selected area), without the defect term of
 * eq. (map_res).  Writes the displacement t(x, y; d) - (x, y) of every pixel
 * (domain units, interleaved x, y) into the context's field and, if
 * disp_xy_out is not NULL, into device float[2*N*N]; advect_samples() then
 * moves samples to the bilinearly interpolated mapping.
 *   density     : device float[N*N], row-major [j][i], 16-byte aligned; not
 *                 modified.
 *   density_mean: a hint that centres the float sums (the density's mean,
 *                 or 0); the mapping does not depend on it, only the
 *                 rounding does.
 * Float arithmetic as in displacement_field, N <= 2048.  With the
 * density's mean as density_mean the pixel position cancels in exact
 * integers before any rounding and the result is within 1e-4 px of FP64;
 * with 0, t is formed as an O(1) float first (about 6 N 2^-24 px).  A
 * density without mass has no mapping: the field is written as zero and the
 * status word reports DC_ERR_INVALID_ARG.  Asynchronous.  Errors:
 * DC_ERR_INVALID_ARG for a null or misaligned pointer, a negative or
 * non-finite density_mean or N > 2048 (nothing is launched); DC_ERR_CUDA for
 * a failed launch. */
dc_status lens_field(dc_ctx *ctx, const float *density, float density_mean, float *disp_xy_out);

/* Contour lines of a density (Sec. 5: the original density's contours,
 * shown again after the transformation by moving their vertices, e.g. as
 * tracers of regularize_tracers).  Marching squares over the pixel nodes at
 * the positions of the context's pixel convention: cell (i, j),
 * 0 <= i, j < N - 1, has the corners f(i, j), f(i+1, j), f(i+1, j+1),
 * f(i, j+1); a corner is inside when f >= level; a crossed edge holds the
 * linearly interpolated vertex; the two saddle cases follow the cell
 * centre, the mean of the four corners.
 *   field   : device float[N*N], row-major [j][i] (e.g. d_r from
 *             splat_density); not modified.
 *   segs_out: device float[8 (N-1)^2], 16-byte aligned: for cell
 *             c = j (N-1) + i, slots 2c and 2c+1 of (x0, y0, x1, y1) in domain
 *             units; a cell with fewer than two segments writes NaN into the
 *             unused slots (so the output order is the cell order).
 * Asynchronous.  Errors: DC_ERR_INVALID_ARG for a null or misaligned
 * pointer or a non-finite level (nothing is launched); DC_ERR_CUDA for a
 * failed launch. */
dc_status contour_segments(dc_ctx *ctx, const float *field, float level, float *segs_out);

/* Step (d), Sec. 4.2: in place, z <- z + bilinear(D)(z) for the n samples,
 * with the field of the last displacement_field (or lens_field) call; corner indices are
 * clamped to the grid, and with clamp_positions the result to [0, 1]^2. */
dc_status advect_samples(dc_ctx *ctx, float *pos_xy, int64_t n);

/* Sec. 4.3: iters full iterations (a)-(d) in place on pos_xy, launched as
 * one CUDA graph captured on the first call for this (pos_xy, n, iters,
 * metrics) combination and replayed afterwards.
 *   uniformity_out: host double[iters], or NULL.  When given, entry k is the
 *   Sec. 6.2 regularity measure (std of the sample counts of 4x4-pixel bins)
 *   after iteration k + 1, and the call synchronises and returns the device
 *   status; otherwise the call is asynchronous. */
dc_status regularize(dc_ctx *ctx, float *pos_xy, int64_t n, int32_t iters, double *uniformity_out);

/* regularize() that also moves n_tracers massless tracers (device
 * float[2 n_tracers]) by each iteration's field without splatting them, e.g.
 * the pixel nodes, whose final minus initial positions are the displacement
 * field composed over the iterations (the deformed grid of Sec. 5).
 * Asynchronous; not captured into a graph. */
dc_status regularize_tracers(dc_ctx *ctx, float *pos_xy, int64_t n, float *tracer_xy, int64_t n_tracers,
                             int32_t iters);

/* regularize() on HOST samples float[2n], updated in place; synchronises.
 * Pinned or registered host memory (cudaHostAlloc, cudaHostRegister) with
 * keep_order = 0: the iterations run on the host array directly, reading it
 * over the host link in the first splat and the reordering and writing the
 * result back in the final gather (no staging copies).  Otherwise the array
 * is copied to a context-owned device buffer and back.  The context option
 * DC_OPT_STAGE_HOST forces the copies.
 * uniformity_out as for regularize(). */
dc_status regularize_host(dc_ctx *ctx, float *host_pos_xy, int64_t n, int32_t iters,
                          double *uniformity_out);

/* Sec. 4.3 step 4: iterations of regularize() until a stopping criterion
 * holds, decided on the GPU after every iteration, in one CUDA graph launch
 * (captured on the first call for this (pos_xy, n, max_iters) and replayed
 * afterwards; the criteria are read at launch time).  After iteration k the
 * run stops when
 *   - k = max_iters (1..1024), or
 *   - target_cv > 0 and the Sec. 6.2 bin std over the mean bin count of the
 *     moved samples is <= target_cv (a regularity measure), or
 *   - min_move_px > 0 and the largest distance a sample moved in iteration k
 *     is <= min_move_px pixels (the impact of the last iteration), or
 *   - max_ms > 0 and the device time since the graph started is >= max_ms.
 * Iterations 2..max_iters sit in conditional graph nodes whose condition
 * the previous iteration's check sets, so at most max_iters iterations run
 * whatever the data.  The positions are those of regularize() with the
 * same number of iterations, bit for bit.
 *   iters_out  : host int32, iterations done (or NULL).
 *   cv_out, move_px_out: host double[max_iters] (or NULL): the measure and
 *                the largest move of every iteration done.
 * Synchronises.  Errors: DC_ERR_INVALID_ARG for n = 0, max_iters outside
 * 1..1024 or a negative or non-finite criterion. */
dc_status regularize_adaptive(dc_ctx *ctx, float *pos_xy, int64_t n, int32_t max_iters, double target_cv,
                              double min_move_px, double max_ms, int32_t *iters_out, double *cv_out,
                              double *move_px_out);

/* Sec. 1: the continuous transition between the original and the
 * regularised scatterplot, as a per-sample blend of the two positions:
 * out = (1 - s) from + s to, rounded to float32 after each operation in
 * that order, so s = 0 gives from and s = 1 gives to exactly.
 *   from_xy, to_xy, out_xy: device float[2n] (out may alias either input).
 *   s: 0 <= s <= 1.
 * Asynchronous.  Errors: DC_ERR_INVALID_ARG for s outside [0, 1], a null or
 * misaligned pointer. */
dc_status transition_positions(dc_ctx *ctx, const float *from_xy, const float *to_xy, int64_t n, float s,
                               float *out_xy);

/* Sec. 6.2: how well the regularised layout keeps the original's local
 * structure, by the two measures the paper reports: trustworthiness
 * (Venna and Kaski) and orthogonal ordering (Misue et al.).  Positions are
 * taken on the lattice X = rint(float32(x * 65535)) (x clamped to [0, 1]);
 * distances are squared lattice distances, ties broken by sample index.
 * Over the query samples Q (m of them):
 *   out[0] = T = 1 - 2 / (m k (2n - 3k - 1)) * sum_{i in Q} sum_{j in U_k(i)} (r(i, j) - k),
 *            U_k(i) = the k nearest neighbours of i in reg that are not
 *            among its k nearest in orig, r(i, j) = the rank of j by
 *            distance from i in orig (nearest = 1);
 *   out[1] = O = 1 - (sum_{i in Q} #{j : sign(X_i - X_j) or sign(Y_i - Y_j)
 *            differs between orig and reg}) / (m (n - 1)).
 * With every sample a query these are the exact measures; a random subset
 * estimates them at O(m n) cost.
 *   orig_xy, reg_xy: device float[2n], n < 2^31.
 *   queries: device uint32[n_queries] sample indices, or NULL for
 *            0 .. n_queries - 1 (n_queries <= n).
 *   k: 1..32, k < n / 2.
 *   out: host double[2]; terms_out: host int64[2 n_queries] or NULL, the
 *        per-query integer sums (T's inner sum, O's count).
 * Synchronises.  Errors: DC_ERR_INVALID_ARG for bad sizes or pointers,
 * DC_ERR_RANGE for a query index outside [0, n). */
dc_status layout_metrics(dc_ctx *ctx, const float *orig_xy, const float *reg_xy, int64_t n,
                         const uint32_t *queries, int32_t n_queries, int32_t k, double *out, int64_t *terms_out);

/* Sec. 5, the density background texture: a texture given at the N x N
 * pixel nodes (e.g. d_r from splat_density), drawn on the mesh of those
 * nodes after they moved to nodes_xy (e.g. the tracers of
 * regularize_tracers started at the pixel positions), into an M x M raster,
 * M = 2^out_log2.  Every cell (i, j) of the node mesh is split into the
 * triangles 2c = (i, j), (i+1, j), (i+1, j+1) and 2c + 1 = (i, j),
 * (i+1, j+1), (i, j+1), c = j (N - 1) + i.  Output pixel (p, q) has its
 * centre at ((p + 1/2) / M, (q + 1/2) / M); it is covered by the triangles
 * whose interior holds the centre, or whose edge holds it under a fill rule
 * that gives points on a shared edge or vertex to exactly one of the
 * triangles (vertices snapped to 1/256 pixel; exact integer tests); where
 * triangles overlap, the lowest index wins.  A covered pixel takes the
 * texture at the source point with the same barycentric coordinates in the
 * undeformed triangle (bilinear lookup between nodes); uncovered pixels are
 * 0.  DC_WARP_MASS multiplies by the undeformed over the deformed triangle
 * area, the push-forward density, whose sum is the texture's mass.
 *   nodes_xy: device float[2 N N] (domain units; clamped to [-1, 2]).
 *   texture : device float[N N], row-major [j][i].
 *   out     : device float[M M]; tri_out: device int32[M M] receiving the
 *             winning triangle (-1: none), or NULL (context scratch).
 * Asynchronous.  Errors: DC_ERR_INVALID_ARG for null or misaligned pointers,
 * out_log2 outside 4..13 or an unknown mode. */
enum { DC_WARP_VALUE = 0, DC_WARP_MASS = 1 };
dc_status warp_texture(dc_ctx *ctx, const float *nodes_xy, const float *texture, int32_t out_log2, int32_t mode,
                       float *out, int32_t *tri_out);

/* Sec. 5 transfer function: rgba_out[k] = lut[i] with
 * i = rint((values[k] - lo) * s), s = 255 / (hi - lo), clamped to 0..255
 * (float32, each operation rounded in that order; NaN -> 0).
 *   values: device float[count]; lut: device uint32[256] (RGBA8);
 *   rgba_out: device uint32[count].
 * Asynchronous.  Errors: DC_ERR_INVALID_ARG for null or misaligned pointers
 * or unless lo < hi, both finite. */
dc_status transfer_function(dc_ctx *ctx, const float *values, int64_t count, float lo, float hi,
                            const uint32_t *lut, uint32_t *rgba_out);

/* The count grid c(i, j) of Sec. 4.1 (Sec. 4.3 step 1) that the context
 * holds: that of the last splat_density() call or, after regularize(),
 * that of the last splat the iterations performed.  Inside regularize()
 * the advection of every iteration but the last splats the moved samples
 * into the next iteration's grid; with uniformity_out given, the last
 * iteration does too, so the grid is that of the returned positions;
 * without it, the grid is the input of the last iteration.
 *   counts_out: device uint32[N*N], 4-byte aligned, row-major [j][i].
 * Asynchronous (a device-to-device copy on the context's stream).  Errors:
 * DC_ERR_INVALID_ARG for a null or misaligned pointer, DC_ERR_STATE before
 * any splat. */
dc_status declutter_counts(dc_ctx *ctx, uint32_t *counts_out);

/* Sec. 6.2 quality measures of the count grid of the last splat_density
 * call; synchronises.  out (host double[3]): [0] std of the 4x4-bin counts,
 * [1] that std over the mean bin count, [2] overplotting =
 * (n - occupied pixels) / n. */
dc_status quality_metrics(dc_ctx *ctx, double *out);

/* Wait for the context's stream; returns the first CUDA error or the sticky
 * device status, and clears the latter. */
dc_status declutter_sync(dc_ctx *ctx);

/* Per-kernel device time of regularize(), measured with CUDA events on the
 * context's stream.  The iteration sequence is captured as a graph exactly
 * as regularize() captures it and run reps times (after two warm-up runs):
 * its mean duration goes to *step_ms_out.  Then, for each kernel kind, a
 * graph in which every launch of that kind is issued twice in a row is run
 * the same way; the increase of the mean duration over the plain graph is
 * that kind's in-graph device time per regularize() call, written to
 * kernel_ms_out[kind] (host float[DC_KERNEL_KINDS]).  launches_out[kind]
 * (host int32[DC_KERNEL_KINDS]) receives the launches per call.
 *   pos_xy   : device samples, moved in place by every run.
 *   reset_src: device float[2n] copied into pos_xy before each run (outside
 *              the timed span), or NULL to let the samples keep moving.
 * Any output pointer may be NULL.  Synchronises. */
#define DC_KERNEL_KINDS 10
dc_status declutter_profile_regularize(dc_ctx *ctx, float *pos_xy, const float *reset_src, int64_t n,
                                       int32_t iters, int32_t reps, float *step_ms_out,
                                       float *kernel_ms_out, int32_t *launches_out);

/* Name of kernel kind k (0 <= k < DC_KERNEL_KINDS), or NULL. */
const char *declutter_kernel_name(int32_t k);

const char *declutter_status_string(dc_status s);
const char *declutter_last_error(void);

/* ------------------------------------------------------------------------
 * Batched regularisation of many independent scatterplots, e.g. all
 * dimension-pair panels of a scatterplot matrix, with per-panel resolution
 * and sample count (not in the paper; the paper regularises one plot).
 * Every panel is an independent problem with its own context; one call runs
 * all panels' iterations as the independent branches of one CUDA graph
 * (captured on the first call for the given sample pointers, sizes,
 * iterations and metrics flag, replayed afterwards).
 * ------------------------------------------------------------------------ */
typedef struct dc_batch dc_batch;

/* base: shared parameters (its log2_res is ignored); log2_res[p] and
 * max_samples[p] (host arrays of n_panels entries): each panel's resolution
 * and the largest sample count it will be given.  Panels run on cuda_stream
 * (or a library stream when NULL). */
dc_status declutter_batch_create(const dc_params *base, const uint32_t *log2_res, const int64_t *max_samples,
                                 int32_t n_panels, int device, void *cuda_stream, dc_batch **out);
dc_status declutter_batch_destroy(dc_batch *batch);

/* pos_xy: host array of n_panels device pointers (float[2 n[p]] each, moved in
 * place); n: host array of sample counts (<= max_samples).  uniformity_out:
 * host double[n_panels * iters] (panel-major) of the Sec. 6.2 bin std after
 * each iteration, or NULL (then the call is asynchronous).  Results are
 * identical to regularize() on each panel alone. */
dc_status declutter_batch_regularize(dc_batch *batch, float *const *pos_xy, const int64_t *n, int32_t iters,
                                     double *uniformity_out);

/* Wait for the batch's stream; returns the first CUDA error or device status. */
dc_status declutter_batch_sync(dc_batch *batch);

/* Autotuner of the integral-image band height (rows per band): times
 * regularize(iters) on a copy of the given samples for every band height
 * 1, 2, 4, ... 64 with at most 1024 bands and for the automatic height, and
 * returns the fastest in
 * *best_out (its median time in *best_ms_out, or -1 when the answer came
 * from the cache).  Answers are cached per (GPU model, resolution, radius,
 * carry mode, keep_order, floor(log2 n)), see declutter_autotune_save.  The samples are not
 * modified.  Synchronises. */
dc_status declutter_autotune_band_rows(const dc_params *params, int device, void *cuda_stream, const float *pos_xy,
                                       int64_t n, int32_t iters, int32_t *best_out, float *best_ms_out);

/* The autotuner over band heights and launch sequences: times
 * regularize(iters) on a copy of the samples for every band height 1, 2, 4,
 * .. 64 (at most 1024 bands) and the automatic one, each with the default
 * launch sequence, DC_OPT_SEPARATE_SMOOTH (float mode) and
 * DC_OPT_FUSED_BANDS (below 2048 x 2048), and writes params with the
 * fastest band_rows and options into *best_out (host).  The launch
 * options never change the results; in float mode the band height changes
 * the order of the float sums (every height within the float bound).  The
 * answer is cached per (GPU model and SM count,
 * resolution, radius, carry mode, keep_order, floor(log2 n)); *best_ms_out
 * (host, or NULL) is the median time, -1 for a cached answer.  The samples
 * are not modified.  Synchronises. */
dc_status declutter_autotune(const dc_params *params, int device, void *cuda_stream, const float *pos_xy, int64_t n,
                             int32_t iters, dc_params *best_out, float *best_ms_out);

/* The autotuner's cache in a text file (host paths), so that tuned settings
 * carry over to later runs on the same GPU model: save writes every entry,
 * load adds the file's entries (DC_ERR_INVALID_ARG for an unreadable or
 * malformed file, nothing added), clear empties the cache.  No device is
 * used. */
dc_status declutter_autotune_save(const char *path);
dc_status declutter_autotune_load(const char *path);
dc_status declutter_autotune_clear(void);

/* Autotunes every resolution of a batch on its largest panel and rebuilds the
 * panels' contexts with the chosen band heights (band_rows_out: host
 * int32[n_panels] or NULL). */
dc_status declutter_batch_autotune(dc_batch *batch, float *const *pos_xy, const int64_t *n, int32_t iters,
                                   int32_t *band_rows_out);

/* ------------------------------------------------------------------------
 * Learned surrogate (not in the paper): a convolutional encoder-decoder that
 * maps a density grid to the displacement field composed over several plain
 * iterations, trained on pairs the plain method generates.  BF16 weights and
 * activations, FP32 accumulation on tensor cores (tcgen05 or mma.sync, see
 * surrogate_set_tensor_path), FP32
 * master weights and Adam.  Layers, in order: enc{l}a, enc{l}b for
 * l = 0..L-1 (widths c_l = base_channels * 2^l), dec{l}up, dec{l}c for
 * l = L-2..0, head (2 outputs); 3x3 convolutions with zero padding, ReLU
 * after every layer but the head, 2x2 average pooling down, nearest
 * upsampling and additive skips up.  Tensors are [batch][y][x][channel].
 * Inputs: the scaled density, and with in_channels = 3 also the field of
 * one plain iteration (x, y in pixels), which carries the method's global
 * integrals past the network's receptive field; the output is then
 * kappa * field + the network's output (kappa from surrogate_set_skip).
 * ------------------------------------------------------------------------ */
typedef struct dc_surrogate dc_surrogate;

/* Input and output grids are 2^log2_res square; levels 1..6 with
 * log2_res >= levels + 2; base_channels a multiple of 8 (<= 256);
 * in_channels 1 (density) or 3 (density and one iteration's field); batches
 * of at most max_batch; He-normal initial weights from seed; kappa 0. */
dc_status surrogate_create(int32_t log2_res, int32_t levels, int32_t base_channels, int32_t in_channels,
                           int32_t max_batch, uint64_t seed, int device, void *cuda_stream, dc_surrogate **out);
/* kappa of the output skip kappa * field (in_channels = 3). */
dc_status surrogate_set_skip(dc_surrogate *sg, float kappa);

/* Tensor-core path of the forward convolutions with 64..256 output
 * channels: DC_SG_MMA_SYNC (warp-level mma.sync), DC_SG_TCGEN05
 * (fifth-generation tcgen05.mma with the accumulator in tensor memory, the
 * weights staged by tensor memory access) or DC_SG_AUTO (default: tcgen05
 * in batches of two or more samples, mma.sync for a single one, where each
 * measured faster).  The paths sum in different orders (results within FP32
 * rounding). */
enum { DC_SG_MMA_SYNC = 0, DC_SG_TCGEN05 = 1, DC_SG_AUTO = 2 };
dc_status surrogate_set_tensor_path(dc_surrogate *sg, int32_t path);
dc_status surrogate_destroy(dc_surrogate *sg);

/* Parameter counts in the unpadded layout used by get/set: for every layer
 * in order, weights [out][3][3][in] (all layers' weights concatenated) and
 * biases [out] (all layers' biases concatenated). */
dc_status surrogate_num_params(const dc_surrogate *sg, int64_t *weights, int64_t *biases);
dc_status surrogate_get_params(dc_surrogate *sg, float *w_host, float *b_host);
/* Sets the FP32 master weights (BF16 copies follow) and resets Adam. */
dc_status surrogate_set_params(dc_surrogate *sg, const float *w_host, const float *b_host);
/* Weight and bias gradients of the last surrogate_loss_grad / train_step. */
dc_status surrogate_get_grads(dc_surrogate *sg, float *gw_host, float *gb_host);

/* density: device float[batch][H][W], multiplied on input by scales[b]
 * (device float[batch], e.g. N^2 / n so that the even layout reads 1; NULL
 * means 1); field: device float[batch][H][W][2] (pixels; required when
 * in_channels = 3, ignored otherwise); out: device float[batch][H][W][2]
 * (pixels), or NULL. */
dc_status surrogate_forward(dc_surrogate *sg, const float *density, const float *scales, const float *field,
                            int32_t batch, float *out);
/* Forward + backward for 0.5 * mean((out - target)^2), target device
 * float[batch][H][W][2]; *loss_out (host) after synchronising, if given. */
dc_status surrogate_loss_grad(dc_surrogate *sg, const float *density, const float *scales, const float *field,
                              const float *target, int32_t batch, float *loss_out);
/* surrogate_loss_grad followed by one Adam step (beta 0.9 / 0.999). */
dc_status surrogate_train_step(dc_surrogate *sg, const float *density, const float *scales, const float *field,
                               const float *target, int32_t batch, float lr, float *loss_out);
/* One-shot regularisation of device samples with the surrogate (context in
 * float mode at the surrogate's resolution): predict the composed field from
 * the samples' density (and, with in_channels = 3, the field of one plain
 * iteration, computed here), move every sample once by it, then, if the
 * Sec. 6.2 bin std / mean of the moved samples exceeds target_cv, run plain
 * iterations as regularize_adaptive() does (one graph launch, stopped on the
 * GPU after the first iteration that meets target_cv; at most
 * max_plain_iters, 0..1024; target_cv = 0 runs all of them).  Returns the
 * plain iterations used and the final ratio.  Synchronises.  Errors:
 * DC_ERR_INVALID_ARG also for max_plain_iters outside 0..1024 or a negative
 * or non-finite target_cv. */
dc_status surrogate_apply(dc_ctx *ctx, dc_surrogate *sg, float *pos_xy, int64_t n, float target_cv,
                          int32_t max_plain_iters, int32_t *plain_iters_out, double *cv_out);

/* No-allocation variant of integral_images_u32(), for callers that cannot
 * allocate device memory when they need the result: applications that hand
 * out all device memory from their own pool or budget and do not let a
 * library allocate behind their back, and latency-bound loops that cannot
 * afford the device-wide synchronisation cudaMalloc and cudaFree may imply.
 * The paper has no counterpart; it is a deployment variant of the same
 * computation.
 *
 * Needs no context.  Writes the exact uint64 alpha and alpha_t of the device
 * uint32[N*N] array grid, N = 2^log2_res, into alpha_out / alpha_t_out
 * (device, 16-byte aligned, either may be NULL), on cuda_stream (NULL = the
 * legacy default stream), asynchronously, on the calling thread's current
 * device; grid and the outputs must be memory of that device (checked with
 * cudaPointerGetAttributes before anything is launched: DC_ERR_INVALID_ARG
 * otherwise).  Results are bit-identical to integral_images_u32().
 *
 * Scratch: one fixed device array inside the library,
 * DC_NOALLOC_SCRATCH_BYTES long, held by every GPU that loads the library
 * until the process exits.  No cudaMalloc, cudaFree or allocating library
 * routine is called.  log2_res above DC_NOALLOC_MAX_LOG2_RES (grids larger
 * than 1024 x 1024) is rejected with DC_ERR_INVALID_ARG, below 4 with
 * DC_ERR_NOT_POW2; declutter_last_error() gives the reason.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and sets the kernels' shared-memory attributes with
 * that device current; later calls reuse both.  All
 * calls share the one array and it keeps the last call's contents (none of
 * it needs to start at zero): calls that overlap on the GPU, for instance on
 * two streams, race and must not be issued.
 * There is no status word on this path: from 1024 x 1024 the kernels' bulk
 * copies are waited for with a bounded wait, and if such a wait expired the
 * results would be wrong with nothing reported (the context path reports it
 * as DC_ERR_TIMEOUT from declutter_sync). */
#define DC_NOALLOC_MAX_LOG2_RES 10
#define DC_NOALLOC_SCRATCH_BYTES 8912896
dc_status integral_images_u32_noalloc(const uint32_t *grid, uint32_t log2_res, uint64_t *alpha_out,
                                      uint64_t *alpha_t_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DECLUTTER_H */
