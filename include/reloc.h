/*
 * reloc.h -- C ABI of the GB300 relocalization hot path of 3DGS-ReLoc
 * (arXiv 2403.11367): load a Gaussian map, pick the 2D-voxel block near a
 * coarse pose, render RGB and depth of many candidate poses, score each
 * against the query by normalised cross-correlation and return the best view
 * with its depth (Sec. III-C.1, "Initial ReLocalization").
 *
 * Conventions (every call):
 *   - A pose is a row-major 4x4 world-to-camera matrix W (the paper's W_t,
 *     Sec. III-A) in double; camera axes are x right, y down, z forward.
 *   - Images are planar float32 [C][H][W] (C = 3 for RGB), values in [0, 1].
 *     Depth and accumulated alpha are float32 [H][W].
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; all
 *     other pointers are host pointers owned by the caller.  The library owns
 *     only its context, the device copy of the map and its workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls that return host results synchronise that stream before
 *     returning; reloc_render also synchronises (it checks workspace capacity).
 *   - Every call returns a reloc_status; nothing aborts and no C++ exception
 *     crosses the ABI.  On error, reloc_last_error() gives a message for the
 *     calling thread.  The map and workspace stay valid after an error.
 *   - Thread safety: a context is used by one host thread at a time.
 */
#ifndef RELOC_H
#define RELOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int reloc_status;
enum {
    RELOC_OK = 0,
    RELOC_EINVAL = 1,     /* bad argument (null pointer, size, config)          */
    RELOC_ENOMEM = 2,     /* host or device allocation failed                   */
    RELOC_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed        */
    RELOC_ETIMEOUT = 4,   /* a bounded device wait gave up                      */
    RELOC_ENOMAP = 5,     /* no map loaded                                      */
    RELOC_ENUMERIC = 6,   /* non-finite pose or intrinsics                      */
    RELOC_EOVERFLOW = 7   /* workspace capacity exceeded and could not grow     */
};

enum { RELOC_FP32 = 0, RELOC_FP16 = 1, RELOC_BF16 = 2 };   /* map attribute storage */

/* Every constant of the path, explicit.  reloc_default_config() fills the
 * values given in the comments. */
typedef struct reloc_config {
    int32_t tile_w, tile_h;    /* blend tile, pixels: 16 x 16 (8x8, 32x8 allowed)      */
    float near_plane;          /* cull if camera depth <= near: 0.2 m                  */
    float fov_clamp;           /* J uses tx/tz clamped to +-fov_clamp*tan(half FOV): 1.3 */
    float eps2d;               /* low-pass dilation added to Sigma' diagonal: 0.3 px^2 */
    float alpha_min;           /* skip a Gaussian at a pixel if alpha < this: 1/255    */
    float alpha_max;           /* alpha clamp: 0.99                                    */
    float t_min;               /* stop a pixel when T (1 - alpha) < this: 1e-4         */
    float cut;                 /* footprint radius in sigmas (inclusion d'S^-1 d <= cut^2): 3 */
    float det_fp64;            /* invert Sigma' in FP64 when its det < this: 1e-6 px^4 */
    double block_size;         /* 2D voxel block edge: 20 m                            */
    int64_t inst_capacity;     /* tile instances per view to start with; 0 = from the
                                  subset size (learned ratio): 0                       */
    int32_t blend_rpl;         /* blend: records staged per lane per warp step (1, 2): 1 */
    int32_t ncc_gray;          /* NCC samples (Eq. ncc, "intensity"): 0 = all 3 H W RGB
                                  samples as one vector; 1 = the H W gray values
                                  (R + G + B) / 3 of render and query: 0             */
    int32_t reserved[6];
} reloc_config;

typedef struct reloc_camera {
    int32_t width, height;     /* pixels (1 .. 16383)                                  */
    double fx, fy, cx, cy;     /* pinhole intrinsics, pixels; pixel centres at +0.5    */
} reloc_camera;

/* Host map, one row per Gaussian g_i = [mu, S, R, c, o] (Sec. III-A). */
typedef struct reloc_gaussians_host {
    const float *mean;         /* [n][3] world position, metres                        */
    const float *scale;        /* [n][3] activated standard deviations, metres (> 0)   */
    const float *quat;         /* [n][4] rotation (w, x, y, z); normalised on use      */
    const float *opacity;      /* [n]    in [0, 1]                                     */
    const float *sh;           /* [n][K][3], K = (deg+1)^2; degree 0 = plain RGB       */
} reloc_gaussians_host;

/* A contiguous run [begin, end) of the block-ordered map (reloc_map_order). */
typedef struct reloc_range { int64_t begin, end; } reloc_range;

/* Candidate grid around a coarse pose (Sec. III-C.1; Sec. IV-A uses 2 m, 10 deg):
 * offsets (dx, dy) in the world ground plane and a yaw about world z through
 * the camera centre, all centred on zero; height, pitch and roll are the
 * coarse pose's.  Candidate index = ix + nx * (iy + ny * iyaw). */
typedef struct reloc_grid {
    int32_t nx, ny, nyaw;
    double step_xy;            /* metres  */
    double step_yaw_deg;       /* degrees */
} reloc_grid;

typedef struct reloc_result {
    int32_t best_index;        /* argmax of NCC, lowest index on ties (-1: none)       */
    int32_t n_candidates;
    double best_score;         /* NCC of the best candidate                            */
    double best_pose[16];      /* its world-to-camera pose                             */
    int64_t n_gauss;           /* Gaussians in the selected block subset               */
    int32_t n_blocks;          /* blocks selected                                      */
    int32_t degenerate;        /* 1 if the best render or the query has zero variance  */
    int32_t n_scored;          /* candidates rendered and scored (all, unless the
                                  learned proposal picked a top-k or a random search
                                  visited a part)                                      */
    int32_t stopped_early;     /* random search: 1 if the NCC threshold ended it      */
} reloc_result;

/* Work counts of the last render/score/localize call (sums over views). */
typedef struct reloc_counts {
    int64_t n_views;
    int64_t n_gauss;           /* subset size                                           */
    int64_t n_visible;         /* (view, Gaussian) pairs that survived the cull         */
    int64_t n_instances;       /* (view, tile, Gaussian) entries sorted                 */
    int64_t inst_stride;       /* per-view instance capacity used                       */
    int32_t retries;           /* capacity grow-and-retry rounds taken                  */
    int32_t kernel_launches;   /* CUDA kernels the call launched (all attempts)         */
} reloc_counts;

/* Stage indices of reloc_stage_times(). */
enum {
    RELOC_STAGE_CULL = 0,      /* block subset gather (K1)                              */
    RELOC_STAGE_PROJECT,       /* EWA projection + SH (K2)                              */
    RELOC_STAGE_DEPTH_SORT,    /* visibility compaction + depth radix sort             */
    RELOC_STAGE_TILE_COUNT,    /* per-chunk tile counts, scan into tile ranges (K3)     */
    RELOC_STAGE_TILE_EMIT,     /* instances into depth-ordered tile lists (K4)          */
    RELOC_STAGE_BLEND,         /* blend + fused NCC partials (K6, K7 partials)          */
    RELOC_STAGE_SCORE,         /* NCC finalise + argmax + winner export (K7, K8)        */
    RELOC_STAGE_COUNT
};

typedef struct reloc_ctx reloc_ctx;

/* Library version string (static storage). */
const char *reloc_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *reloc_last_error(void);

/* Fill cfg with the defaults listed in reloc_config. */
void reloc_default_config(reloc_config *cfg);

/* Create a context on CUDA device `device` (that device becomes current for
 * the calling thread).  cfg NULL = defaults.  Errors: EINVAL (bad config:
 * tile sizes not in {8,16,32}x{8,16,32} or tile_w*tile_h > 512, non-positive
 * constants), ECUDA (no such device), ENOMEM. */
reloc_status reloc_create(const reloc_config *cfg, int device, reloc_ctx **out);

/* Free the context and all device memory it owns.  NULL is a no-op. */
reloc_status reloc_destroy(reloc_ctx *ctx);

/* Load (or replace) the map: partition into 2D voxel blocks of
 * cfg.block_size (Sec. III-B.2: block = (floor(x/B), floor(y/B)); the map is
 * reordered by block key (bx, by), index order inside a block), build the
 * KD-tree over block centres, and copy the attributes to the device as SoA
 * in `precision` (RELOC_FP32, RELOC_FP16 or RELOC_BF16 for scale, rotation,
 * opacity and SH; means stay FP32).  sh_degree in 0..3.  The host arrays are
 * read during the call only.  Errors: EINVAL, ENOMEM, ECUDA. */
reloc_status reloc_load_map(reloc_ctx *ctx, const reloc_gaussians_host *g, int64_t n,
                            int sh_degree, int precision);

/* Block order: order_out[p] = original index of the Gaussian at block-ordered
 * position p (n entries, host).  Errors: ENOMAP, EINVAL. */
reloc_status reloc_map_order(reloc_ctx *ctx, int64_t *order_out);

/* Select every block whose centre lies within `radius` metres of (x, y)
 * (Sec. III-C.1, submap retrieval; KD-tree range query, Sec. III-B.2).  Writes
 * up to max_ranges merged runs of the block-ordered map in ascending block-key
 * order to ranges_out (host), their number to *n_ranges, the Gaussian count
 * to *n_gauss and the block count to *n_blocks (any of the three may be
 * NULL).  EINVAL if more than max_ranges runs are needed (*n_ranges then
 * holds the number needed). */
reloc_status reloc_select_block(reloc_ctx *ctx, double x, double y, double radius,
                                reloc_range *ranges_out, int max_ranges, int *n_ranges,
                                int64_t *n_gauss, int *n_blocks);

/* Render n_views poses (host, [n_views][16]) of the subset given by `ranges`
 * (host, n_ranges runs; the subset's Gaussian order -- the tie order of equal
 * depths -- is the concatenation of the runs).  Writes, for each view v,
 * rgb_dev[v][3][H][W], depth_dev[v][H][W] (Sec. III-A depth compositing,
 * unnormalised) and alpha_dev[v][H][W] = 1 - T; any of the three may be NULL.
 * 1 <= n_views <= 4096.  Errors: EINVAL, ENOMAP, ENUMERIC, ECUDA, EOVERFLOW. */
reloc_status reloc_render(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges,
                          const double *poses, int n_views, const reloc_camera *cam,
                          float *rgb_dev, float *depth_dev, float *alpha_dev, void *stream);

/* Render as reloc_render and score each view against query_dev ([3][H][W],
 * device) with NCC (Eq. ncc) over all 3*H*W samples; writes scores_host
 * [n_views] (NCC, 0 for a zero-variance image) and, if not NULL,
 * degenerate_host[n_views] (1 = zero variance).  Images are not exported. */
reloc_status reloc_score(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges,
                         const double *poses, int n_views, const reloc_camera *cam,
                         const float *query_dev, double *scores_host, int *degenerate_host,
                         void *stream);

/* Render as reloc_score and also return, for each view, the gradient of its
 * NCC (Eq. ncc) with respect to its pose: grads_host[n_views][6] =
 * dNCC/d(rho_x, rho_y, rho_z, phi_x, phi_y, phi_z) for the left update
 * W(delta) = [Exp(phi) R | Exp(phi) t + rho] at delta = 0 -- the direction
 * of direct pose ascent on NCC that the paper names as future work.  The
 * derivative is that of the render with its inclusion, alpha-skip, clamp and
 * stop decisions fixed (the rendered image is piecewise smooth in the pose).
 * The map must have SH degree 0 (view-independent colour, the paper's map);
 * otherwise EINVAL.  scores_host[n_views] as reloc_score.  Errors: EINVAL,
 * ENOMAP, ENUMERIC, ECUDA, EOVERFLOW. */
reloc_status reloc_score_grad(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges,
                              const double *poses, int n_views, const reloc_camera *cam,
                              const float *query_dev, double *scores_host, double *grads_host,
                              void *stream);

/* The whole initial relocalization of one query (Sec. III-C.1): select the
 * blocks within `radius` of the coarse pose's camera centre, build the
 * candidate grid around the coarse pose, render every candidate, score it
 * against query_dev by NCC, take the argmax (lowest index on ties) and export
 * the winner's RGB [3][H][W], depth [H][W] and alpha [H][W] to the *_dev
 * buffers (each may be NULL).  scores_host[n_candidates] may be NULL.
 * Errors: EINVAL, ENOMAP, ENUMERIC, ECUDA, EOVERFLOW. */
reloc_status reloc_localize(reloc_ctx *ctx, const float *query_dev, const double *coarse_pose,
                            double radius, const reloc_grid *grid, const reloc_camera *cam,
                            reloc_result *out, double *scores_host, float *best_rgb_dev,
                            float *best_depth_dev, float *best_alpha_dev, void *stream);

/* Random search with early stop (Sec. IV-A, initial relocalization): instead
 * of the whole grid, visit a share of its cells in random order, a batch at
 * a time, and stop after the first batch whose best NCC reaches a threshold.
 * The paper visits 20% of a 2 m x 10 deg grid over (-15, 15) m and a full
 * turn; it gives no threshold value, and its second stop test (enough
 * feature matches for the refinement) needs a learned matcher and is not
 * part of this call.
 *   fraction   share of the grid's cells visited, in (0, 1]; the visit is
 *              the first ceil(fraction * n_cells) cells of the order
 *   ncc_stop   stop after the batch in which the best NCC so far is >= this
 *              (+inf: never stop early)
 *   batch      cells rendered and scored together, 1..4096
 *   seed       the visiting order when `order` is NULL: the cells 0..n-1
 *              shuffled by Fisher-Yates (for i = n-1 down to 1, swap cell i
 *              with cell j = x mod (i + 1), x the next SplitMix64 output of
 *              a generator started at `seed`)
 *   order      explicit visiting order (cell indices, each in 0..n-1, no
 *              repeats), n_order entries, visited in full (fraction
 *              ignored); the caller keeps ownership
 */
typedef struct reloc_search {
    double fraction;
    double ncc_stop;
    int32_t batch;
    int32_t n_order;
    uint64_t seed;
    const int32_t *order;
    int32_t reserved[4];
} reloc_search;

/* Cells are numbered as in reloc_localize (index = ix + nx (iy + ny iyaw),
 * offsets centred on the coarse pose) but the grid may hold up to 2^20 cells.
 * out: best_index = best visited cell (highest NCC, lowest cell on ties),
 * n_candidates = cells in the grid, n_scored = cells visited, stopped_early.
 * scores_host[n_cells] (may be NULL) gets each visited cell's NCC and NaN for
 * the others.  The winner's images go to the *_dev buffers as in
 * reloc_localize.  The host reads the batch's scores after each batch (one
 * synchronisation per batch).  Errors: EINVAL (bad options, grid or order),
 * ENOMAP, ENUMERIC, ECUDA, EOVERFLOW. */
reloc_status reloc_localize_random(reloc_ctx *ctx, const float *query_dev, const double *coarse_pose,
                                   double radius, const reloc_grid *grid, const reloc_camera *cam,
                                   const reloc_search *search, reloc_result *out, double *scores_host,
                                   float *best_rgb_dev, float *best_depth_dev, float *best_alpha_dev,
                                   void *stream);

/* reloc_localize for callers holding HOST buffers: copies query_host
 * ([3][H][W]) to the device and the winner's RGB/depth back to best_rgb_host
 * ([3][H][W]) and best_depth_host ([H][W]) (either may be NULL), through the
 * context's own device buffers, on `stream`.  Pinned host memory makes the
 * copies asynchronous. */
reloc_status reloc_localize_host(reloc_ctx *ctx, const float *query_host, const double *coarse_pose,
                                 double radius, const reloc_grid *grid, const reloc_camera *cam,
                                 reloc_result *out, float *best_rgb_host, float *best_depth_host,
                                 void *stream);

/* Pose refinement step of Sec. III-C.2 without its learned matcher: the
 * caller supplies matched pixel pairs between a view rendered at
 * pose_render (its depth and alpha from reloc_render / reloc_localize) and
 * the query image; each render pixel is back-projected with the rendered
 * depth, and the query's world-to-camera pose is estimated from the
 * resulting 2D-3D pairs by Perspective-n-Point.  Iterating render -> match
 * -> refine is the paper's refinement loop.
 *   depth_dev, alpha_dev  [H][W] float32, device: Eq. (depth) D and
 *                         1 - T of the view (caller-owned)
 *   pairs_dev             [n_pairs][4] float32, device: (u_r, v_r, u_q, v_q)
 *                         pixel coordinates, pixel (x, y) centred at
 *                         (x + 0.5, y + 0.5)
 *   pose_init             world-to-camera start (typically pose_render)
 * Back-projection: D and A are sampled bilinearly at (u_r - 0.5, v_r - 0.5)
 * in pixel-index space (the 2 x 2 neighbourhood must lie in the image); a
 * pair is used when A >= alpha_min, with depth z = D / A and camera point
 * z ((u_r - cx) / fx, (v_r - cy) / fy, 1), mapped to the world by
 * pose_render.  PnP: minimise sum_i huber(|pi(W X_i) - (u_q, v_q)|) over W
 * (Huber threshold huber_px; points with camera z <= 1e-6 are ignored) by
 * iteratively reweighted Gauss-Newton in FP64: the update delta = (rho, phi)
 * solves (H + 1e-9 tr(H)/6 I) delta = -g, W <- [Exp(phi) R | Exp(phi) t +
 * rho]; a step that does not lower the cost is halved up to 10 times, then
 * the solve stops; it also stops when max |delta| < tol or after max_iters.
 * Errors: EINVAL (NULL pointer, n_pairs < 1, bad options), ENUMERIC
 * (non-finite pose or fewer than 3 usable pairs), ECUDA. */
typedef struct reloc_pnp_options {
    int32_t max_iters;         /* default 30                                          */
    int32_t reserved0;
    double huber_px;           /* default 2 px                                        */
    double alpha_min;          /* default 0.5                                         */
    double tol;                /* default 1e-12                                       */
    int32_t reserved[4];
} reloc_pnp_options;

typedef struct reloc_pnp_result {
    double pose[16];           /* refined world-to-camera pose                        */
    double rms_px;             /* RMS reprojection error of the used pairs (px)       */
    double cost;               /* final Huber cost                                    */
    int32_t n_used;            /* pairs with a usable depth                           */
    int32_t iters;             /* Gauss-Newton iterations run                         */
    int32_t reserved[2];
} reloc_pnp_result;

void reloc_default_pnp_options(reloc_pnp_options *opt);
reloc_status reloc_refine_pnp(reloc_ctx *ctx, const double *pose_render, const double *pose_init,
                              const reloc_camera *cam, const float *depth_dev, const float *alpha_dev,
                              const float *pairs_dev, int n_pairs, const reloc_pnp_options *opt,
                              reloc_pnp_result *out, void *stream);

/* ---- map training (Sec. III-B.3) ------------------------------------------
 * The loss of Eq. 6, L = w_photo L_photo + w_reproj L_reproj, with L_photo =
 * L_rgb(R(G, W_t), I_t) (Eq. 4) averaged over the training views and L_rgb =
 * (1 - lambda) L1 + lambda D-SSIM (Eq. 3); L1 is the mean absolute difference
 * over the 3 H W samples of a view.  The paper gives no values for lambda,
 * w_photo and w_reproj; the defaults are 3D Gaussian Splatting's lambda = 0.2
 * and w_photo = w_reproj = 1.  The derivative is that of the render with its
 * inclusion, alpha-skip, clamp and stop decisions fixed, and the right
 * derivative of |x| at 0.  D-SSIM = 1 - mean SSIM over the view's pixels
 * and channels, SSIM of Wang, Bovik, Sheikh and Simoncelli (2004) with an
 * 11 x 11 Gaussian window (standard deviation 1.5 px), samples outside the
 * image counting as 0, C1 = 0.01^2, C2 = 0.03^2.  L_reproj (Eq. 5) is read
 * as: for each pair of consecutive views (t, t+1) in the order given, a
 * pixel p of view t whose rendered alpha A (= sum w) reaches
 * reproj_alpha_min takes the depth d = D / A (D = sum w z, the depth
 * equation of Sec. III-A), is lifted to d ((x + 0.5 - cx) / fx, (y + 0.5 -
 * cy) / fy, 1), carried into view t+1 by the two poses and projected; in
 * front of the near plane, with its four bilinear neighbours (pixel centres
 * at +0.5) inside the image, the re-projected image at p is I_{t+1} sampled
 * bilinearly there, otherwise I_t(p); L_reproj averages L_rgb(re-projected
 * image, I_t) over the V - 1 pairs (0 when V = 1).  Its gradient reaches the
 * map through D and A.
 * Adam (Kingma and Ba 2015) updates 3D Gaussian Splatting's latent
 * parameters: mean, log scale, quaternion (as stored; normalised on use),
 * logit opacity, colour, each group with its own learning rate; the scale
 * and opacity stored in the map are the activated values. */
typedef struct reloc_train_options {
    double lambda_dssim;       /* lambda of Eq. 3: 0.2                                */
    double w_photo, w_reproj;  /* omega_1, omega_2 of Eq. 6: 1, 1                     */
    double lr_mean;            /* metres per step: 1.6e-4                             */
    double lr_scale;           /* log-scale per step: 5e-3                            */
    double lr_quat;            /* 1e-3                                                */
    double lr_opacity;         /* logit per step: 5e-2                                */
    double lr_color;           /* 2.5e-3                                              */
    double beta1, beta2, eps;  /* Adam: 0.9, 0.999, 1e-15                             */
    double reproj_alpha_min;   /* pixels of L_reproj need rendered alpha >= this: 0.5 */
    int32_t views_per_group;   /* views rendered per group (one gathered copy of the
                                  subset each; bounds the workspace): 16              */
    int32_t reserved[7];
} reloc_train_options;

void reloc_default_train_options(reloc_train_options *opt);

/* The loss over n_views training views at poses[n_views][16] (world-to-camera,
 * row-major, host) of the Gaussians in `ranges` (the block-ordered map;
 * reloc_select_block or [0, n)), against targets_dev[n_views][3][H][W]
 * (device, FP32, channel-planar), written to *loss_host, and its gradient
 * with respect to every Gaussian's parameters written to grad_dev[14][n]
 * (device, FP32, zeroed by the call first; rows: mean x, y, z, scale x, y,
 * z, quaternion w, x, y, z, opacity, red, green, blue; columns in block
 * order; Gaussians outside `ranges` get 0).  The map must have SH degree 0
 * and FP32 attributes.  Per-Gaussian sums are FP32 atomics (their order
 * varies from call to call).  Synchronous on `stream`.  Errors: EINVAL,
 * ENOMAP, ENUMERIC, ECUDA, EOVERFLOW. */
reloc_status reloc_train_grad(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges,
                              const double *poses, int n_views, const reloc_camera *cam,
                              const float *targets_dev, const reloc_train_options *opt,
                              double *loss_host, float *grad_dev, void *stream);

/* One training step: the loss and gradient as reloc_train_grad (into a
 * context-owned buffer), then one Adam step on the device map.  *loss_host is
 * the loss before the step.  The Adam moments and step count live in the
 * context; reloc_load_map and reloc_train_reset start them afresh.  The map's
 * block partition is not rebuilt: reload the map read back with
 * reloc_read_map to re-partition moved Gaussians.  opt NULL: defaults.
 * Synchronous on `stream`.  Errors: as reloc_train_grad. */
reloc_status reloc_train_step(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges,
                              const double *poses, int n_views, const reloc_camera *cam,
                              const float *targets_dev, const reloc_train_options *opt,
                              double *loss_host, void *stream);
reloc_status reloc_train_reset(reloc_ctx *ctx);

/* Copy the device map back to host arrays in block order (reloc_map_order
 * gives each row's original index), in the layout of reloc_gaussians_host:
 * mean[n][3], scale[n][3], quat[n][4], opacity[n], sh[n][K][3]; any pointer
 * may be NULL.  FP32 maps only.  Errors: EINVAL, ENOMAP, ECUDA. */
reloc_status reloc_read_map(reloc_ctx *ctx, float *mean, float *scale, float *quat, float *opacity,
                            float *sh);

/* One query of a batch (Sec. III-C.1 applied to many queries at once). */
typedef struct reloc_query {
    const float *query_dev;    /* [3][H][W] device image of the query (caller-owned)   */
    double coarse_pose[16];    /* world-to-camera coarse pose                          */
    double radius;             /* block-selection radius around its camera centre, m   */
    reloc_grid grid;           /* candidate grid (counts may differ between queries)   */
} reloc_query;

/* reloc_localize for n_queries queries at once, each with its own subset and
 * candidate count.  Every stage runs as one launch over all (query, candidate)
 * views of a sub-batch; sub-batches are formed so that their workspace stays
 * within the memory budget of reloc_set_batch_options, and (use_graph) the
 * launches of the whole call are captured and replayed as one CUDA graph.
 * results[n_queries] (host) as reloc_localize; scores_host, if not NULL,
 * receives every candidate's NCC in query order (sum of candidate counts);
 * best_rgb_dev [n_queries][3][H][W] and best_depth_dev [n_queries][H][W]
 * (device, may be NULL) receive the winners.  Results equal those of
 * n_queries separate reloc_localize calls.  Errors: as reloc_localize. */
reloc_status reloc_localize_batch(reloc_ctx *ctx, const reloc_query *queries, int n_queries,
                                  const reloc_camera *cam, reloc_result *results, double *scores_host,
                                  float *best_rgb_dev, float *best_depth_dev, void *stream);

typedef struct reloc_batch_options {
    int32_t use_graph;         /* capture each batch call in one CUDA graph: 1          */
    int32_t reserved0;
    int64_t mem_budget;        /* workspace bytes per sub-batch (>= 64 MiB): 16 GiB     */
    int32_t reserved[8];
} reloc_batch_options;

/* Set the batch options of the context.  Errors: EINVAL. */
reloc_status reloc_set_batch_options(reloc_ctx *ctx, const reloc_batch_options *opt);

typedef struct reloc_tune_result {
    int32_t tile_w, tile_h;    /* chosen blend tile                                     */
    int32_t blend_rpl;         /* chosen records per lane per warp step                 */
    int32_t from_table;        /* 1: taken from the table without timing                */
    double ms_per_query;       /* measured (or tabled) time per sample query            */
    int32_t n_tried;           /* configurations timed                                  */
    int32_t reserved[5];
} reloc_tune_result;

/* Autotuner (no counterpart in the paper: a scheduling choice of this build).
 * Times reloc_localize_batch on the sample queries with every supported
 * (tile_w, tile_h, blend_rpl) -- 16x16, 8x8, 32x8, 16x8, 8x16, 32x16 tiles,
 * 1 or 2 records per lane -- and keeps the fastest in the context's config.
 * table_path (may be NULL): a text table keyed by image size, SH degree,
 * precision and the log2 buckets of the sample's mean candidate count and
 * subset size; a matching line is used without timing unless force != 0, and
 * a timed result is appended.  Runs on `stream`, synchronises it.
 * Errors: EINVAL, ENOMAP, ECUDA (no configuration ran). */
reloc_status reloc_autotune(reloc_ctx *ctx, const reloc_query *sample, int n_sample, const reloc_camera *cam,
                            const char *table_path, int force, reloc_tune_result *out, void *stream);

/* ---- learned candidate proposal ------------------------------------------
 * No counterpart in the paper (its Sec. II points at learned relocalization
 * as related work): a CNN ranks the 64 cells of a 4 x 4 x 4 candidate grid
 * from gray 176 x 47 views (box average over f x f pixels, f = H / 47 =
 * W / 176) of the query and of the render at the coarse pose; only the top-k
 * cells are rendered and scored, and the full 64-candidate sweep runs
 * whenever the softmax margin p1 - p2 is below the threshold.  Architecture:
 * five 3x3 stride-2 convolutions 2-32-64-64-128-128 with ReLU, FC 1536-1024
 * ReLU, FC 1024-64; BF16 weights and activations, FP32 accumulation on the
 * tensor cores; softmax cross-entropy; Adam.  Flat parameter layout (FP32,
 * RELOC_PROPOSAL_PARAMS values): per conv layer W[Cout][3][3][Cin], b[Cout];
 * FC1 W[1024][1536], b[1024]; FC2 W[64][1024], b[64].  Network input: NHWC
 * BF16 [batch][47][176][2] (channel 0 query, 1 coarse render), passed as
 * uint16_t bit patterns. */
#define RELOC_PROPOSAL_H 47
#define RELOC_PROPOSAL_W 176
#define RELOC_PROPOSAL_CLASSES 64
#define RELOC_PROPOSAL_PARAMS 1916960

/* Create (or re-create) the network with He-normal weights from `seed`.
 * Errors: ENOMEM, ECUDA. */
reloc_status reloc_proposal_init(reloc_ctx *ctx, uint64_t seed);

/* Copy the parameters (which = 0) or the gradients of the last train step
 * (which = 1) to flat_host [RELOC_PROPOSAL_PARAMS], or load parameters from
 * it (reloc_proposal_set_params, which also resets the Adam state).
 * Errors: EINVAL (no network), ECUDA. */
reloc_status reloc_proposal_get(reloc_ctx *ctx, int which, float *flat_host);
reloc_status reloc_proposal_set_params(reloc_ctx *ctx, const float *flat_host);

/* Network input of one sample from a query image and the render at its coarse
 * pose (both [3][H][W] device, H = 47 f, W = 176 f) into input_dev
 * [47][176][2].  Errors: EINVAL. */
reloc_status reloc_proposal_make_input(reloc_ctx *ctx, const float *query_dev, const float *coarse_rgb_dev,
                                       const reloc_camera *cam, uint16_t *input_dev, void *stream);

/* Logits [batch][64] (FP32, device) of inputs_dev [batch][47][176][2]. */
reloc_status reloc_proposal_forward(reloc_ctx *ctx, const uint16_t *inputs_dev, int batch, float *logits_dev,
                                    void *stream);

/* One training step on a batch (batch a multiple of 64): forward, mean
 * softmax cross-entropy against labels_dev [batch] (int32 grid cell), backward;
 * Adam update with learning rate lr if update != 0.  *loss_host = mean loss.
 * Synchronises `stream`.  Errors: EINVAL, ECUDA, ETIMEOUT (a tensor-core wait
 * gave up). */
reloc_status reloc_proposal_train_step(reloc_ctx *ctx, const uint16_t *inputs_dev, const int32_t *labels_dev,
                                       int batch, float lr, int update, float *loss_host, void *stream);

/* The proposal's dense contraction, exposed for callers and checks:
 * C[m][n] = sum_k A[m][k] B[n][k] (+ bias[n], ReLU if relu != 0), A [M][K] and
 * B [N][K] row-major BF16 (uint16_t bit patterns, 16-byte aligned), C [M][N]
 * FP32, all device; FP32 accumulation on the tensor cores (tcgen05).  K a
 * multiple of 64; split_k > 1 splits K into that many parts (K / split_k a
 * multiple of 64) summed in a fixed order.  Synchronises `stream`.
 * Errors: EINVAL, ECUDA, ETIMEOUT (a tensor-core wait gave up). */
reloc_status reloc_gemm_bf16(reloc_ctx *ctx, const uint16_t *A_dev, const uint16_t *B_dev, const float *bias_dev,
                             float *C_dev, int M, int N, int K, int relu, int split_k, void *stream);

/* Use the proposal in reloc_localize / reloc_localize_batch for queries with a
 * 4 x 4 x 4 grid: render and score the top_k (2..32) cells, or all 64 when
 * p1 - p2 < margin.  enabled = 0 restores the full sweep.  Errors: EINVAL. */
reloc_status reloc_set_proposal(reloc_ctx *ctx, int enabled, int top_k, float margin);

/* Work counts of the last render/score/localize call. */
reloc_status reloc_last_counts(reloc_ctx *ctx, reloc_counts *out);

/* Stage timing with CUDA events on the call's stream: enable (1) or disable
 * (0) and reset the accumulators.  reloc_stage_times writes, for each stage
 * s < RELOC_STAGE_COUNT, the accumulated milliseconds ms_out[s] and the
 * number of timed calls calls_out[s] since the last reset (either may be NULL). */
reloc_status reloc_set_profiling(reloc_ctx *ctx, int enabled);
reloc_status reloc_stage_times(reloc_ctx *ctx, double *ms_out, int64_t *calls_out);

/* Copy intermediate results of the LAST render/score/localize call, for
 * parity checks (device pointers, any may be NULL; sizes from reloc_last_counts):
 *   records_dev [n_views][n_gauss][12] float: u, v, depth, log2(opacity),
 *                k alpha_x, k alpha_y, k beta_x, k beta_y, red, green, blue, 0
 *                (alpha, beta: the footprint's principal axes scaled by the
 *                inverse square roots of the dilated Sigma''s eigenvalues,
 *                so that the conic Sigma'^-1 = alpha alpha^T + beta beta^T
 *                and the power is -((alpha . d)^2 + (beta . d)^2) / 2;
 *                k = sqrt(log2(e) / 2), the blend's base-2 scale; valid where
 *                visible)
 *   rects_dev   [n_views][n_gauss][4] int32: tile rectangle tx0, ty0, tx1, ty1
 *                inclusive; all -1 where not visible
 *   inst_tiles_dev / inst_gauss_dev [n_views][inst_stride] uint32: the sorted
 *                tile list of each view (tile id, Gaussian subset index);
 *                entries past the view's count are undefined
 *   inst_count_host [n_views] int64: instances per view
 *   ranges_dev  [n_views][n_tiles][2] int32: [begin, end) of each tile in the
 *                view's sorted list (relative to the view), empty = [0, 0).
 * Synchronises `stream`. */
reloc_status reloc_export_debug(reloc_ctx *ctx, float *records_dev, int32_t *rects_dev,
                                uint32_t *inst_tiles_dev, uint32_t *inst_gauss_dev,
                                int64_t *inst_count_host, int32_t *ranges_dev, void *stream);

/* Fault injection for failure-detection tests.  The paper has no
 * counterpart: it lets a test make the library's failure paths run without
 * faulting the GPU.  Process-wide; count = 0 clears a kind.
 *   RELOC_FAULT_GEMM_WAIT  the next `count` tensor-core GEMM launches (the
 *                          proposal's and reloc_gemm_bf16's) have their MMA
 *                          lanes wait on a barrier that nothing completes:
 *                          each CTA gives up after the wait limit (about a
 *                          second), issues no MMA, waits for its own copies
 *                          in flight, frees its tensor memory and records the
 *                          failure; the call returns RELOC_ETIMEOUT and the
 *                          context stays usable.
 *   RELOC_FAULT_ALLOC      the next `count` device allocations fail; the call
 *                          that needed them returns RELOC_ENOMEM and the
 *                          context stays usable.
 * Errors: EINVAL (unknown kind, count < 0). */
#define RELOC_FAULT_GEMM_WAIT 1
#define RELOC_FAULT_ALLOC 2
reloc_status reloc_inject_faults(int kind, int count);

/* Measured arithmetic throughput of `device`, the denominators of the
 * projection's and the blend's rooflines.  The paper has no counterpart: it
 * is a measurement utility.  Register-resident microbenchmarks (independent
 * dependency chains per thread, four waves of the SM count) give
 *   fp32_scalar_tflops  FP32 fused multiply-add, 2 flop each (TFLOP/s)
 *   fp32_packed_tflops  the same with packed two-lane f32x2 FMAs (TFLOP/s)
 *   ex2_gops            base-2 exponentials, ex2.approx (10^9 per second)
 * Any output pointer may be NULL.  Takes some milliseconds, allocates 1 KB
 * of device memory for the duration of the call and synchronises the
 * device.  Errors: ECUDA (no such device or a launch failure). */
reloc_status reloc_measure_peaks(int device, double *fp32_scalar_tflops, double *fp32_packed_tflops,
                                 double *ex2_gops);

/* NCC of already-rendered images against a query, without allocating.
 * The paper has no counterpart: this entry point is for callers that must not
 * allocate device memory after start-up -- e.g. a real-time relocalization
 * loop whose memory is reserved up front (cudaMalloc/cudaFree may synchronise
 * the whole device and take milliseconds) or a process whose device memory
 * belongs to another framework's pool.  For images the caller rendered it
 * computes the Pearson correlation of each image with the query over all
 * 3*H*W samples (the RGB score of reloc_score with ncc_gray = 0; the gray
 * option is not offered here), with every per-sample sum in FP64, and score 0
 * with degenerate = 1 for a zero-variance image.  reloc_score sums each
 * 64-pixel block in compensated FP32 before its FP64 combine, so the two agree
 * to rounding (within 2e-6), not bit for bit.
 *   images_dev      [n_views][3][height][width] float32, device, caller-owned
 *   query_dev       [3][height][width] float32, device, caller-owned
 *   scores_dev      [n_views] double, device, written (caller-owned)
 *   degenerate_dev  [n_views] int, device, written (may be NULL)
 * Its only scratch is a fixed 393,728-byte device array inside the library,
 * held by every GPU that loads the library until the process exits; no
 * cudaMalloc, cudaFree or allocating library routine is called.  The first
 * call on a device looks up that array's device address (with the device
 * current) and should come before any stream capture.  Asynchronous on
 * `stream`.  All calls share the one array: calls that overlap on the GPU
 * race and must be ordered by the caller.  Errors: EINVAL (NULL pointer,
 * n_views outside 1..RELOC_NOALLOC_MAX_VIEWS, image size outside 1..16383),
 * ECUDA. */
#define RELOC_NOALLOC_MAX_VIEWS 512
reloc_status reloc_ncc_images_noalloc(const float *images_dev, int n_views, int height, int width,
                                      const float *query_dev, double *scores_dev, int *degenerate_dev,
                                      void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RELOC_H */
