// internal.cuh -- declarations shared by the translation units of libreloc.
//
// Data layout in device memory (one context, one GPU):
//   map        mean x/y/z: float[N] each (SoA), block-ordered;
//              attr: storage type T (float | __half | __nv_bfloat16),
//              component-major [NCOMP][N]: scale 0..2, quat 3..6 (w,x,y,z),
//              opacity 7, SH coefficient k channel ch at 8 + 3k + ch.
//   per call   V views over a subset of S Gaussians; every per-(view, Gaussian)
//              array is view-major with stride S; every per-(view, instance)
//              array is view-major with stride inst_stride.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace reloc {

constexpr int ATTR_SCALE = 0;
constexpr int ATTR_QUAT = 3;
constexpr int ATTR_OPAC = 7;
constexpr int ATTR_SH = 8;
inline int attr_components(int sh_degree) { return ATTR_SH + 3 * (sh_degree + 1) * (sh_degree + 1); }

// One candidate view.  The camera centre is split into a float head and tail
// (c = hi + lo) so mu - c is formed to ~1e-7 relative of |mu - c| even for
// maps hundreds of metres from the origin.
struct ViewParams {
    float R[9];        // world-to-camera rotation, row-major
    float c_hi[3];
    float c_lo[3];
    float pad;
};
static_assert(sizeof(ViewParams) == 64, "ViewParams is 64 bytes");

struct CamParams {
    int width, height, ntx, nty, tile_w, tile_h, n_tiles, tile_bits;
    float fx, fy, cx, cy, limx, limy;
    float near_plane, eps2d, cut, det_fp64;
    float alpha_min, alpha_max, t_min;
    int blend_rpl;     // records per lane per warp step in K6 (1 or 2)
    int ncc_gray;      // NCC over gray values (R + G + B) / 3 instead of RGB samples
    int bin_chunk;     // depth-ordered Gaussians per tile-binning chunk (K3, K4)
};

// Stable LSD radix sort over view-strided segments (sort.cu).
constexpr int SORT_THREADS = 256;
constexpr int SORT_IPT = 8;
constexpr int SORT_CHUNK = SORT_THREADS * SORT_IPT;   // 2048 items per block
constexpr int RADIX = 256;
// Tile binning (sort.cu): chunks of bin_chunk depth-ordered Gaussians.
constexpr int BIN_CHUNK_MIN = 2048;
constexpr int BIN_TILES_PER_CHUNK_STEP = 8192;        // bin_chunk grows by 2048 per 8192 tiles
constexpr int TILE_COUNT_SMEM = 48 * 1024;            // difference-array band
constexpr int TILE_EMIT_WARPS = 8;                    // tile rows per K4 block
constexpr int TILE_EMIT_SMEM_MAX = 64 * 1024;         // slot counters: 8 rows x ntx <= 2048

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---- per-call layout ----------------------------------------------------------
// A call renders Q queries (each: a Gaussian subset and V_q candidate views)
// in one pass of every stage.  Views are numbered 0..V-1 across the queries
// of the call; every per-(view, Gaussian) array places view v at vd_off[v]
// (length S of its query) and every per-(view, instance) array at io_off[v]
// (capacity io_off[v+1] - io_off[v]).  The chunk bases map a block index to
// its view and chunk for the sort, binning and scan kernels.  All tables are
// built on the host and live in device memory for the call.
struct Layout {
    int Q, V;
    const int32_t *view_q;     // [V]   query of each view
    const int64_t *vd_off;     // [V+1] dense offsets
    const int64_t *io_off;     // [V+1] instance offsets
    const int32_t *c1_base;    // [V+1] depth-sort chunk base (SORT_CHUNK)
    const int32_t *cb_base;    // [V+1] tile-binning chunk base (bin_chunk)
    const int64_t *q_gsub;     // [Q+1] subset offsets into the gathered index list
    const int32_t *q_view;     // [Q+1] first view of each query
    const int32_t *q_pblk;     // [Q+1] projection block base
    const float *const *q_img; // [Q]   query images (device pointers) or null
};

// Largest s in [0, n] with base[s] <= x (base ascending): the segment of x.
__device__ __forceinline__ int find_segment(const int32_t *base, int n, int x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int PROJ_THREADS = 128;

// ---- launchers (each returns the launch error) -------------------------------

// K1: subset gather.  run_begin/run_off: n_runs block-ordered runs and their
// exclusive prefix of lengths (device); writes gidx[total] map positions.
cudaError_t launch_gather_subset(const int64_t *run_begin, const int64_t *run_off, int n_runs,
                                 int64_t total, uint32_t *gidx, cudaStream_t st);

// K2: projection of every query's subset into that query's views.
// n_blocks = q_pblk[Q] (host copy).
cudaError_t launch_project(const float *mx, const float *my, const float *mz, const void *attr,
                           int precision, int sh_degree, int64_t n_map, const uint32_t *gidx,
                           const Layout &L, int n_blocks, const ViewParams *views, const CamParams &cam,
                           float4 *rec, uint2 *rect, uint32_t *dkey, cudaStream_t st);

// Stable LSD radix sort pass over segments (views).  Segment s holds
// seg_off[s+1] - seg_off[s] slots at seg_off[s], of which len[s] are valid
// (len null: all).  filt != null: pass over dense arrays keeping items with
// filt != 0 and implicit values (the index in the segment); len_out receives
// the kept counts.  hist: RADIX words per chunk.
struct RadixPass {
    // drop_culled: pass over dense (view, Gaussian) arrays, dropping keys of
    // 0xFFFFFFFF (culled pairs; visible depth keys are positive finite floats)
    const uint32_t *keys_in, *vals_in, *len;
    int drop_culled;
    uint32_t *keys_out, *vals_out, *len_out, *hist;
    uint32_t *dtot;    // per (segment, digit) totals of the pass, zeroed by the caller
    const int64_t *seg_off;
    const int32_t *chunk_base;
    int n_seg, total_chunks, shift;
    uint32_t mask;
};
cudaError_t launch_radix_pass(const RadixPass &p, cudaStream_t st);

// K3: per chunk of each view's depth-ordered visible Gaussians (sorted_g,
// n_vis[v] at vd_off[v]) the number covering each tile -> bhist[chunk][tile]
// (n_chunks = cb_base[V], host copy); rectangles in depth order -> srect;
// then per view the chunk prefix per tile (in place), ranges[v][tile] =
// [begin, end) of the tile's list relative to io_off[v] (empty [0, 0)) and
// n_inst[v].  A view over its capacity sets *overflow.
cudaError_t launch_tile_count(const uint32_t *sorted_g, const uint32_t *n_vis, const uint2 *rect, const Layout &L,
                              const CamParams &cp, int n_chunks, uint2 *srect, uint32_t *bhist, int2 *ranges,
                              uint32_t *n_inst, int *overflow, cudaStream_t st);

// K4: every (tile, Gaussian) instance into inst_gauss at io_off[v] + its slot,
// each tile's list in (depth, index) order.  Views over capacity emit nothing.
cudaError_t launch_tile_emit(const uint32_t *sorted_g, const uint2 *srect, const uint32_t *n_vis,
                             const uint32_t *n_inst, const uint32_t *bhist, const int2 *ranges, const Layout &L,
                             const CamParams &cp, int n_chunks, uint32_t *inst_gauss, cudaStream_t st);

// Allow K4 its largest shared-memory footprint (once per device, before any capture).
cudaError_t configure_tile_kernels();

// Pose refinement by PnP on one view's depth (pnp.cu), one cooperative launch:
// out_dev[20] = pose[16], rms, cost, n_used, iterations; X_scratch: 4 doubles
// per pair, then per-block sums and the solver state (under 256 KB).
cudaError_t launch_refine_pnp(const double *pose_render, const double *pose_init, double fx, double fy, double cx,
                              double cy, int width, int height, const float *depth, const float *alpha,
                              const float *pairs, int n, int max_iters, double huber, double alpha_min, double tol,
                              double *X_scratch, double *out_dev, cudaStream_t st);

// FP32 (scalar and packed) FMA and ex2 throughput of the current device (peaks.cu).
cudaError_t measure_peaks(double *fp32_scalar_tflops, double *fp32_packed_tflops, double *ex2_gops);

// Tile id of each instance of one view from its ranges (debug export).
cudaError_t launch_fill_tiles(const int2 *ranges_view, int n_tiles, uint32_t *tiles_view, cudaStream_t st);

// Query statistics S_q, S_qq over n samples of each of the Q query images
// -> qstats[Q][2] (double).  block_scratch: Q * 2 * 152 doubles.
// Query sums (sum q, sum q^2) over its 3 H W samples, or over its H W gray
// values (R + G + B) / 3 when gray.
cudaError_t launch_query_stats(const Layout &L, int64_t HW, bool gray, double *block_scratch, double *qstats,
                               cudaStream_t st);

// K6 (+ K7 partials): blend every (view, tile) of the layout, a warp per
// 64-pixel block; optional image export (slot = view) and NCC partials
// [V][blend_units(cam)][3] = {S_r, S_rr, S_rq} per warp block.
// view_sel != null: blend only the n_sel views view_sel[0..n_sel), image
// slot k for view_sel[k].  queue: blend_queue_ints(cam, n) device ints for n
// views, the launch's work counter and list of heavy tiles (zeroed on the
// stream as needed).  blend_launches(n) launches.
cudaError_t launch_blend(const float4 *rec, const Layout &L, const uint32_t *inst_gauss, const int2 *ranges,
                         const CamParams &cam, double *partials, float *rgb, float *depth, float *alpha,
                         const int *view_sel, int n_sel, const int *overflow, int *queue, cudaStream_t st);

// 64-pixel warp blocks of one view: the blend's unit of work and of NCC partials.
inline int blend_units(const CamParams &cam) { return cam.n_tiles * (cam.tile_w * cam.tile_h / 64); }
// Units (64-pixel blocks over all views) of one blend launch at most: the
// work queue's tickets (heavy units counted twice) and its heavy-tile
// entries stay far inside int32.  Sub-batches are cut to respect it.
constexpr int64_t BLEND_MAX_UNITS = (int64_t)1 << 29;
// Work-queue ints of a blend launch over n views.
inline int64_t blend_queue_ints(const CamParams &cam, int64_t n) { return 4 + n * cam.n_tiles; }
// Kernel launches of a blend over n views: the heavy-tile listing runs for
// launches of several views (a one-view launch ends on its longest unit
// whatever the order).
__host__ __device__ __forceinline__ int blend_launches(int64_t n) { return n >= 4 ? 2 : 1; }

// K7: NCC per view from its n_units partials and its query's statistics;
// coef (may be null): [V][4] = 1/sqrt(var_r var_q), NCC/var_r, mean r, mean q.
cudaError_t launch_ncc_finalize(const double *partials, const double *qstats, const Layout &L, int n_units,
                                int64_t n_samples, double *scores, int *degenerate, double *coef, cudaStream_t st);

// K6 backward: per (view, Gaussian) gradients with respect to the projected
// mean and conic.  gimg null: of the view's NCC (coef from K7), added into
// gout[vd_off[v] + i][5] (u, v, a, b, c).  gimg [V][3][H][W] = dL/dC of an
// image loss (gda [V][2][H][W] = dL/d(depth, alpha), may be null): added into
// gout[vd_off[v] + i][10] (u, v, a, b, c, r, g, b, opacity, z); cimg (may be
// null) [V][3][H][W] the views' forward render (cdep, calp [V][H][W] its depth
// and alpha, needed with gda) so the colour need not be composited again.
cudaError_t launch_blend_grad(const float4 *rec, const Layout &L, const uint32_t *inst_gauss, const int2 *ranges,
                              const CamParams &cam, const double *coef, const float *gimg, const float *gda,
                              const float *cimg, const float *cdep, const float *calp, float *gout,
                              const int *overflow, cudaStream_t st);

// Chain of gin to each view's left pose update: out[V][6] (rho, phi);
// part: n_blocks * V * 6 doubles of scratch.
cudaError_t launch_pose_chain(const float *mx, const float *my, const float *mz, const void *attr, int precision,
                              int64_t n_map, const uint32_t *gidx, const Layout &L, int n_blocks,
                              const ViewParams *views, const CamParams &cam, const float *gin, double *part,
                              double *out, cudaStream_t st);

// ---- map training (train.cu) -------------------------------------------------
// L1 samples: loss += scale * sum |rgb - target|, gimg (=|+=) scale * sign.
cudaError_t launch_photo_l1(const float *rgb, const float *target, int64_t n, double scale, float *gimg,
                            bool accumulate, double *loss, cudaStream_t st);
// D-SSIM over planes channel planes [H][W]: loss += scale * sum (1 - SSIM),
// gimg += its gradient; abc: 3 * planes * H * W floats of scratch.
cudaError_t launch_ssim(const float *rgb, const float *target, int planes, int H, int W, double scale, float *abc,
                        float *gimg, double *loss, cudaStream_t st);
// Re-projection of Eq. 5 for n_views consecutive pairs: targets holds views
// 0 .. n_views (n_views + 1 images), rel [n_views][12] the relative poses;
// warped, jac [n_views][3][H][W]; then gda [n_views][2][H][W] = dL/d(D, A).
cudaError_t launch_reproj_warp(const float *dep, const float *alp, const float *targets, const float *rel,
                               int n_views, const CamParams &cam, float alpha_min, float *warped, float *jac,
                               cudaStream_t st);
cudaError_t launch_reproj_back(const float *gw, const float *jac, const float *dep, const float *alp, int n_views,
                               int64_t HW, float alpha_min, float *gda, cudaStream_t st);
// gin [VS][10] (launch_blend_grad, image mode) -> gmap [14][n_map] (added):
// mean xyz, scale xyz, quat wxyz, opacity, rgb.  FP32 attributes only.
cudaError_t launch_param_chain(const float *mx, const float *my, const float *mz, const float *attr, int64_t n_map,
                               const uint32_t *gidx, const Layout &L, int n_blocks, const ViewParams *views,
                               const CamParams &cam, const float *gin, float *gmap, cudaStream_t st);
struct AdamParams {
    float lr[5];          // mean, scale, quaternion, opacity, colour
    float beta1, beta2, eps, bc1, bc2, o_min;
};
cudaError_t launch_adam(float *mean, float *attr, const float *grad, float *m1, float *m2, int64_t n,
                        const AdamParams &P, cudaStream_t st);

// K8: per query, argmax over its views (lowest index on ties):
// best[q] (index within the query), best_score[q], view_sel[q] (view index).
cudaError_t launch_argmax(const double *scores, const Layout &L, int *best, double *best_score, int *view_sel,
                          cudaStream_t st);

// ---- learned candidate proposal (proposal.cu, cnn.cu, gemm.cu) ----------------
constexpr int PROPOSAL_H = 47;
constexpr int PROPOSAL_W = 176;
constexpr int PROPOSAL_CLASSES = 64;
struct ProposalNet;
int64_t proposal_param_count();
ProposalNet *proposal_create(uint64_t seed, cudaError_t *err);
void proposal_destroy(ProposalNet *P);
cudaError_t proposal_get(const ProposalNet *P, int which, float *flat);   // 0 params, 1 grads
cudaError_t proposal_set(ProposalNet *P, const float *flat);
cudaError_t proposal_forward(ProposalNet *P, const __nv_bfloat16 *in, int B, float *out, cudaStream_t st);
cudaError_t proposal_train_step(ProposalNet *P, const __nv_bfloat16 *in, const int32_t *labels, int B, float lr,
                                bool update, float *loss_rows_dev, cudaStream_t st);
const float *proposal_logits(const ProposalNet *P);
int *proposal_status(const ProposalNet *P);
cudaError_t proposal_make_input(const float *query, const float *seed_rgb, int H, int W, __nv_bfloat16 *out,
                                cudaStream_t st);
cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias, float *Cf,
                             __nv_bfloat16 *Cb, int M, int N, int K, int lda, int ldb, int ldc, int relu, int split_k,
                             float *partials, int *status, cudaStream_t st, int inject = 0);

// Fault injection for tests (reloc_inject_faults): the number of upcoming
// GEMM launches whose tensor-core waits are made to run out, and of upcoming
// device allocations made to fail.  take_fault consumes one if any is set.
enum { FAULT_GEMM_WAIT = 0, FAULT_ALLOC = 1, FAULT_KINDS = 2 };
bool take_fault(int kind);
cudaError_t launch_topk(const float *logits, int B, int C, int k, int32_t *idx, float *margin, cudaStream_t st);

// Record msg as the calling thread's last error; returns st.
int reloc_internal_fail(int st, const char *msg);

}  // namespace reloc
