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
};

// Stable LSD radix sort over view-strided segments (sort.cu).
constexpr int SORT_THREADS = 256;
constexpr int SORT_IPT = 16;
constexpr int SORT_CHUNK = SORT_THREADS * SORT_IPT;   // 4096 items per block
constexpr int RADIX = 256;
constexpr int EMIT_THREADS = 256;
constexpr int EMIT_IPT = 8;
constexpr int EMIT_CHUNK = EMIT_THREADS * EMIT_IPT;   // 2048 items per block

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---- launchers (each returns the launch error) -------------------------------

// K1: subset gather.  run_begin/run_off: n_runs block-ordered runs and their
// exclusive prefix of lengths (device); writes gidx[S] map positions.
cudaError_t launch_gather_subset(const int64_t *run_begin, const int64_t *run_off, int n_runs,
                                 int64_t S, uint32_t *gidx, cudaStream_t st);

// K2: projection of S Gaussians into V views.
cudaError_t launch_project(const float *mx, const float *my, const float *mz, const void *attr,
                           int precision, int sh_degree, int64_t n_map, const uint32_t *gidx,
                           int64_t S, const ViewParams *views, int V, const CamParams &cam,
                           float4 *rec, uint2 *rect, uint32_t *ntiles, uint32_t *dkey,
                           cudaStream_t st);

// Radix sort pass over V segments of stride `stride`.  filt != null: first
// pass over dense (view, Gaussian) arrays keeping items with filt != 0 and
// implicit values (the Gaussian index); len_out receives the kept counts.
// len == null: every segment is `stride` long.
struct RadixPass {
    const uint32_t *keys_in, *vals_in, *filt, *len;
    uint32_t *keys_out, *vals_out, *len_out;
    uint32_t *hist;           // [V][RADIX][cps] scratch
    int64_t stride;
    int V, cps, shift;
    uint32_t mask;
};
cudaError_t launch_radix_pass(const RadixPass &p, cudaStream_t st);
int64_t radix_hist_words(int V, int64_t stride);

// K3: scan of tile counts in depth order + instance emission.
// sorted_g: [V][S] Gaussian indices in depth order (n_vis[v] valid),
// ntiles/rect: dense [V][S]; writes inst_tile/inst_gauss [V][inst_stride] in
// (depth, index) order and n_inst[V].  If a view needs more than inst_stride
// entries nothing is emitted for it, *overflow is set and *need raised.
cudaError_t launch_emit(const uint32_t *sorted_g, const uint32_t *n_vis, const uint32_t *ntiles,
                        const uint2 *rect, int64_t S, int V, int ntx, int64_t inst_stride,
                        uint32_t *chunk_sums, uint32_t *inst_tile, uint32_t *inst_gauss,
                        uint32_t *n_inst, unsigned long long *need, int *overflow, cudaStream_t st);
int64_t emit_chunk_words(int V, int64_t S);

// K5: per (view, tile) [begin, end) into the sorted instance list.
cudaError_t launch_ranges(const uint32_t *inst_tile, const uint32_t *n_inst, int64_t inst_stride,
                          int V, int n_tiles, int2 *ranges, const int *overflow, cudaStream_t st);

// Query statistics S_q, S_qq over 3*H*W samples -> qstats[2] (double).
cudaError_t launch_query_stats(const float *query, int64_t n, double *block_scratch, double *qstats,
                               cudaStream_t st);

// K6 (+ K7 partials): blend every (view, tile); optional image export and NCC
// partials [V][n_tiles][3] = {S_r, S_rr, S_rq}.  view_sel != null: render only
// the view *view_sel (grid has one view), writing images at view slot 0.
cudaError_t launch_blend(const float4 *rec, int64_t S, const uint32_t *inst_gauss, int64_t inst_stride,
                         const int2 *ranges, int V, const CamParams &cam, const float *query,
                         double *partials, float *rgb, float *depth, float *alpha,
                         const int *view_sel, const int *overflow, cudaStream_t st);

// K7: NCC per view from partials and the query statistics.
cudaError_t launch_ncc_finalize(const double *partials, const double *qstats, int V, int n_tiles,
                                int64_t n_samples, double *scores, int *degenerate, cudaStream_t st);

// K8: argmax (lowest index on ties) -> best[0] = index, best_score[0].
cudaError_t launch_argmax(const double *scores, int V, int *best, double *best_score, cudaStream_t st);

// Record msg as the calling thread's last error; returns st.
int reloc_internal_fail(int st, const char *msg);

}  // namespace reloc
