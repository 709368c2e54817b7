// api.cu -- the C ABI of reloc.h: context, map load, block selection,
// candidate grid, and the per-call orchestration of the kernels
// (K1 gather -> K2 project -> depth sort -> K3 tile counts + ranges ->
//  K4 tile emission -> K6 blend + NCC partials -> K7 NCC -> K8 argmax -> export).
//
// All stages run on the caller's stream with device-resident counts, so a
// call needs one host synchronisation at its end (to return scores and to
// check workspace capacity).  If a view produced more tile instances than
// the workspace holds, the call grows the workspace to the size the device
// reported and re-runs the call.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "blockindex.h"
#include "internal.cuh"
#include "reloc.h"

using namespace reloc;

// Pending injected faults (reloc_inject_faults; tests only), process-wide.
static std::atomic<int> g_faults[FAULT_KINDS];

bool reloc::take_fault(int kind)
{
    int n = g_faults[kind].load();
    while (n > 0)
        if (g_faults[kind].compare_exchange_weak(n, n - 1)) return true;
    return false;
}

namespace {

thread_local std::string g_err;

reloc_status fail(reloc_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return fail(RELOC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

#define CKS(call)                                                                                       \
    do {                                                                                                \
        reloc_status s_ = (call);                                                                       \
        if (s_ != RELOC_OK) return s_;                                                                  \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    reloc_status ensure(size_t n)
    {
        if (n <= bytes && p) return RELOC_OK;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (take_fault(FAULT_ALLOC)) return fail(RELOC_ENOMEM, "device allocation failed (injected)");
        size_t want = n < 256 ? 256 : n;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(RELOC_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", want, cudaGetErrorString(e));
        }
        bytes = want;
        return RELOC_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T *as() const { return (T *)p; }
};

struct PinBuf {
    void *p = nullptr;
    size_t bytes = 0;
    reloc_status ensure(size_t n)
    {
        if (n <= bytes && p) return RELOC_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMallocHost(&p, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(RELOC_ENOMEM, "cudaMallocHost(%zu) failed: %s", n, cudaGetErrorString(e));
        }
        bytes = n;
        return RELOC_OK;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
    }
};

}  // namespace

struct reloc_ctx {
    reloc_config cfg{};
    int device = 0;
    // map
    int64_t n = 0;
    int sh_degree = 0;
    int precision = 0;
    DevBuf mean, attr;
    std::vector<int64_t> order;
    BlockIndex blocks;
    // workspace (sized for the largest sub-batch of a call)
    DevBuf gidx, tables, rec, rect, dkey, k1a, v1a, k1b, v1b, hist1, chunk_sums, dtot;
    DevBuf srect, bhist, inst, ranges, partials, qpart, qstats;
    // per-call results (all views / queries of the call)
    DevBuf nvis, ninst, scores, degen, best, best_score, view_sel, flags;
    DevBuf bqueue;                       // the blend's work counter and heavy-tile list
    DevBuf hq, hrgb, hdepth;
    DevBuf pnp_X, pnp_out;
    DevBuf gbuf, gcoef, gpart, gpose;    // NCC pose gradients
    // map training: render and dL/dC scratch, loss, parameter gradients, Adam moments
    DevBuf trgb, tgimg, tabc, tloss, tgrad, adam_m, adam_v;
    DevBuf tdep, talp, twarp, tjac, tgw, tgda, trel;     // re-projection loss
    int64_t adam_t = 0;
    PinBuf pin;
    double inst_ratio = 3.0;        // instance capacity per (view, subset Gaussian), learned
    // batch options
    int use_graph = 1;
    int64_t mem_budget = (int64_t)16 << 30;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // last call (debug export covers its first sub-batch)
    int last_V = 0;
    int64_t last_S = 0;
    CamParams last_cam{};
    bool last_valid = false;
    std::vector<int64_t> last_ninst, last_io_off, last_vd_off;
    reloc_counts counts{};
    // learned candidate proposal
    ProposalNet *prop = nullptr;
    int prop_enabled = 0, prop_k = 8;
    float prop_margin = 0.f;
    DevBuf prop_in, prop_seed, prop_logits, prop_idx, prop_mrg, prop_loss;
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev;    // (RELOC_STAGE_COUNT + 1) per sub-batch
    double stage_ms[RELOC_STAGE_COUNT] = {};
    int64_t stage_calls[RELOC_STAGE_COUNT] = {};
};

// ============================================================ small pieces ==

int reloc::reloc_internal_fail(int st, const char *msg) { return fail(st, "%s", msg); }

static const char *kVersion = "gs-reloc-gb300 0.1 (sm_103a)";

extern "C" const char *reloc_version(void) { return kVersion; }
extern "C" const char *reloc_last_error(void) { return g_err.c_str(); }

extern "C" void reloc_default_config(reloc_config *cfg)
{
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->near_plane = 0.2f;
    cfg->fov_clamp = 1.3f;
    cfg->eps2d = 0.3f;
    cfg->alpha_min = 1.0f / 255.0f;
    cfg->alpha_max = 0.99f;
    cfg->t_min = 1e-4f;
    cfg->cut = 3.0f;
    cfg->det_fp64 = 1e-6f;
    cfg->block_size = 20.0;
    cfg->inst_capacity = 0;
    cfg->blend_rpl = 1;
    cfg->ncc_gray = 0;
}

static bool tile_ok(int w, int h)
{
    auto p2 = [](int x) { return x == 8 || x == 16 || x == 32; };
    return p2(w) && p2(h) && w * h <= 512;
}

static reloc_status check_config(const reloc_config &c)
{
    if (!tile_ok(c.tile_w, c.tile_h)) return fail(RELOC_EINVAL, "tile %dx%d not supported", c.tile_w, c.tile_h);
    if (!(c.near_plane > 0) || !(c.fov_clamp > 0) || !(c.eps2d >= 0) || !(c.alpha_min > 0) ||
        !(c.alpha_max > c.alpha_min) || !(c.alpha_max <= 1) || !(c.t_min > 0) || !(c.t_min < 1) || !(c.cut > 0) ||
        !(c.det_fp64 >= 0) || !(c.block_size > 0) || c.inst_capacity < 0 || c.blend_rpl < 1 || c.blend_rpl > 2 ||
        c.ncc_gray < 0 || c.ncc_gray > 1)
        return fail(RELOC_EINVAL, "invalid constant in reloc_config");
    return RELOC_OK;
}

extern "C" reloc_status reloc_create(const reloc_config *cfg, int device, reloc_ctx **out)
{
    if (!out) return fail(RELOC_EINVAL, "out is NULL");
    *out = nullptr;
    reloc_config c;
    if (cfg) c = *cfg; else reloc_default_config(&c);
    CKS(check_config(c));
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(RELOC_ECUDA, "device %d not present (%d devices)", device, ndev);
    CK(cudaSetDevice(device));
    reloc_ctx *ctx = new (std::nothrow) reloc_ctx();
    if (!ctx) return fail(RELOC_ENOMEM, "host allocation failed");
    ctx->cfg = c;
    ctx->device = device;
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        reloc_destroy(ctx);
        return fail(RELOC_ECUDA, "stream/event creation failed");
    }
    if (configure_tile_kernels() != cudaSuccess) {
        cudaGetLastError();
        reloc_destroy(ctx);
        return fail(RELOC_ECUDA, "kernel attribute setup failed");
    }
    *out = ctx;
    return RELOC_OK;
}

extern "C" reloc_status reloc_destroy(reloc_ctx *ctx)
{
    if (!ctx) return RELOC_OK;
    cudaSetDevice(ctx->device);
    DevBuf *bufs[] = {&ctx->mean, &ctx->attr, &ctx->gidx, &ctx->tables, &ctx->rec, &ctx->rect,
                      &ctx->dkey, &ctx->k1a, &ctx->v1a, &ctx->k1b, &ctx->v1b, &ctx->hist1, &ctx->chunk_sums,
                      &ctx->srect, &ctx->bhist, &ctx->inst, &ctx->ranges, &ctx->partials,
                      &ctx->qpart, &ctx->qstats, &ctx->nvis, &ctx->ninst, &ctx->scores, &ctx->degen,
                      &ctx->best, &ctx->best_score, &ctx->view_sel, &ctx->flags, &ctx->bqueue, &ctx->hq, &ctx->hrgb,
                      &ctx->hdepth, &ctx->prop_in, &ctx->prop_seed, &ctx->prop_logits, &ctx->prop_idx,
                      &ctx->prop_mrg, &ctx->prop_loss, &ctx->pnp_X, &ctx->pnp_out, &ctx->gbuf, &ctx->gcoef,
                      &ctx->gpart, &ctx->gpose};
    for (DevBuf *b : bufs) b->release();
    if (ctx->prop) proposal_destroy(ctx->prop);
    ctx->pin.release();
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return RELOC_OK;
}

// ================================================================ map load ==

template <typename T> static T cvt(float x);
template <> float cvt<float>(float x) { return x; }
template <> __half cvt<__half>(float x) { return __float2half_rn(x); }
template <> __nv_bfloat16 cvt<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <typename T>
static void pack_attr(const reloc_gaussians_host *g, const std::vector<int64_t> &order, int64_t n, int deg,
                      std::vector<T> &out)
{
    const int K = (deg + 1) * (deg + 1);
    const int nc = attr_components(deg);
    out.resize((size_t)nc * n);
    for (int64_t p = 0; p < n; ++p) {
        const int64_t i = order[p];
        for (int k = 0; k < 3; ++k) out[(size_t)(ATTR_SCALE + k) * n + p] = cvt<T>(g->scale[3 * i + k]);
        for (int k = 0; k < 4; ++k) out[(size_t)(ATTR_QUAT + k) * n + p] = cvt<T>(g->quat[4 * i + k]);
        out[(size_t)ATTR_OPAC * n + p] = cvt<T>(g->opacity[i]);
        for (int k = 0; k < 3 * K; ++k) out[(size_t)(ATTR_SH + k) * n + p] = cvt<T>(g->sh[(size_t)3 * K * i + k]);
    }
}

extern "C" reloc_status reloc_load_map(reloc_ctx *ctx, const reloc_gaussians_host *g, int64_t n, int sh_degree,
                                       int precision)
{
    if (!ctx || !g) return fail(RELOC_EINVAL, "NULL argument");
    if (n < 1 || n > (int64_t)UINT32_MAX) return fail(RELOC_EINVAL, "map size %lld out of range", (long long)n);
    if (sh_degree < 0 || sh_degree > 3) return fail(RELOC_EINVAL, "sh_degree %d not in 0..3", sh_degree);
    if (precision < RELOC_FP32 || precision > RELOC_BF16) return fail(RELOC_EINVAL, "precision %d unknown", precision);
    if (!g->mean || !g->scale || !g->quat || !g->opacity || !g->sh) return fail(RELOC_EINVAL, "NULL attribute array");
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(g->mean[3 * i]) || !std::isfinite(g->mean[3 * i + 1]) || !std::isfinite(g->mean[3 * i + 2]))
            return fail(RELOC_ENUMERIC, "non-finite mean at %lld", (long long)i);
    CK(cudaSetDevice(ctx->device));
    ctx->n = 0;
    ctx->last_valid = false;
    std::vector<int64_t> order;
    ctx->blocks.build(g->mean, n, ctx->cfg.block_size, order);
    std::vector<float> m((size_t)3 * n);
    for (int64_t p = 0; p < n; ++p)
        for (int k = 0; k < 3; ++k) m[(size_t)k * n + p] = g->mean[3 * order[p] + k];
    CKS(ctx->mean.ensure(sizeof(float) * 3 * n));
    CK(cudaMemcpy(ctx->mean.p, m.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice));
    const size_t nc = attr_components(sh_degree);
    if (precision == RELOC_FP32) {
        std::vector<float> a;
        pack_attr(g, order, n, sh_degree, a);
        CKS(ctx->attr.ensure(sizeof(float) * nc * n));
        CK(cudaMemcpy(ctx->attr.p, a.data(), sizeof(float) * nc * n, cudaMemcpyHostToDevice));
    } else if (precision == RELOC_FP16) {
        std::vector<__half> a;
        pack_attr(g, order, n, sh_degree, a);
        CKS(ctx->attr.ensure(sizeof(__half) * nc * n));
        CK(cudaMemcpy(ctx->attr.p, a.data(), sizeof(__half) * nc * n, cudaMemcpyHostToDevice));
    } else {
        std::vector<__nv_bfloat16> a;
        pack_attr(g, order, n, sh_degree, a);
        CKS(ctx->attr.ensure(sizeof(__nv_bfloat16) * nc * n));
        CK(cudaMemcpy(ctx->attr.p, a.data(), sizeof(__nv_bfloat16) * nc * n, cudaMemcpyHostToDevice));
    }
    ctx->order.swap(order);
    ctx->n = n;
    ctx->sh_degree = sh_degree;
    ctx->precision = precision;
    ctx->adam_t = 0;
    return RELOC_OK;
}

extern "C" reloc_status reloc_map_order(reloc_ctx *ctx, int64_t *order_out)
{
    if (!ctx || !order_out) return fail(RELOC_EINVAL, "NULL argument");
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    memcpy(order_out, ctx->order.data(), sizeof(int64_t) * ctx->n);
    return RELOC_OK;
}

static void merge_runs(const BlockIndex &B, const std::vector<int> &ids, std::vector<reloc_range> &runs)
{
    runs.clear();
    for (int b : ids) {
        if (!runs.empty() && runs.back().end == B.begin[b]) runs.back().end = B.end[b];
        else runs.push_back({B.begin[b], B.end[b]});
    }
}

extern "C" reloc_status reloc_select_block(reloc_ctx *ctx, double x, double y, double radius, reloc_range *ranges_out,
                                           int max_ranges, int *n_ranges, int64_t *n_gauss, int *n_blocks)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(radius) || radius < 0)
        return fail(RELOC_ENUMERIC, "non-finite position or radius");
    std::vector<int> ids;
    ctx->blocks.range(x, y, radius, ids);
    std::vector<reloc_range> runs;
    merge_runs(ctx->blocks, ids, runs);
    int64_t cnt = 0;
    for (auto &r : runs) cnt += r.end - r.begin;
    if (n_ranges) *n_ranges = (int)runs.size();
    if (n_gauss) *n_gauss = cnt;
    if (n_blocks) *n_blocks = (int)ids.size();
    if ((int)runs.size() > max_ranges)
        return fail(RELOC_EINVAL, "%d runs needed, max_ranges = %d", (int)runs.size(), max_ranges);
    if (!runs.empty()) {
        if (!ranges_out) return fail(RELOC_EINVAL, "ranges_out is NULL");
        memcpy(ranges_out, runs.data(), sizeof(reloc_range) * runs.size());
    }
    return RELOC_OK;
}

// =========================================================== candidate grid ==
// Offsets in the world ground plane and a yaw about world z through the camera
// centre (Sec. III-C.1 brute-force grid; Sec. IV-A: 2 m x 10 deg).
static void grid_poses(const double *W, const reloc_grid &g, std::vector<double> &out)
{
    const int V = g.nx * g.ny * g.nyaw;
    out.assign((size_t)16 * V, 0.0);
    double C[3];
    for (int i = 0; i < 3; ++i) C[i] = -(W[i] * W[3] + W[4 + i] * W[7] + W[8 + i] * W[11]);
    for (int iyaw = 0; iyaw < g.nyaw; ++iyaw)
        for (int iy = 0; iy < g.ny; ++iy)
            for (int ix = 0; ix < g.nx; ++ix) {
                const int k = ix + g.nx * (iy + g.ny * iyaw);
                const double dx = (ix - 0.5 * (g.nx - 1)) * g.step_xy;
                const double dy = (iy - 0.5 * (g.ny - 1)) * g.step_xy;
                const double psi = (iyaw - 0.5 * (g.nyaw - 1)) * g.step_yaw_deg * (M_PI / 180.0);
                const double cs = std::cos(psi), sn = std::sin(psi);
                double *o = out.data() + 16 * k;
                // new rotation: each camera axis (row of R) rotated about world z by psi
                for (int r = 0; r < 3; ++r) {
                    const double a = W[4 * r], b = W[4 * r + 1], c = W[4 * r + 2];
                    o[4 * r] = cs * a - sn * b;
                    o[4 * r + 1] = sn * a + cs * b;
                    o[4 * r + 2] = c;
                }
                const double Cn[3] = {C[0] + dx, C[1] + dy, C[2]};
                for (int r = 0; r < 3; ++r)
                    o[4 * r + 3] = -(o[4 * r] * Cn[0] + o[4 * r + 1] * Cn[1] + o[4 * r + 2] * Cn[2]);
                o[15] = 1.0;
            }
}

// ============================================================= the pipeline ==

static reloc_status make_cam(const reloc_ctx *ctx, const reloc_camera *cam, CamParams &cp)
{
    if (!cam) return fail(RELOC_EINVAL, "camera is NULL");
    if (cam->width < 1 || cam->height < 1 || cam->width > 16383 || cam->height > 16383)
        return fail(RELOC_EINVAL, "image size %dx%d out of range", cam->width, cam->height);
    if (!std::isfinite(cam->fx) || !std::isfinite(cam->fy) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy) ||
        !(cam->fx > 0) || !(cam->fy > 0))
        return fail(RELOC_ENUMERIC, "invalid intrinsics");
    const reloc_config &c = ctx->cfg;
    cp.width = cam->width;
    cp.height = cam->height;
    cp.tile_w = c.tile_w;
    cp.tile_h = c.tile_h;
    cp.ntx = (cam->width + c.tile_w - 1) / c.tile_w;
    cp.nty = (cam->height + c.tile_h - 1) / c.tile_h;
    cp.n_tiles = cp.ntx * cp.nty;
    int tb = 0;
    while ((1 << tb) < cp.n_tiles) ++tb;
    cp.tile_bits = tb;
    cp.bin_chunk = BIN_CHUNK_MIN * (int)std::max<int64_t>(1, ceil_div(cp.n_tiles, BIN_TILES_PER_CHUNK_STEP));
    cp.fx = (float)cam->fx;
    cp.fy = (float)cam->fy;
    cp.cx = (float)cam->cx;
    cp.cy = (float)cam->cy;
    cp.limx = (float)(c.fov_clamp * (0.5 * cam->width) / cam->fx);
    cp.limy = (float)(c.fov_clamp * (0.5 * cam->height) / cam->fy);
    cp.near_plane = c.near_plane;
    cp.eps2d = c.eps2d;
    cp.cut = c.cut;
    cp.det_fp64 = c.det_fp64;
    cp.alpha_min = c.alpha_min;
    cp.alpha_max = c.alpha_max;
    cp.t_min = c.t_min;
    cp.blend_rpl = c.blend_rpl;
    cp.ncc_gray = c.ncc_gray;
    return RELOC_OK;
}

static reloc_status make_view(const double *W, int v, ViewParams &P)
{
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(W[k])) return fail(RELOC_ENUMERIC, "non-finite pose %d", v);
    memset(&P, 0, sizeof P);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) P.R[3 * r + c] = (float)W[4 * r + c];
    for (int i = 0; i < 3; ++i) {
        const double C = -(W[i] * W[3] + W[4 + i] * W[7] + W[8 + i] * W[11]);
        P.c_hi[i] = (float)C;
        P.c_lo[i] = (float)(C - (double)P.c_hi[i]);
    }
    return RELOC_OK;
}

// One query of a call: its Gaussian subset (block-ordered runs) and views.
struct QuerySpec {
    std::vector<reloc_range> runs;
    int64_t S = 0;
    int V = 0;
    std::vector<double> poses;      // V x 16, world-to-camera
    const float *img = nullptr;     // device query image ([3][H][W]) or null
    int n_blocks = 0;
    int gx = 0, gy = 0, gyaw = 0;    // candidate grid shape (localize calls)
    std::vector<double> coarse;      // coarse pose (localize calls)
    std::vector<int> grid_index;     // view -> grid cell when a subset is rendered
};

// What a call produces.  Per-view device outputs use the call's global view
// index, per-query outputs its query index.
struct CallOut {
    float *rgb = nullptr, *depth = nullptr, *alpha = nullptr;     // [V][...]
    bool score = false;                                         // NCC (needs query images)
    bool argmax = false;                                        // per query argmax
    float *brgb = nullptr, *bdepth = nullptr, *balpha = nullptr; // winners [Q][...]
    double *grad = nullptr;                                     // NCC pose gradients [V][6] (device)
    const float *target = nullptr;  // training: target images [V][3][H][W] (device)
    double l1_scale = 0.0;          // training: weight of sum |C - I| in the loss
    double ssim_scale = 0.0;        // training: weight of sum (1 - SSIM) in the loss
    int n_views_total = 0;          // training: views of the call (pairs are (t, t+1))
    double rp_l1_scale = 0.0, rp_ssim_scale = 0.0;   // training: re-projection loss weights
    float rp_alpha_min = 0.5f;
    const float *rel = nullptr;     // training: relative poses [n_views_total][12] (device)
    float *tgrad = nullptr;         // training: dL/dparameters [14][n] (device, accumulated)
    std::vector<double> scores;
    std::vector<int> degen, best;
    std::vector<double> best_score;
};

// A run of consecutive queries whose workspace fits the memory budget.
struct SubBatch {
    int q0 = 0, q1 = 0, v0 = 0, v1 = 0;
    int64_t S_tot = 0, VS = 0, VI = 0;
    int c1 = 0, cb = 0, pblk = 0, n_runs = 0;
    std::vector<int32_t> view_q, c1_base, cb_base, q_view, q_pblk;
    std::vector<int64_t> vd_off, io_off, q_gsub, run_begin, run_off;
    std::vector<ViewParams> views;
    std::vector<const float *> q_img;
    size_t tab_off = 0, tab_bytes = 0;
    Layout L{};
    const int64_t *d_run_begin = nullptr, *d_run_off = nullptr;
    const ViewParams *d_views = nullptr;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int64_t inst_cap(const reloc_ctx *ctx, int64_t S, int64_t override_cap)
{
    int64_t c = override_cap > 0 ? override_cap
                                 : (ctx->cfg.inst_capacity > 0 ? ctx->cfg.inst_capacity
                                                               : (int64_t)(ctx->inst_ratio * (double)S) + 4096);
    return ceil_div(c, SORT_CHUNK) * SORT_CHUNK;
}

// Workspace bytes of one query: per view, the per-Gaussian arrays (records,
// rectangle, tile count, depth key, two key/value radix buffers, depth-ordered
// rectangle, radix histograms), the instance list, ranges, NCC partials per
// warp block and the per-chunk tile counts; plus the gathered subset.
static int64_t query_bytes(int64_t S, int V, int64_t cap, const CamParams &cp)
{
    const int64_t per_view = S * 89 + cap * 4 + (int64_t)cp.n_tiles * 8 + (int64_t)blend_units(cp) * 24 +
                             4 * (int64_t)cp.n_tiles * ceil_div(S, cp.bin_chunk) + 1024;
    return (int64_t)V * per_view + S * 4 + 4096;
}

// Split the call into sub-batches and build each one's host tables.
static void plan_batches(const reloc_ctx *ctx, const std::vector<QuerySpec> &qs, const std::vector<int64_t> &caps,
                         const CamParams &cp, std::vector<SubBatch> &out)
{
    out.clear();
    const int Q = (int)qs.size();
    int q = 0, vglob = 0;
    while (q < Q) {
        SubBatch sb;
        sb.q0 = q;
        sb.v0 = vglob;
        int64_t bytes = 0, units = 0;
        while (q < Q) {
            const int64_t b = query_bytes(qs[q].S, qs[q].V, caps[q], cp);
            const int64_t un = (int64_t)qs[q].V * blend_units(cp);
            if (q > sb.q0 && (bytes + b > ctx->mem_budget || units + un > BLEND_MAX_UNITS)) break;
            bytes += b;
            units += un;
            vglob += qs[q].V;
            ++q;
        }
        sb.q1 = q;
        sb.v1 = vglob;
        const int nq = sb.q1 - sb.q0, nv = sb.v1 - sb.v0;
        sb.vd_off.assign(nv + 1, 0);
        sb.io_off.assign(nv + 1, 0);
        sb.c1_base.assign(nv + 1, 0);
        sb.cb_base.assign(nv + 1, 0);
        sb.view_q.assign(nv, 0);
        sb.q_gsub.assign(nq + 1, 0);
        sb.q_view.assign(nq + 1, 0);
        sb.q_pblk.assign(nq + 1, 0);
        sb.q_img.assign(nq, nullptr);
        sb.views.resize(nv);
        sb.run_off.push_back(0);
        int v = 0;
        for (int k = 0; k < nq; ++k) {
            const QuerySpec &Qs = qs[sb.q0 + k];
            const int64_t cap = inst_cap(ctx, Qs.S, caps[sb.q0 + k]);
            sb.q_gsub[k + 1] = sb.q_gsub[k] + Qs.S;
            sb.q_view[k + 1] = sb.q_view[k] + Qs.V;
            sb.q_pblk[k + 1] = sb.q_pblk[k] + (int32_t)ceil_div(Qs.S, PROJ_THREADS);
            sb.q_img[k] = Qs.img;
            for (auto &r : Qs.runs) {
                sb.run_begin.push_back(r.begin);
                sb.run_off.push_back(sb.run_off.back() + (r.end - r.begin));
            }
            for (int j = 0; j < Qs.V; ++j, ++v) {
                sb.view_q[v] = k;
                make_view(Qs.poses.data() + 16 * j, v, sb.views[v]);
                sb.vd_off[v + 1] = sb.vd_off[v] + Qs.S;
                sb.io_off[v + 1] = sb.io_off[v] + cap;
                sb.c1_base[v + 1] = sb.c1_base[v] + (int32_t)ceil_div(Qs.S, SORT_CHUNK);
                sb.cb_base[v + 1] = sb.cb_base[v] + (int32_t)ceil_div(Qs.S, cp.bin_chunk);
            }
        }
        sb.S_tot = sb.q_gsub[nq];
        sb.VS = sb.vd_off[nv];
        sb.VI = sb.io_off[nv];
        sb.c1 = sb.c1_base[nv];
        sb.cb = sb.cb_base[nv];
        sb.pblk = sb.q_pblk[nq];
        sb.n_runs = (int)sb.run_begin.size();
        if (sb.run_begin.empty()) sb.run_begin.push_back(0);
        // table bytes (each array 256-aligned)
        size_t t = 0;
        t += align256(4 * (size_t)nv) + 2 * align256(8 * (size_t)(nv + 1)) + 2 * align256(4 * (size_t)(nv + 1));
        t += align256(8 * (size_t)(nq + 1)) + 2 * align256(4 * (size_t)(nq + 1)) + align256(8 * (size_t)nq);
        t += align256(8 * sb.run_begin.size()) + align256(8 * sb.run_off.size()) + align256(sizeof(ViewParams) * nv);
        sb.tab_bytes = t;
        out.push_back(std::move(sb));
    }
}

// Write a sub-batch's tables into host staging at base + sb.tab_off and set
// its device pointers relative to dev.
static void stage_tables(SubBatch &sb, char *host, char *dev)
{
    size_t o = sb.tab_off;
    auto put = [&](const void *src, size_t bytes) -> char * {
        memcpy(host + o, src, bytes);
        char *d = dev + o;
        o += align256(bytes);
        return d;
    };
    const int nq = sb.q1 - sb.q0, nv = sb.v1 - sb.v0;
    sb.L.Q = nq;
    sb.L.V = nv;
    sb.L.view_q = (const int32_t *)put(sb.view_q.data(), 4 * (size_t)nv);
    sb.L.vd_off = (const int64_t *)put(sb.vd_off.data(), 8 * (size_t)(nv + 1));
    sb.L.io_off = (const int64_t *)put(sb.io_off.data(), 8 * (size_t)(nv + 1));
    sb.L.c1_base = (const int32_t *)put(sb.c1_base.data(), 4 * (size_t)(nv + 1));
    sb.L.cb_base = (const int32_t *)put(sb.cb_base.data(), 4 * (size_t)(nv + 1));
    sb.L.q_gsub = (const int64_t *)put(sb.q_gsub.data(), 8 * (size_t)(nq + 1));
    sb.L.q_view = (const int32_t *)put(sb.q_view.data(), 4 * (size_t)(nq + 1));
    sb.L.q_pblk = (const int32_t *)put(sb.q_pblk.data(), 4 * (size_t)(nq + 1));
    sb.L.q_img = (const float *const *)put(sb.q_img.data(), 8 * (size_t)nq);
    sb.d_run_begin = (const int64_t *)put(sb.run_begin.data(), 8 * sb.run_begin.size());
    sb.d_run_off = (const int64_t *)put(sb.run_off.data(), 8 * sb.run_off.size());
    sb.d_views = (const ViewParams *)put(sb.views.data(), sizeof(ViewParams) * (size_t)nv);
}

static void stage_mark(reloc_ctx *ctx, int sbi, int s, cudaStream_t st, bool capturing)
{
    if (ctx->prof && !capturing) cudaEventRecord(ctx->ev[(size_t)sbi * (RELOC_STAGE_COUNT + 1) + s], st);
}

// Enqueue every kernel of one sub-batch on st.  Returns the launch count.
static reloc_status enqueue_subbatch(reloc_ctx *ctx, SubBatch &sb, int sbi, const CamParams &cp, const CallOut &o,
                                     cudaStream_t st, bool capturing, int &launches)
{
    const int64_t HW = (int64_t)cp.width * cp.height;
    const Layout &L = sb.L;
    int *d_overflow = ctx->flags.as<int>();
    uint32_t *nvis = ctx->nvis.as<uint32_t>() + sb.v0;
    uint32_t *ninst = ctx->ninst.as<uint32_t>() + sb.v0;

    stage_mark(ctx, sbi, RELOC_STAGE_CULL, st, capturing);
    if (sb.S_tot > 0) {
        CK(launch_gather_subset(sb.d_run_begin, sb.d_run_off, sb.n_runs, sb.S_tot, ctx->gidx.as<uint32_t>(), st));
        launches += 1;
    }
    stage_mark(ctx, sbi, RELOC_STAGE_PROJECT, st, capturing);
    if (sb.pblk > 0) {
        CK(launch_project(ctx->mean.as<float>(), ctx->mean.as<float>() + ctx->n, ctx->mean.as<float>() + 2 * ctx->n,
                          ctx->attr.p, ctx->precision, ctx->sh_degree, ctx->n, ctx->gidx.as<uint32_t>(), L, sb.pblk,
                          sb.d_views, cp, ctx->rec.as<float4>(), ctx->rect.as<uint2>(), ctx->dkey.as<uint32_t>(), st));
        launches += 1;
    }
    stage_mark(ctx, sbi, RELOC_STAGE_DEPTH_SORT, st, capturing);
    CK(cudaMemsetAsync(nvis, 0, 4 * (size_t)L.V, st));
    CK(cudaMemsetAsync(ninst, 0, 4 * (size_t)L.V, st));
    if (sb.c1 > 0) {
        RadixPass p{};
        p.seg_off = L.vd_off;
        p.chunk_base = L.c1_base;
        p.n_seg = L.V;
        p.total_chunks = sb.c1;
        p.hist = ctx->hist1.as<uint32_t>();
        p.mask = 0xFF;
        // per (view, digit) totals, one slice per pass
        uint32_t *dtot = ctx->dtot.as<uint32_t>();
        CK(cudaMemsetAsync(dtot, 0, 16 * (size_t)RADIX * L.V, st));
        p.dtot = dtot;
        uint32_t *ka = ctx->k1a.as<uint32_t>(), *va = ctx->v1a.as<uint32_t>();
        uint32_t *kb = ctx->k1b.as<uint32_t>(), *vb = ctx->v1b.as<uint32_t>();
        // pass 0: dense (view, Gaussian) arrays; culled pairs are dropped
        p.keys_in = ctx->dkey.as<uint32_t>();
        p.vals_in = nullptr;
        p.drop_culled = 1;
        p.len = nullptr;
        p.keys_out = ka;
        p.vals_out = va;
        p.len_out = nvis;
        p.shift = 0;
        CK(launch_radix_pass(p, st));
        launches += 3;
        p.drop_culled = 0;
        p.len = nvis;
        p.len_out = nullptr;
        for (int pass = 1; pass < 4; ++pass) {
            p.shift = 8 * pass;
            p.dtot = dtot + (size_t)pass * RADIX * L.V;
            p.keys_in = (pass & 1) ? ka : kb;
            p.vals_in = (pass & 1) ? va : vb;
            p.keys_out = (pass & 1) ? kb : ka;
            p.vals_out = (pass & 1) ? vb : va;
            CK(launch_radix_pass(p, st));
            launches += 3;
        }
    }
    stage_mark(ctx, sbi, RELOC_STAGE_TILE_COUNT, st, capturing);
    CK(launch_tile_count(ctx->v1b.as<uint32_t>(), nvis, ctx->rect.as<uint2>(), L, cp, sb.cb, ctx->srect.as<uint2>(),
                         ctx->bhist.as<uint32_t>(), ctx->ranges.as<int2>(), ninst, d_overflow, st));
    launches += sb.cb > 0 ? 3 : 2;
    stage_mark(ctx, sbi, RELOC_STAGE_TILE_EMIT, st, capturing);
    if (sb.cb > 0) {
        CK(launch_tile_emit(ctx->v1b.as<uint32_t>(), ctx->srect.as<uint2>(), nvis, ninst, ctx->bhist.as<uint32_t>(),
                            ctx->ranges.as<int2>(), L, cp, sb.cb, ctx->inst.as<uint32_t>(), st));
        launches += 1;
    }
    const uint32_t *fgauss = ctx->inst.as<uint32_t>();
    stage_mark(ctx, sbi, RELOC_STAGE_BLEND, st, capturing);
    if (o.score) {
        CK(launch_query_stats(L, HW, cp.ncc_gray != 0, ctx->qpart.as<double>(), ctx->qstats.as<double>(), st));
        launches += 2;
    }
    float *rgb_out = o.target ? ctx->trgb.as<float>() : (o.rgb ? o.rgb + (int64_t)sb.v0 * 3 * HW : nullptr);
    const bool rp = o.target && o.rel;
    float *dep_out = rp ? ctx->tdep.as<float>() : (o.depth ? o.depth + (int64_t)sb.v0 * HW : nullptr);
    float *alp_out = rp ? ctx->talp.as<float>() : (o.alpha ? o.alpha + (int64_t)sb.v0 * HW : nullptr);
    CK(launch_blend(ctx->rec.as<float4>(), L, fgauss, ctx->ranges.as<int2>(), cp,
                    o.score ? ctx->partials.as<double>() : nullptr, rgb_out, dep_out, alp_out,
                    nullptr, 0, d_overflow, ctx->bqueue.as<int>(), st));
    launches += blend_launches(L.V);
    stage_mark(ctx, sbi, RELOC_STAGE_SCORE, st, capturing);
    if (o.target) {
        // map training: the image loss and dL/dC, then back through the blend and the projection
        CK(launch_photo_l1(ctx->trgb.as<float>(), o.target + (int64_t)sb.v0 * 3 * HW, (int64_t)L.V * 3 * HW,
                           o.l1_scale, ctx->tgimg.as<float>(), false, ctx->tloss.as<double>(), st));
        if (o.ssim_scale > 0) {
            CK(launch_ssim(ctx->trgb.as<float>(), o.target + (int64_t)sb.v0 * 3 * HW, 3 * L.V, cp.height, cp.width,
                           o.ssim_scale, ctx->tabc.as<float>(), ctx->tgimg.as<float>(), ctx->tloss.as<double>(), st));
            launches += 2;
        }
        if (rp) {
            // re-projection loss over the pairs (t, t+1) whose first view is in this sub-batch
            const int np = std::max(0, std::min(L.V, o.n_views_total - 1 - sb.v0));
            const float *tg = o.target + (int64_t)sb.v0 * 3 * HW;
            CK(cudaMemsetAsync(ctx->tgda.p, 0, 8 * (size_t)L.V * HW, st));
            if (np > 0) {
                CK(launch_reproj_warp(ctx->tdep.as<float>(), ctx->talp.as<float>(), tg, o.rel + 12 * (int64_t)sb.v0,
                                      np, cp, o.rp_alpha_min, ctx->twarp.as<float>(), ctx->tjac.as<float>(), st));
                CK(launch_photo_l1(ctx->twarp.as<float>(), tg, (int64_t)np * 3 * HW, o.rp_l1_scale,
                                   ctx->tgw.as<float>(), false, ctx->tloss.as<double>(), st));
                launches += 2;
                if (o.rp_ssim_scale > 0) {
                    CK(launch_ssim(ctx->twarp.as<float>(), tg, 3 * np, cp.height, cp.width, o.rp_ssim_scale,
                                   ctx->tabc.as<float>(), ctx->tgw.as<float>(), ctx->tloss.as<double>(), st));
                    launches += 2;
                }
                CK(launch_reproj_back(ctx->tgw.as<float>(), ctx->tjac.as<float>(), ctx->tdep.as<float>(),
                                      ctx->talp.as<float>(), np, HW, o.rp_alpha_min, ctx->tgda.as<float>(), st));
                launches += 1;
            }
        }
        CK(cudaMemsetAsync(ctx->gbuf.p, 0, 40 * (size_t)sb.VS, st));
        CK(launch_blend_grad(ctx->rec.as<float4>(), L, fgauss, ctx->ranges.as<int2>(), cp, nullptr,
                             ctx->tgimg.as<float>(), rp ? ctx->tgda.as<float>() : nullptr, ctx->trgb.as<float>(),
                             rp ? ctx->tdep.as<float>() : nullptr, rp ? ctx->talp.as<float>() : nullptr,
                             ctx->gbuf.as<float>(), d_overflow, st));
        CK(launch_param_chain(ctx->mean.as<float>(), ctx->mean.as<float>() + ctx->n,
                              ctx->mean.as<float>() + 2 * ctx->n, ctx->attr.as<float>(), ctx->n,
                              ctx->gidx.as<uint32_t>(), L, sb.pblk, sb.d_views, cp, ctx->gbuf.as<float>(), o.tgrad,
                              st));
        launches += 3;
    }
    if (o.score) {
        CK(launch_ncc_finalize(ctx->partials.as<double>(), ctx->qstats.as<double>(), L, blend_units(cp),
                               cp.ncc_gray ? HW : 3 * HW,
                               ctx->scores.as<double>() + sb.v0, ctx->degen.as<int>() + sb.v0,
                               o.grad ? ctx->gcoef.as<double>() : nullptr, st));
        launches += 1;
        if (o.grad) {
            CK(cudaMemsetAsync(ctx->gbuf.p, 0, 20 * (size_t)sb.VS, st));
            CK(launch_blend_grad(ctx->rec.as<float4>(), L, fgauss, ctx->ranges.as<int2>(), cp,
                                 ctx->gcoef.as<double>(), nullptr, nullptr, nullptr, nullptr, nullptr,
                                 ctx->gbuf.as<float>(), d_overflow, st));
            CK(launch_pose_chain(ctx->mean.as<float>(), ctx->mean.as<float>() + ctx->n,
                                 ctx->mean.as<float>() + 2 * ctx->n, ctx->attr.p, ctx->precision, ctx->n,
                                 ctx->gidx.as<uint32_t>(), L, sb.pblk, sb.d_views, cp, ctx->gbuf.as<float>(),
                                 ctx->gpart.as<double>(), o.grad + 6 * (int64_t)sb.v0, st));
            launches += 3;
        }
        if (o.argmax) {
            int *vsel = ctx->view_sel.as<int>() + sb.q0;
            CK(launch_argmax(ctx->scores.as<double>() + sb.v0, L, ctx->best.as<int>() + sb.q0,
                             ctx->best_score.as<double>() + sb.q0, vsel, st));
            launches += 1;
            if (o.brgb || o.bdepth || o.balpha) {
                const int nq = sb.q1 - sb.q0;
                CK(launch_blend(ctx->rec.as<float4>(), L, fgauss, ctx->ranges.as<int2>(), cp, nullptr,
                                o.brgb ? o.brgb + (int64_t)sb.q0 * 3 * HW : nullptr,
                                o.bdepth ? o.bdepth + (int64_t)sb.q0 * HW : nullptr,
                                o.balpha ? o.balpha + (int64_t)sb.q0 * HW : nullptr, vsel, nq, d_overflow,
                                ctx->bqueue.as<int>(), st));
                launches += blend_launches(nq);
            }
        }
    }
    stage_mark(ctx, sbi, RELOC_STAGE_COUNT, st, capturing);
    return RELOC_OK;
}

static reloc_status run_batch(reloc_ctx *ctx, std::vector<QuerySpec> &qs, const reloc_camera *cam, cudaStream_t ust,
                              CallOut &o, bool allow_graph)
{
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    const int Q = (int)qs.size();
    if (Q < 1) return fail(RELOC_EINVAL, "no queries");
    int64_t Vtot = 0;
    for (auto &q : qs) {
        if (q.V < 1 || q.V > 4096) return fail(RELOC_EINVAL, "a query has %d views (1..4096 allowed)", q.V);
        if (o.score && !q.img) return fail(RELOC_EINVAL, "query image is NULL");
        Vtot += q.V;
        q.S = 0;
        for (auto &r : q.runs) {
            if (r.begin < 0 || r.end < r.begin || r.end > ctx->n)
                return fail(RELOC_EINVAL, "range [%lld, %lld) outside the map", (long long)r.begin, (long long)r.end);
            q.S += r.end - r.begin;
        }
        if (q.S > (int64_t)UINT32_MAX / 4) return fail(RELOC_EINVAL, "subset too large");
        for (int j = 0; j < q.V; ++j)
            for (int k = 0; k < 16; ++k)
                if (!std::isfinite(q.poses[16 * j + k])) return fail(RELOC_ENUMERIC, "non-finite pose %d", j);
    }
    if (Vtot > (1 << 24)) return fail(RELOC_EINVAL, "too many views in one call");
    CamParams cp;
    CKS(make_cam(ctx, cam, cp));
    for (auto &q : qs)
        if ((int64_t)q.V * blend_units(cp) > BLEND_MAX_UNITS)
            return fail(RELOC_EINVAL, "a query's %d views of %d x %d pixels exceed %lld blend units", q.V, cp.width,
                        cp.height, (long long)BLEND_MAX_UNITS);
    CK(cudaSetDevice(ctx->device));
    ctx->last_valid = false;
    const int64_t HW = (int64_t)cp.width * cp.height;
    const bool graph = allow_graph && ctx->use_graph;

    std::vector<int64_t> caps(Q, 0);
    std::vector<SubBatch> sbs;
    int retries = 0, launches = 0;
    for (;;) {
        plan_batches(ctx, qs, caps, cp, sbs);
        // ---- workspace: the largest sub-batch --------------------------------
        int64_t S_tot = 1, VS = 1, VI = 1, c1 = 1, cb = 1, V = 1, Qm = 1;
        size_t tab = 0;
        for (auto &sb : sbs) {
            S_tot = std::max(S_tot, sb.S_tot);
            VS = std::max(VS, sb.VS);
            VI = std::max(VI, sb.VI);
            c1 = std::max<int64_t>(c1, sb.c1);
            cb = std::max<int64_t>(cb, sb.cb);
            V = std::max<int64_t>(V, sb.v1 - sb.v0);
            Qm = std::max<int64_t>(Qm, sb.q1 - sb.q0);
            sb.tab_off = tab;
            tab += sb.tab_bytes;
        }
        CKS(ctx->gidx.ensure(4 * (size_t)S_tot));
        CKS(ctx->rec.ensure(48 * (size_t)VS));
        CKS(ctx->rect.ensure(8 * (size_t)VS));
        CKS(ctx->dkey.ensure(4 * (size_t)VS));
        CKS(ctx->k1a.ensure(4 * (size_t)VS));
        CKS(ctx->v1a.ensure(4 * (size_t)VS));
        CKS(ctx->k1b.ensure(4 * (size_t)VS));
        CKS(ctx->v1b.ensure(4 * (size_t)VS));
        CKS(ctx->hist1.ensure(4 * (size_t)RADIX * c1));
        CKS(ctx->dtot.ensure(16 * (size_t)RADIX * V));
        CKS(ctx->srect.ensure(8 * (size_t)VS));
        CKS(ctx->bhist.ensure(4 * (size_t)cp.n_tiles * cb));
        CKS(ctx->inst.ensure(4 * (size_t)VI));
        CKS(ctx->ranges.ensure(sizeof(int2) * (size_t)V * cp.n_tiles));
        CKS(ctx->partials.ensure(24 * (size_t)V * blend_units(cp)));
        if (o.target) {
            CKS(ctx->trgb.ensure(12 * (size_t)V * HW));
            CKS(ctx->tgimg.ensure(12 * (size_t)V * HW));
            CKS(ctx->gbuf.ensure(40 * (size_t)VS));
            if (o.ssim_scale > 0 || o.rp_ssim_scale > 0) CKS(ctx->tabc.ensure(36 * (size_t)V * HW));
            if (o.rel) {
                CKS(ctx->tdep.ensure(4 * (size_t)V * HW));
                CKS(ctx->talp.ensure(4 * (size_t)V * HW));
                CKS(ctx->twarp.ensure(12 * (size_t)V * HW));
                CKS(ctx->tjac.ensure(12 * (size_t)V * HW));
                CKS(ctx->tgw.ensure(12 * (size_t)V * HW));
                CKS(ctx->tgda.ensure(8 * (size_t)V * HW));
            }
        }
        if (o.grad) {
            int64_t pb = 1;
            for (auto &sb : sbs) pb = std::max<int64_t>(pb, (int64_t)sb.pblk * (sb.v1 - sb.v0));
            CKS(ctx->gbuf.ensure(20 * (size_t)VS));
            CKS(ctx->gcoef.ensure(32 * (size_t)V));
            CKS(ctx->gpart.ensure(48 * (size_t)pb));
        }
        CKS(ctx->qpart.ensure(16 * 152 * (size_t)Qm));
        CKS(ctx->qstats.ensure(16 * (size_t)Qm));
        CKS(ctx->nvis.ensure(4 * (size_t)Vtot));
        CKS(ctx->ninst.ensure(4 * (size_t)Vtot));
        CKS(ctx->scores.ensure(8 * (size_t)Vtot));
        CKS(ctx->degen.ensure(4 * (size_t)Vtot));
        CKS(ctx->best.ensure(4 * (size_t)Q));
        CKS(ctx->best_score.ensure(8 * (size_t)Q));
        CKS(ctx->view_sel.ensure(4 * (size_t)Q));
        CKS(ctx->flags.ensure(64));
        CKS(ctx->bqueue.ensure(4 * (size_t)blend_queue_ints(cp, std::max<int64_t>(V, Qm))));
        CKS(ctx->tables.ensure(tab));
        // pinned staging: tables, then readback
        const size_t rb_off = align256(tab);
        const size_t rb_bytes = 64 + (4 + 4 + 8 + 4) * (size_t)Vtot + (4 + 8) * (size_t)Q;
        CKS(ctx->pin.ensure(rb_off + rb_bytes));
        char *pin = (char *)ctx->pin.p;
        for (auto &sb : sbs) stage_tables(sb, pin, ctx->tables.as<char>());
        // readback block: doubles first (8-byte aligned), then 32-bit words
        int *h_overflow = (int *)(pin + rb_off);
        double *h_scores = (double *)(pin + rb_off + 64);
        double *h_bscore = h_scores + Vtot;
        uint32_t *h_nvis = (uint32_t *)(h_bscore + Q);
        uint32_t *h_ninst = h_nvis + Vtot;
        int *h_degen = (int *)(h_ninst + Vtot);
        int *h_best = h_degen + Vtot;
        if (ctx->prof) {
            const size_t need = sbs.size() * (RELOC_STAGE_COUNT + 1);
            while (ctx->ev.size() < need) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                ctx->ev.push_back(e);
            }
        }
        // ---- enqueue -------------------------------------------------------------
        cudaStream_t st = ust;
        if (graph) {
            CK(cudaEventRecord(ctx->ev_in, ust));
            CK(cudaStreamWaitEvent(ctx->cap_stream, ctx->ev_in, 0));
            st = ctx->cap_stream;
        }
        CK(cudaMemcpyAsync(ctx->tables.p, pin, tab, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(ctx->flags.p, 0, 64, st));
        if (o.target) {     // every attempt starts from zero (an overflow retry re-runs the call)
            CK(cudaMemsetAsync(ctx->tloss.p, 0, 8, st));
            CK(cudaMemsetAsync(o.tgrad, 0, sizeof(float) * 14 * (size_t)ctx->n, st));
        }
        launches = 0;
        if (graph) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            reloc_status rs = RELOC_OK;
            for (size_t k = 0; k < sbs.size() && rs == RELOC_OK; ++k)
                rs = enqueue_subbatch(ctx, sbs[k], (int)k, cp, o, st, true, launches);
            cudaError_t ce_ = cudaStreamEndCapture(st, &g);
            if (rs != RELOC_OK) {
                if (g) cudaGraphDestroy(g);
                return rs;
            }
            if (ce_ != cudaSuccess) return fail(RELOC_ECUDA, "graph capture: %s", cudaGetErrorString(ce_));
            ce_ = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (ce_ != cudaSuccess) return fail(RELOC_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce_));
            ce_ = cudaGraphLaunch(ge, st);
            cudaGraphExecDestroy(ge);
            if (ce_ != cudaSuccess) return fail(RELOC_ECUDA, "graph launch: %s", cudaGetErrorString(ce_));
        } else {
            for (size_t k = 0; k < sbs.size(); ++k) CKS(enqueue_subbatch(ctx, sbs[k], (int)k, cp, o, st, false, launches));
        }
        // ---- readback --------------------------------------------------------------
        CK(cudaMemcpyAsync(h_overflow, ctx->flags.p, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_nvis, ctx->nvis.p, 4 * (size_t)Vtot, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_ninst, ctx->ninst.p, 4 * (size_t)Vtot, cudaMemcpyDeviceToHost, st));
        if (o.score) {
            CK(cudaMemcpyAsync(h_scores, ctx->scores.p, 8 * (size_t)Vtot, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(h_degen, ctx->degen.p, 4 * (size_t)Vtot, cudaMemcpyDeviceToHost, st));
            if (o.argmax) {
                CK(cudaMemcpyAsync(h_best, ctx->best.p, 4 * (size_t)Q, cudaMemcpyDeviceToHost, st));
                CK(cudaMemcpyAsync(h_bscore, ctx->best_score.p, 8 * (size_t)Q, cudaMemcpyDeviceToHost, st));
            }
        }
        if (graph) {
            CK(cudaEventRecord(ctx->ev_out, st));
            CK(cudaStreamWaitEvent(ust, ctx->ev_out, 0));
        }
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        if (ctx->prof && !graph) {
            for (size_t k = 0; k < sbs.size(); ++k)
                for (int s = 0; s < RELOC_STAGE_COUNT; ++s) {
                    float ms = 0;
                    const size_t e0 = k * (RELOC_STAGE_COUNT + 1) + s;
                    if (cudaEventElapsedTime(&ms, ctx->ev[e0], ctx->ev[e0 + 1]) == cudaSuccess) {
                        ctx->stage_ms[s] += ms;
                        if (k == 0) ctx->stage_calls[s] += 1;
                    } else {
                        cudaGetLastError();
                    }
                }
        }
        if (!*h_overflow) {
            // learn the instance ratio for later calls (capacity = ratio * S + slack)
            int64_t vglob = 0;
            for (int q = 0; q < Q; ++q)
                for (int j = 0; j < qs[q].V; ++j, ++vglob)
                    if (qs[q].S > 0)
                        ctx->inst_ratio = std::max(ctx->inst_ratio, 1.15 * (double)h_ninst[vglob] / (double)qs[q].S);
            // results
            ctx->counts = reloc_counts{};
            ctx->counts.n_views = Vtot;
            for (auto &q : qs) ctx->counts.n_gauss += q.S;
            ctx->last_ninst.assign(h_ninst, h_ninst + (sbs[0].v1 - sbs[0].v0));
            for (int64_t v = 0; v < Vtot; ++v) {
                ctx->counts.n_visible += h_nvis[v];
                ctx->counts.n_instances += h_ninst[v];
            }
            ctx->counts.inst_stride = sbs[0].io_off.size() > 1 ? sbs[0].io_off[1] - sbs[0].io_off[0] : 0;
            ctx->counts.retries = retries;
            ctx->counts.kernel_launches = launches;
            if (o.score) {
                o.scores.assign(h_scores, h_scores + Vtot);
                o.degen.assign(h_degen, h_degen + Vtot);
                if (o.argmax) {
                    o.best.assign(h_best, h_best + Q);
                    o.best_score.assign(h_bscore, h_bscore + Q);
                }
            }
            break;
        }
        // ---- overflow: grow the capacity of every query that did not fit -------
        if (++retries > 3) return fail(RELOC_EOVERFLOW, "tile-instance workspace still too small after %d grows", retries);
        int64_t vglob = 0;
        for (int q = 0; q < Q; ++q) {
            int64_t need = 0;
            for (int j = 0; j < qs[q].V; ++j, ++vglob) need = std::max<int64_t>(need, h_ninst[vglob]);
            const int64_t cap = inst_cap(ctx, qs[q].S, caps[q]);
            if (need > cap) caps[q] = need + need / 8 + 4096;
            if (qs[q].S > 0) ctx->inst_ratio = std::max(ctx->inst_ratio, 1.15 * (double)need / (double)qs[q].S);
        }
    }
    // ---- debug export state (first sub-batch) ----------------------------------
    ctx->last_V = sbs[0].v1 - sbs[0].v0;
    ctx->last_S = qs[0].S;
    ctx->last_cam = cp;
    ctx->last_io_off = sbs[0].io_off;
    ctx->last_vd_off = sbs[0].vd_off;
    ctx->last_valid = sbs.size() == 1 && sbs[0].q1 - sbs[0].q0 == 1;
    return RELOC_OK;
}

// ============================================================== entry points ==

static reloc_status one_query(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges, const double *poses, int V,
                              QuerySpec &q)
{
    if (V < 1 || V > 4096) return fail(RELOC_EINVAL, "n_views %d not in 1..4096", V);
    if (!poses) return fail(RELOC_EINVAL, "poses is NULL");
    if (n_ranges < 0 || (n_ranges > 0 && !ranges)) return fail(RELOC_EINVAL, "bad ranges");
    q.runs.assign(ranges, ranges + n_ranges);
    q.V = V;
    q.poses.assign(poses, poses + 16 * (size_t)V);
    return RELOC_OK;
}

extern "C" reloc_status reloc_render(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges, const double *poses,
                                     int n_views, const reloc_camera *cam, float *rgb_dev, float *depth_dev,
                                     float *alpha_dev, void *stream)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    std::vector<QuerySpec> qs(1);
    CKS(one_query(ctx, ranges, n_ranges, poses, n_views, qs[0]));
    CallOut o;
    o.rgb = rgb_dev;
    o.depth = depth_dev;
    o.alpha = alpha_dev;
    return run_batch(ctx, qs, cam, (cudaStream_t)stream, o, false);
}

extern "C" reloc_status reloc_score(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges, const double *poses,
                                    int n_views, const reloc_camera *cam, const float *query_dev, double *scores_host,
                                    int *degenerate_host, void *stream)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    if (!query_dev || !scores_host) return fail(RELOC_EINVAL, "query_dev and scores_host are required");
    std::vector<QuerySpec> qs(1);
    CKS(one_query(ctx, ranges, n_ranges, poses, n_views, qs[0]));
    qs[0].img = query_dev;
    CallOut o;
    o.score = true;
    CKS(run_batch(ctx, qs, cam, (cudaStream_t)stream, o, false));
    memcpy(scores_host, o.scores.data(), sizeof(double) * n_views);
    if (degenerate_host) memcpy(degenerate_host, o.degen.data(), sizeof(int) * n_views);
    return RELOC_OK;
}

// Block selection + candidate grid of one localization query.
static reloc_status make_localize_query(reloc_ctx *ctx, const float *query_dev, const double *coarse_pose,
                                        double radius, const reloc_grid *grid, QuerySpec &q)
{
    if (!query_dev || !coarse_pose || !grid) return fail(RELOC_EINVAL, "NULL argument");
    if (grid->nx < 1 || grid->ny < 1 || grid->nyaw < 1 || (int64_t)grid->nx * grid->ny * grid->nyaw > 4096)
        return fail(RELOC_EINVAL, "grid %dx%dx%d not in 1..4096 candidates", grid->nx, grid->ny, grid->nyaw);
    if (!std::isfinite(grid->step_xy) || !std::isfinite(grid->step_yaw_deg) || !std::isfinite(radius))
        return fail(RELOC_ENUMERIC, "non-finite grid step or radius");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(coarse_pose[k])) return fail(RELOC_ENUMERIC, "non-finite coarse pose");
    const double *W = coarse_pose;
    const double Cx = -(W[0] * W[3] + W[4] * W[7] + W[8] * W[11]);
    const double Cy = -(W[1] * W[3] + W[5] * W[7] + W[9] * W[11]);
    std::vector<int> ids;
    ctx->blocks.range(Cx, Cy, radius, ids);
    merge_runs(ctx->blocks, ids, q.runs);
    q.n_blocks = (int)ids.size();
    grid_poses(coarse_pose, *grid, q.poses);
    q.V = grid->nx * grid->ny * grid->nyaw;
    q.img = query_dev;
    q.gx = grid->nx;
    q.gy = grid->ny;
    q.gyaw = grid->nyaw;
    q.coarse.assign(coarse_pose, coarse_pose + 16);
    return RELOC_OK;
}

static void fill_result(const QuerySpec &q, const CallOut &o, int qi, int v0, reloc_result *out)
{
    memset(out, 0, sizeof *out);
    const int b = o.best[qi];
    out->best_index = q.grid_index.empty() ? b : q.grid_index[b];
    out->n_candidates = q.grid_index.empty() ? q.V : q.gx * q.gy * q.gyaw;
    out->n_scored = q.V;
    out->best_score = o.best_score[qi];
    if (b >= 0 && b < q.V) {
        memcpy(out->best_pose, q.poses.data() + 16 * b, sizeof(double) * 16);
        out->degenerate = o.degen[v0 + b];
    }
    out->n_gauss = q.S;
    out->n_blocks = q.n_blocks;
}

// Learned proposal: for every query with a 4 x 4 x 4 grid, render the coarse
// view, rank the cells with the CNN and keep the top-k (ascending cell order,
// so ties still resolve to the lowest cell), or all cells when p1 - p2 < margin.
static reloc_status apply_proposal(reloc_ctx *ctx, std::vector<QuerySpec> &qs, const reloc_camera *cam,
                                   cudaStream_t st)
{
    std::vector<int> sel;
    for (int i = 0; i < (int)qs.size(); ++i)
        if (qs[i].gx == 4 && qs[i].gy == 4 && qs[i].gyaw == 4) sel.push_back(i);
    if (sel.empty()) return RELOC_OK;
    const int H = cam->height, W = cam->width;
    if (H % PROPOSAL_H || W % PROPOSAL_W || H / PROPOSAL_H != W / PROPOSAL_W)
        return fail(RELOC_EINVAL, "the proposal needs H = 47 f and W = 176 f (got %dx%d)", W, H);
    const int Ql = (int)sel.size();
    const int64_t HW = (int64_t)H * W;
    CKS(ctx->prop_seed.ensure(12 * (size_t)HW * Ql));
    CKS(ctx->prop_in.ensure(2 * (size_t)PROPOSAL_H * PROPOSAL_W * 2 * Ql));
    CKS(ctx->prop_logits.ensure(4 * (size_t)PROPOSAL_CLASSES * Ql));
    CKS(ctx->prop_idx.ensure(4 * (size_t)32 * Ql));
    CKS(ctx->prop_mrg.ensure(4 * (size_t)Ql));
    // (a) coarse-pose renders
    std::vector<QuerySpec> seeds(Ql);
    for (int j = 0; j < Ql; ++j) {
        seeds[j].runs = qs[sel[j]].runs;
        seeds[j].V = 1;
        seeds[j].poses = qs[sel[j]].coarse;
    }
    CallOut ro;
    ro.rgb = ctx->prop_seed.as<float>();
    CKS(run_batch(ctx, seeds, cam, st, ro, false));
    // (b) inputs, (c) logits and top-k
    __nv_bfloat16 *in = ctx->prop_in.as<__nv_bfloat16>();
    for (int j = 0; j < Ql; ++j)
        CK(proposal_make_input(qs[sel[j]].img, ctx->prop_seed.as<float>() + (int64_t)j * 3 * HW, H, W,
                               in + (int64_t)j * PROPOSAL_H * PROPOSAL_W * 2, st));
    CK(proposal_forward(ctx->prop, in, Ql, ctx->prop_logits.as<float>(), st));
    CK(launch_topk(ctx->prop_logits.as<float>(), Ql, PROPOSAL_CLASSES, ctx->prop_k, ctx->prop_idx.as<int32_t>(),
                   ctx->prop_mrg.as<float>(), st));
    std::vector<int32_t> idx((size_t)Ql * ctx->prop_k);
    std::vector<float> mrg(Ql);
    int status = 0;
    CK(cudaMemcpyAsync(idx.data(), ctx->prop_idx.p, 4 * idx.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(mrg.data(), ctx->prop_mrg.p, 4 * (size_t)Ql, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&status, proposal_status(ctx->prop), 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (status) return fail(RELOC_ETIMEOUT, "proposal: a tensor-core wait gave up");
    // (d) the candidate subsets
    for (int j = 0; j < Ql; ++j) {
        QuerySpec &q = qs[sel[j]];
        if (mrg[j] < ctx->prop_margin) continue;       // low confidence: full sweep
        std::vector<int> cells(idx.begin() + (size_t)j * ctx->prop_k, idx.begin() + (size_t)(j + 1) * ctx->prop_k);
        std::sort(cells.begin(), cells.end());
        std::vector<double> poses;
        for (int c : cells) poses.insert(poses.end(), q.poses.begin() + 16 * c, q.poses.begin() + 16 * (c + 1));
        q.poses.swap(poses);
        q.V = (int)cells.size();
        q.grid_index = cells;
    }
    return RELOC_OK;
}

// scores of a query in grid order (NaN for cells the proposal did not render)
static void grid_scores(const QuerySpec &q, const double *sc, double *out)
{
    if (q.grid_index.empty()) {
        memcpy(out, sc, sizeof(double) * q.V);
        return;
    }
    const int n = q.gx * q.gy * q.gyaw;
    for (int c = 0; c < n; ++c) out[c] = std::nan("");
    for (int j = 0; j < q.V; ++j) out[q.grid_index[j]] = sc[j];
}

static reloc_status localize_impl(reloc_ctx *ctx, const float *query_dev, const double *coarse_pose, double radius,
                                  const reloc_grid *grid, const reloc_camera *cam, reloc_result *out,
                                  double *scores_host, float *brgb, float *bdepth, float *balpha, cudaStream_t st)
{
    if (!ctx || !cam || !out) return fail(RELOC_EINVAL, "NULL argument");
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    std::vector<QuerySpec> qs(1);
    CKS(make_localize_query(ctx, query_dev, coarse_pose, radius, grid, qs[0]));
    if (ctx->prop_enabled && ctx->prop) CKS(apply_proposal(ctx, qs, cam, st));
    CallOut o;
    o.score = true;
    o.argmax = true;
    o.brgb = brgb;
    o.bdepth = bdepth;
    o.balpha = balpha;
    CKS(run_batch(ctx, qs, cam, st, o, false));
    fill_result(qs[0], o, 0, 0, out);
    if (scores_host) grid_scores(qs[0], o.scores.data(), scores_host);
    return RELOC_OK;
}

extern "C" reloc_status reloc_localize(reloc_ctx *ctx, const float *query_dev, const double *coarse_pose, double radius,
                                       const reloc_grid *grid, const reloc_camera *cam, reloc_result *out,
                                       double *scores_host, float *best_rgb_dev, float *best_depth_dev,
                                       float *best_alpha_dev, void *stream)
{
    return localize_impl(ctx, query_dev, coarse_pose, radius, grid, cam, out, scores_host, best_rgb_dev,
                         best_depth_dev, best_alpha_dev, (cudaStream_t)stream);
}

// ================================================ random search (Sec. IV-A) ==
// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): a Weyl sequence with step 0x9E3779B97F4A7C15
// passed through the variant-13 64-bit finaliser.
static uint64_t splitmix64_next(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" reloc_status reloc_localize_random(reloc_ctx *ctx, const float *query_dev, const double *coarse_pose,
                                              double radius, const reloc_grid *grid, const reloc_camera *cam,
                                              const reloc_search *search, reloc_result *out, double *scores_host,
                                              float *best_rgb_dev, float *best_depth_dev, float *best_alpha_dev,
                                              void *stream)
{
    if (!ctx || !cam || !out || !search || !grid || !query_dev || !coarse_pose) return fail(RELOC_EINVAL, "NULL argument");
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    const int64_t n_cells = (int64_t)grid->nx * grid->ny * grid->nyaw;
    if (grid->nx < 1 || grid->ny < 1 || grid->nyaw < 1 || n_cells > (1 << 20))
        return fail(RELOC_EINVAL, "grid %dx%dx%d not in 1..2^20 cells", grid->nx, grid->ny, grid->nyaw);
    if (search->batch < 1 || search->batch > 4096) return fail(RELOC_EINVAL, "batch %d not in 1..4096", search->batch);
    if (!std::isfinite(grid->step_xy) || !std::isfinite(grid->step_yaw_deg) || !std::isfinite(radius))
        return fail(RELOC_ENUMERIC, "non-finite grid step or radius");
    if (std::isnan(search->ncc_stop)) return fail(RELOC_ENUMERIC, "ncc_stop is NaN");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(coarse_pose[k])) return fail(RELOC_ENUMERIC, "non-finite coarse pose");
    // the visit: an explicit order, or the first ceil(fraction n) cells of a seeded shuffle
    std::vector<int> order;
    if (search->order) {
        if (search->n_order < 1 || search->n_order > n_cells)
            return fail(RELOC_EINVAL, "n_order %d not in 1..%lld", search->n_order, (long long)n_cells);
        std::vector<char> seen((size_t)n_cells, 0);
        for (int i = 0; i < search->n_order; ++i) {
            const int c = search->order[i];
            if (c < 0 || c >= n_cells || seen[c]) return fail(RELOC_EINVAL, "order[%d] = %d invalid or repeated", i, c);
            seen[c] = 1;
            order.push_back(c);
        }
    } else {
        if (!(search->fraction > 0.0 && search->fraction <= 1.0))
            return fail(RELOC_EINVAL, "fraction %g not in (0, 1]", search->fraction);
        std::vector<int> perm((size_t)n_cells);
        for (int64_t i = 0; i < n_cells; ++i) perm[i] = (int)i;
        uint64_t state = search->seed;
        for (int64_t i = n_cells - 1; i > 0; --i) {
            const uint64_t j = splitmix64_next(state) % (uint64_t)(i + 1);
            std::swap(perm[i], perm[j]);
        }
        const int64_t m = std::min<int64_t>(n_cells, (int64_t)std::ceil(search->fraction * (double)n_cells));
        order.assign(perm.begin(), perm.begin() + m);
    }
    // blocks around the coarse pose, every cell's pose
    QuerySpec base;
    {
        const double *W = coarse_pose;
        const double Cx = -(W[0] * W[3] + W[4] * W[7] + W[8] * W[11]);
        const double Cy = -(W[1] * W[3] + W[5] * W[7] + W[9] * W[11]);
        std::vector<int> ids;
        ctx->blocks.range(Cx, Cy, radius, ids);
        merge_runs(ctx->blocks, ids, base.runs);
        base.n_blocks = (int)ids.size();
    }
    std::vector<double> cell_pose;
    grid_poses(coarse_pose, *grid, cell_pose);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> sc_all;
    if (scores_host) sc_all.assign((size_t)n_cells, std::nan(""));
    int best = -1, best_degen = 0;
    double best_sc = -INFINITY;
    int64_t visited = 0, S = 0;
    for (const reloc_range &r : base.runs) S += r.end - r.begin;
    bool stopped = false;
    for (size_t b0 = 0; b0 < order.size(); b0 += (size_t)search->batch) {
        const int nb = (int)std::min<size_t>((size_t)search->batch, order.size() - b0);
        std::vector<QuerySpec> qs(1);
        qs[0].runs = base.runs;
        qs[0].n_blocks = base.n_blocks;
        qs[0].V = nb;
        qs[0].img = query_dev;
        for (int j = 0; j < nb; ++j) {
            const double *p = cell_pose.data() + 16 * (size_t)order[b0 + j];
            qs[0].poses.insert(qs[0].poses.end(), p, p + 16);
        }
        CallOut o;
        o.score = true;
        CKS(run_batch(ctx, qs, cam, st, o, false));
        for (int j = 0; j < nb; ++j) {
            const int c = order[b0 + j];
            const double s_c = o.scores[j];
            if (scores_host) sc_all[c] = s_c;
            if (s_c > best_sc || (s_c == best_sc && c < best)) {
                best = c;
                best_sc = s_c;
                best_degen = o.degen[j];
            }
        }
        visited += nb;
        if (best_sc >= search->ncc_stop) {
            stopped = visited < (int64_t)order.size();
            break;
        }
    }
    if (best >= 0 && (best_rgb_dev || best_depth_dev || best_alpha_dev)) {
        std::vector<QuerySpec> wq(1);
        wq[0].runs = base.runs;
        wq[0].V = 1;
        wq[0].poses.assign(cell_pose.begin() + 16 * (size_t)best, cell_pose.begin() + 16 * (size_t)(best + 1));
        CallOut o;
        o.rgb = best_rgb_dev;
        o.depth = best_depth_dev;
        o.alpha = best_alpha_dev;
        CKS(run_batch(ctx, wq, cam, st, o, false));
    }
    memset(out, 0, sizeof *out);
    out->best_index = best;
    out->n_candidates = (int32_t)n_cells;
    out->best_score = best >= 0 ? best_sc : 0.0;
    if (best >= 0) memcpy(out->best_pose, cell_pose.data() + 16 * (size_t)best, sizeof(double) * 16);
    out->n_gauss = S;
    out->n_blocks = base.n_blocks;
    out->degenerate = best_degen;
    out->n_scored = (int32_t)visited;
    out->stopped_early = stopped ? 1 : 0;
    if (scores_host) memcpy(scores_host, sc_all.data(), sizeof(double) * (size_t)n_cells);
    return RELOC_OK;
}

extern "C" reloc_status reloc_localize_batch(reloc_ctx *ctx, const reloc_query *queries, int n_queries,
                                             const reloc_camera *cam, reloc_result *results, double *scores_host,
                                             float *best_rgb_dev, float *best_depth_dev, void *stream)
{
    if (!ctx || !queries || !cam || !results) return fail(RELOC_EINVAL, "NULL argument");
    if (n_queries < 1) return fail(RELOC_EINVAL, "n_queries %d < 1", n_queries);
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    std::vector<QuerySpec> qs(n_queries);
    for (int i = 0; i < n_queries; ++i)
        CKS(make_localize_query(ctx, queries[i].query_dev, queries[i].coarse_pose, queries[i].radius,
                                &queries[i].grid, qs[i]));
    if (ctx->prop_enabled && ctx->prop) CKS(apply_proposal(ctx, qs, cam, (cudaStream_t)stream));
    CallOut o;
    o.score = true;
    o.argmax = true;
    o.brgb = best_rgb_dev;
    o.bdepth = best_depth_dev;
    CKS(run_batch(ctx, qs, cam, (cudaStream_t)stream, o, true));
    int v0 = 0;
    int64_t g0 = 0;
    for (int i = 0; i < n_queries; ++i) {
        fill_result(qs[i], o, i, v0, &results[i]);
        if (scores_host) grid_scores(qs[i], o.scores.data() + v0, scores_host + g0);
        v0 += qs[i].V;
        g0 += qs[i].grid_index.empty() ? qs[i].V : qs[i].gx * qs[i].gy * qs[i].gyaw;
    }
    return RELOC_OK;
}

extern "C" reloc_status reloc_set_batch_options(reloc_ctx *ctx, const reloc_batch_options *opt)
{
    if (!ctx || !opt) return fail(RELOC_EINVAL, "NULL argument");
    if (opt->mem_budget < ((int64_t)64 << 20)) return fail(RELOC_EINVAL, "mem_budget below 64 MiB");
    ctx->use_graph = opt->use_graph != 0;
    ctx->mem_budget = opt->mem_budget;
    return RELOC_OK;
}

// ================================================================= proposal ==

extern "C" reloc_status reloc_proposal_init(reloc_ctx *ctx, uint64_t seed)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    CK(cudaSetDevice(ctx->device));
    if (ctx->prop) proposal_destroy(ctx->prop);
    ctx->prop = nullptr;
    cudaError_t e = cudaSuccess;
    ctx->prop = proposal_create(seed, &e);
    if (!ctx->prop) return fail(e == cudaErrorMemoryAllocation ? RELOC_ENOMEM : RELOC_ECUDA, "proposal init: %s",
                                cudaGetErrorString(e));
    return RELOC_OK;
}

extern "C" reloc_status reloc_proposal_get(reloc_ctx *ctx, int which, float *flat_host)
{
    if (!ctx || !flat_host || (which != 0 && which != 1)) return fail(RELOC_EINVAL, "bad argument");
    if (!ctx->prop) return fail(RELOC_EINVAL, "no proposal network (reloc_proposal_init)");
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    CK(proposal_get(ctx->prop, which, flat_host));
    return RELOC_OK;
}

extern "C" reloc_status reloc_proposal_set_params(reloc_ctx *ctx, const float *flat_host)
{
    if (!ctx || !flat_host) return fail(RELOC_EINVAL, "bad argument");
    if (!ctx->prop) return fail(RELOC_EINVAL, "no proposal network (reloc_proposal_init)");
    CK(cudaSetDevice(ctx->device));
    CK(proposal_set(ctx->prop, flat_host));
    return RELOC_OK;
}

extern "C" reloc_status reloc_proposal_make_input(reloc_ctx *ctx, const float *query_dev, const float *coarse_rgb_dev,
                                                  const reloc_camera *cam, uint16_t *input_dev, void *stream)
{
    if (!ctx || !query_dev || !coarse_rgb_dev || !cam || !input_dev) return fail(RELOC_EINVAL, "NULL argument");
    if (cam->height % PROPOSAL_H || cam->width % PROPOSAL_W || cam->height / PROPOSAL_H != cam->width / PROPOSAL_W)
        return fail(RELOC_EINVAL, "the proposal needs H = 47 f and W = 176 f");
    CK(cudaSetDevice(ctx->device));
    CK(proposal_make_input(query_dev, coarse_rgb_dev, cam->height, cam->width, (__nv_bfloat16 *)input_dev,
                           (cudaStream_t)stream));
    return RELOC_OK;
}

extern "C" reloc_status reloc_proposal_forward(reloc_ctx *ctx, const uint16_t *inputs_dev, int batch,
                                               float *logits_dev, void *stream)
{
    if (!ctx || !inputs_dev || !logits_dev || batch < 1) return fail(RELOC_EINVAL, "bad argument");
    if (!ctx->prop) return fail(RELOC_EINVAL, "no proposal network (reloc_proposal_init)");
    CK(cudaSetDevice(ctx->device));
    CK(proposal_forward(ctx->prop, (const __nv_bfloat16 *)inputs_dev, batch, logits_dev, (cudaStream_t)stream));
    return RELOC_OK;
}

extern "C" reloc_status reloc_proposal_train_step(reloc_ctx *ctx, const uint16_t *inputs_dev, const int32_t *labels_dev,
                                                  int batch, float lr, int update, float *loss_host, void *stream)
{
    if (!ctx || !inputs_dev || !labels_dev || batch < 64 || batch % 64) return fail(RELOC_EINVAL, "bad argument");
    if (!ctx->prop) return fail(RELOC_EINVAL, "no proposal network (reloc_proposal_init)");
    if (!(lr >= 0) || !std::isfinite(lr)) return fail(RELOC_ENUMERIC, "bad learning rate");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CKS(ctx->prop_loss.ensure(4 * (size_t)batch));
    CK(proposal_train_step(ctx->prop, (const __nv_bfloat16 *)inputs_dev, labels_dev, batch, lr, update != 0,
                           ctx->prop_loss.as<float>(), st));
    std::vector<float> rows(batch);
    int status = 0;
    CK(cudaMemcpyAsync(rows.data(), ctx->prop_loss.p, 4 * (size_t)batch, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&status, proposal_status(ctx->prop), 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (status) return fail(RELOC_ETIMEOUT, "proposal: a tensor-core wait gave up");
    double sum = 0;
    for (float r : rows) sum += r;
    if (loss_host) *loss_host = (float)(sum / batch);
    return RELOC_OK;
}

extern "C" reloc_status reloc_gemm_bf16(reloc_ctx *ctx, const uint16_t *A_dev, const uint16_t *B_dev,
                                        const float *bias_dev, float *C_dev, int M, int N, int K, int relu, int split_k,
                                        void *stream)
{
    if (!ctx || !A_dev || !B_dev || !C_dev) return fail(RELOC_EINVAL, "NULL argument");
    if (M < 1 || N < 1 || K < 64 || K % 64 || split_k < 1 || (K / split_k) % 64 || K % split_k)
        return fail(RELOC_EINVAL, "gemm: K must be a multiple of 64 and of 64 * split_k");
    if (((uintptr_t)A_dev & 15) || ((uintptr_t)B_dev & 15)) return fail(RELOC_EINVAL, "gemm: A, B need 16-byte alignment");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CKS(ctx->flags.ensure(64));
    DevBuf &part = ctx->chunk_sums;     // scratch for split-K partials
    if (split_k > 1) CKS(part.ensure(4 * (size_t)split_k * M * N));
    CK(cudaMemsetAsync(ctx->flags.p, 0, 4, st));
    CK(launch_gemm_bf16((const __nv_bfloat16 *)A_dev, (const __nv_bfloat16 *)B_dev, bias_dev, C_dev, nullptr, M, N, K,
                        K, K, N, relu, split_k, part.as<float>(), ctx->flags.as<int>(), st));
    int status = 0;
    CK(cudaMemcpyAsync(&status, ctx->flags.p, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (status) return fail(RELOC_ETIMEOUT, "gemm: a tensor-core wait gave up");
    return RELOC_OK;
}

extern "C" reloc_status reloc_set_proposal(reloc_ctx *ctx, int enabled, int top_k, float margin)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    if (enabled && !ctx->prop) return fail(RELOC_EINVAL, "no proposal network (reloc_proposal_init)");
    if (top_k < 2 || top_k > 32 || !std::isfinite(margin)) return fail(RELOC_EINVAL, "top_k in 2..32, finite margin");
    ctx->prop_enabled = enabled != 0;
    ctx->prop_k = top_k;
    ctx->prop_margin = margin;
    return RELOC_OK;
}

// ================================================================ autotuner ==
// Tile shape and records-per-step of the blend are chosen by timing a sample
// batch with every supported configuration; the winner is kept in a text
// table (one line per workload key) so later processes reuse it.

static const int kTuneConfigs[][3] = {{16, 16, 1}, {16, 16, 2}, {8, 8, 1}, {8, 8, 2},  {32, 8, 1}, {32, 8, 2},
                                      {16, 8, 1},  {16, 8, 2},  {8, 16, 1}, {8, 16, 2}, {32, 16, 1}, {32, 16, 2}};

static std::string tune_key(const reloc_ctx *ctx, const reloc_camera *cam, double avg_v, double avg_s)
{
    char buf[160];
    snprintf(buf, sizeof buf, "%d %d %d %d %d %d", cam->width, cam->height, ctx->sh_degree, ctx->precision,
             (int)std::lround(std::log2(std::max(1.0, avg_v))), (int)std::lround(std::log2(std::max(1.0, avg_s))));
    return buf;
}

extern "C" reloc_status reloc_autotune(reloc_ctx *ctx, const reloc_query *sample, int n_sample,
                                       const reloc_camera *cam, const char *table_path, int force,
                                       reloc_tune_result *out, void *stream)
{
    if (!ctx || !sample || !cam || !out || n_sample < 1) return fail(RELOC_EINVAL, "NULL argument or empty sample");
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    memset(out, 0, sizeof *out);
    double sv = 0, ss = 0;
    for (int i = 0; i < n_sample; ++i) {
        QuerySpec q;
        CKS(make_localize_query(ctx, sample[i].query_dev, sample[i].coarse_pose, sample[i].radius, &sample[i].grid, q));
        for (auto &r : q.runs) ss += (double)(r.end - r.begin);
        sv += q.V;
    }
    const std::string key = tune_key(ctx, cam, sv / n_sample, ss / n_sample);
    if (table_path && !force) {
        FILE *f = fopen(table_path, "r");
        if (f) {
            char line[256];
            while (fgets(line, sizeof line, f)) {
                int w, h, deg, prec, vb, sb, tw, th, rpl;
                double ms;
                if (sscanf(line, "%d %d %d %d %d %d %d %d %d %lf", &w, &h, &deg, &prec, &vb, &sb, &tw, &th, &rpl, &ms) == 10) {
                    char k2[160];
                    snprintf(k2, sizeof k2, "%d %d %d %d %d %d", w, h, deg, prec, vb, sb);
                    if (key == k2 && tile_ok(tw, th) && (rpl == 1 || rpl == 2)) {
                        ctx->cfg.tile_w = tw;
                        ctx->cfg.tile_h = th;
                        ctx->cfg.blend_rpl = rpl;
                        out->tile_w = tw;
                        out->tile_h = th;
                        out->blend_rpl = rpl;
                        out->ms_per_query = ms;
                        out->from_table = 1;
                    }
                }
            }
            fclose(f);
            if (out->from_table) return RELOC_OK;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<reloc_result> res(n_sample);
    const reloc_config saved = ctx->cfg;
    double best_ms = 1e300;
    int best = -1;
    for (int c = 0; c < (int)(sizeof kTuneConfigs / sizeof kTuneConfigs[0]); ++c) {
        ctx->cfg.tile_w = kTuneConfigs[c][0];
        ctx->cfg.tile_h = kTuneConfigs[c][1];
        ctx->cfg.blend_rpl = kTuneConfigs[c][2];
        reloc_status s = reloc_localize_batch(ctx, sample, n_sample, cam, res.data(), nullptr, nullptr, nullptr, stream);
        if (s != RELOC_OK) continue;          // e.g. a shape this camera cannot tile: skip it
        cudaEventRecord(e0, st);
        s = reloc_localize_batch(ctx, sample, n_sample, cam, res.data(), nullptr, nullptr, nullptr, stream);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        if (s == RELOC_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            out->n_tried++;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cudaGetLastError();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->cfg = saved;
    if (best < 0) return fail(RELOC_ECUDA, "autotune: no configuration ran");
    ctx->cfg.tile_w = kTuneConfigs[best][0];
    ctx->cfg.tile_h = kTuneConfigs[best][1];
    ctx->cfg.blend_rpl = kTuneConfigs[best][2];
    out->tile_w = ctx->cfg.tile_w;
    out->tile_h = ctx->cfg.tile_h;
    out->blend_rpl = ctx->cfg.blend_rpl;
    out->ms_per_query = best_ms / n_sample;
    if (table_path) {
        FILE *f = fopen(table_path, "a");
        if (!f) return fail(RELOC_EINVAL, "autotune: cannot append to %s", table_path);
        fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), out->tile_w, out->tile_h, out->blend_rpl, out->ms_per_query);
        fclose(f);
    }
    return RELOC_OK;
}

extern "C" reloc_status reloc_localize_host(reloc_ctx *ctx, const float *query_host, const double *coarse_pose,
                                            double radius, const reloc_grid *grid, const reloc_camera *cam,
                                            reloc_result *out, float *best_rgb_host, float *best_depth_host,
                                            void *stream)
{
    if (!ctx || !query_host || !cam) return fail(RELOC_EINVAL, "NULL argument");
    if (cam->width < 1 || cam->height < 1 || cam->width > 16383 || cam->height > 16383)
        return fail(RELOC_EINVAL, "image size out of range");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    const size_t HW = (size_t)cam->width * cam->height;
    CKS(ctx->hq.ensure(12 * HW));
    CKS(ctx->hrgb.ensure(12 * HW));
    CKS(ctx->hdepth.ensure(4 * HW));
    CK(cudaMemcpyAsync(ctx->hq.p, query_host, 12 * HW, cudaMemcpyHostToDevice, st));
    CKS(localize_impl(ctx, ctx->hq.as<float>(), coarse_pose, radius, grid, cam, out, nullptr,
                      best_rgb_host ? ctx->hrgb.as<float>() : nullptr, best_depth_host ? ctx->hdepth.as<float>() : nullptr,
                      nullptr, st));
    if (best_rgb_host) CK(cudaMemcpyAsync(best_rgb_host, ctx->hrgb.p, 12 * HW, cudaMemcpyDeviceToHost, st));
    if (best_depth_host) CK(cudaMemcpyAsync(best_depth_host, ctx->hdepth.p, 4 * HW, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return RELOC_OK;
}

extern "C" reloc_status reloc_last_counts(reloc_ctx *ctx, reloc_counts *out)
{
    if (!ctx || !out) return fail(RELOC_EINVAL, "NULL argument");
    *out = ctx->counts;
    return RELOC_OK;
}

extern "C" reloc_status reloc_set_profiling(reloc_ctx *ctx, int enabled)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    ctx->prof = enabled != 0;
    memset(ctx->stage_ms, 0, sizeof ctx->stage_ms);
    memset(ctx->stage_calls, 0, sizeof ctx->stage_calls);
    return RELOC_OK;
}

extern "C" reloc_status reloc_stage_times(reloc_ctx *ctx, double *ms_out, int64_t *calls_out)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    for (int s = 0; s < RELOC_STAGE_COUNT; ++s) {
        if (ms_out) ms_out[s] = ctx->stage_ms[s];
        if (calls_out) calls_out[s] = ctx->stage_calls[s];
    }
    return RELOC_OK;
}

// --------------------------------------------------------------- debug ----

// rectangles of visible pairs (the projection writes none for culled pairs,
// whose depth key is 0xFFFFFFFF)
__global__ void k_unpack_rect(const uint2 *__restrict__ rc, const uint32_t *__restrict__ dkey, int64_t n,
                              int32_t *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (dkey[i] == 0xFFFFFFFFu) {
        out[4 * i] = out[4 * i + 1] = out[4 * i + 2] = out[4 * i + 3] = -1;
    } else {
        const uint2 r = rc[i];
        out[4 * i] = (int32_t)(r.x & 0xFFFF);
        out[4 * i + 1] = (int32_t)(r.y & 0xFFFF);
        out[4 * i + 2] = (int32_t)(r.x >> 16);
        out[4 * i + 3] = (int32_t)(r.y >> 16);
    }
}

extern "C" reloc_status reloc_export_debug(reloc_ctx *ctx, float *records_dev, int32_t *rects_dev,
                                           uint32_t *inst_tiles_dev, uint32_t *inst_gauss_dev, int64_t *inst_count_host,
                                           int32_t *ranges_dev, void *stream)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    if (!ctx->last_valid) return fail(RELOC_EINVAL, "no completed single-query call to export");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    const int64_t VS = (int64_t)ctx->last_V * ctx->last_S;
    const size_t VI = (size_t)ctx->last_io_off.back();
    if (records_dev && VS > 0)
        CK(cudaMemcpyAsync(records_dev, ctx->rec.p, 48 * (size_t)VS, cudaMemcpyDeviceToDevice, st));
    if (rects_dev && VS > 0) {
        k_unpack_rect<<<(unsigned)ceil_div(VS, 256), 256, 0, st>>>(ctx->rect.as<uint2>(), ctx->dkey.as<uint32_t>(), VS,
                                                                  rects_dev);
        CK(cudaGetLastError());
    }
    if (inst_tiles_dev && VI)
        for (int v = 0; v < ctx->last_V; ++v)
            CK(launch_fill_tiles(ctx->ranges.as<int2>() + (int64_t)v * ctx->last_cam.n_tiles, ctx->last_cam.n_tiles,
                                 inst_tiles_dev + ctx->last_io_off[v], st));
    if (inst_gauss_dev && VI)
        CK(cudaMemcpyAsync(inst_gauss_dev, ctx->inst.p, 4 * VI, cudaMemcpyDeviceToDevice, st));
    if (ranges_dev)
        CK(cudaMemcpyAsync(ranges_dev, ctx->ranges.p, sizeof(int2) * (size_t)ctx->last_V * ctx->last_cam.n_tiles,
                           cudaMemcpyDeviceToDevice, st));
    if (inst_count_host)
        for (int v = 0; v < ctx->last_V; ++v) inst_count_host[v] = ctx->last_ninst[v];
    CK(cudaStreamSynchronize(st));
    return RELOC_OK;
}

extern "C" reloc_status reloc_inject_faults(int kind, int count)
{
    if (count < 0 || (kind != RELOC_FAULT_GEMM_WAIT && kind != RELOC_FAULT_ALLOC))
        return fail(RELOC_EINVAL, "inject_faults: kind RELOC_FAULT_GEMM_WAIT or RELOC_FAULT_ALLOC, count >= 0");
    g_faults[kind == RELOC_FAULT_GEMM_WAIT ? FAULT_GEMM_WAIT : FAULT_ALLOC].store(count);
    return RELOC_OK;
}

extern "C" reloc_status reloc_measure_peaks(int device, double *fp32_scalar_tflops, double *fp32_packed_tflops,
                                            double *ex2_gops)
{
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(RELOC_ECUDA, "device %d not present (%d devices)", device, ndev);
    CK(cudaSetDevice(device));
    CK(measure_peaks(fp32_scalar_tflops, fp32_packed_tflops, ex2_gops));
    return RELOC_OK;
}

// ========================================== PnP refinement (Sec. III-C.2) ==
extern "C" void reloc_default_pnp_options(reloc_pnp_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof *opt);
    opt->max_iters = 30;
    opt->huber_px = 2.0;
    opt->alpha_min = 0.5;
    opt->tol = 1e-12;
}

extern "C" reloc_status reloc_refine_pnp(reloc_ctx *ctx, const double *pose_render, const double *pose_init,
                                         const reloc_camera *cam, const float *depth_dev, const float *alpha_dev,
                                         const float *pairs_dev, int n_pairs, const reloc_pnp_options *opt,
                                         reloc_pnp_result *out, void *stream)
{
    if (!ctx || !pose_render || !pose_init || !cam || !depth_dev || !alpha_dev || !pairs_dev || !out)
        return fail(RELOC_EINVAL, "NULL argument");
    if (n_pairs < 1) return fail(RELOC_EINVAL, "n_pairs %d < 1", n_pairs);
    if (cam->width < 2 || cam->height < 2 || cam->width > 16383 || cam->height > 16383)
        return fail(RELOC_EINVAL, "image size %dx%d out of range", cam->width, cam->height);
    if (!(cam->fx > 0) || !(cam->fy > 0) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
        return fail(RELOC_ENUMERIC, "invalid intrinsics");
    reloc_pnp_options o;
    if (opt) o = *opt; else reloc_default_pnp_options(&o);
    if (o.max_iters < 0 || o.max_iters > 1000 || !(o.huber_px > 0) || !(o.tol >= 0) || !std::isfinite(o.alpha_min))
        return fail(RELOC_EINVAL, "bad PnP options");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(pose_render[k]) || !std::isfinite(pose_init[k]))
            return fail(RELOC_ENUMERIC, "non-finite pose");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CKS(ctx->pnp_X.ensure(32 * (size_t)n_pairs + (256 << 10)));   // points, then per-block sums and state
    CKS(ctx->pnp_out.ensure(sizeof(double) * 20));
    CK(launch_refine_pnp(pose_render, pose_init, cam->fx, cam->fy, cam->cx, cam->cy, cam->width, cam->height,
                         depth_dev, alpha_dev, pairs_dev, n_pairs, o.max_iters, o.huber_px, o.alpha_min, o.tol,
                         ctx->pnp_X.as<double>(), ctx->pnp_out.as<double>(), st));
    double h[20];
    CK(cudaMemcpyAsync(h, ctx->pnp_out.p, sizeof h, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    memset(out, 0, sizeof *out);
    memcpy(out->pose, h, sizeof(double) * 16);
    out->rms_px = h[16];
    out->cost = h[17];
    out->n_used = (int32_t)h[18];
    out->iters = (int32_t)h[19];
    if (out->n_used < 3) return fail(RELOC_ENUMERIC, "%d usable pairs (3 needed)", out->n_used);
    return RELOC_OK;
}

// ============================================= NCC pose gradient (NEXT-3) ==
extern "C" reloc_status reloc_score_grad(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges,
                                         const double *poses, int n_views, const reloc_camera *cam,
                                         const float *query_dev, double *scores_host, double *grads_host,
                                         void *stream)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    if (!query_dev || !scores_host || !grads_host) return fail(RELOC_EINVAL, "query_dev, scores_host and grads_host are required");
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    if (ctx->sh_degree != 0) return fail(RELOC_EINVAL, "pose gradients need a map with SH degree 0 (view-independent colour)");
    std::vector<QuerySpec> qs(1);
    CKS(one_query(ctx, ranges, n_ranges, poses, n_views, qs[0]));
    qs[0].img = query_dev;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CKS(ctx->gpose.ensure(48 * (size_t)n_views));
    CallOut o;
    o.score = true;
    o.grad = ctx->gpose.as<double>();
    CKS(run_batch(ctx, qs, cam, st, o, false));
    memcpy(scores_host, o.scores.data(), sizeof(double) * n_views);
    CK(cudaMemcpyAsync(grads_host, ctx->gpose.p, 48 * (size_t)n_views, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return RELOC_OK;
}

// ============================================== map training (NEXT-4) ========
extern "C" void reloc_default_train_options(reloc_train_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof *opt);
    opt->lambda_dssim = 0.2;
    opt->w_photo = 1.0;
    opt->w_reproj = 1.0;
    opt->lr_mean = 1.6e-4;
    opt->lr_scale = 5e-3;
    opt->lr_quat = 1e-3;
    opt->lr_opacity = 5e-2;
    opt->lr_color = 2.5e-3;
    opt->beta1 = 0.9;
    opt->beta2 = 0.999;
    opt->eps = 1e-15;
    opt->reproj_alpha_min = 0.5;
    opt->views_per_group = 16;
}

// The loss of the call and its gradient, added into grad (device [14][n]).
static reloc_status train_loss_grad(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges, const double *poses,
                                    int n_views, const reloc_camera *cam, const float *targets_dev,
                                    const reloc_train_options &o, float *grad, double *loss_host, cudaStream_t st)
{
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    if (ctx->sh_degree != 0) return fail(RELOC_EINVAL, "map training needs SH degree 0 (plain RGB colours)");
    if (ctx->precision != RELOC_FP32) return fail(RELOC_EINVAL, "map training needs FP32 attributes");
    if (!targets_dev || !poses || !cam || !loss_host) return fail(RELOC_EINVAL, "NULL argument");
    if (n_views < 1) return fail(RELOC_EINVAL, "n_views %d < 1", n_views);
    if (!(o.lambda_dssim >= 0 && o.lambda_dssim <= 1) || !(o.w_photo >= 0) || !(o.w_reproj >= 0) ||
        !std::isfinite(o.w_photo) || !std::isfinite(o.w_reproj) || o.views_per_group < 1 || o.views_per_group > 4096)
        return fail(RELOC_EINVAL, "bad training options");
    if (!(o.reproj_alpha_min > 0) || !std::isfinite(o.reproj_alpha_min))
        return fail(RELOC_EINVAL, "reproj_alpha_min must be > 0");
    if (n_ranges < 0 || (n_ranges > 0 && !ranges)) return fail(RELOC_EINVAL, "bad ranges");
    if (cam->width < 1 || cam->height < 1) return fail(RELOC_EINVAL, "bad camera");
    const int64_t HW = (int64_t)cam->width * cam->height;
    std::vector<QuerySpec> qs;
    for (int v0 = 0; v0 < n_views; v0 += o.views_per_group) {
        QuerySpec q;
        CKS(one_query(ctx, ranges, n_ranges, poses + 16 * (size_t)v0, std::min(o.views_per_group, n_views - v0), q));
        qs.push_back(std::move(q));
    }
    CK(cudaSetDevice(ctx->device));
    CKS(ctx->tloss.ensure(8));
    CallOut co;
    co.target = targets_dev;
    co.l1_scale = o.w_photo * (1.0 - o.lambda_dssim) / ((double)n_views * 3.0 * (double)HW);
    co.ssim_scale = o.w_photo * o.lambda_dssim / ((double)n_views * 3.0 * (double)HW);
    co.n_views_total = n_views;
    if (o.w_reproj > 0 && n_views > 1) {
        // relative pose of each view to the next: P_{t+1} = R_rel P_t + t_rel
        std::vector<float> rel((size_t)12 * n_views, 0.f);
        for (int t = 0; t + 1 < n_views; ++t) {
            const double *A = poses + 16 * (size_t)t, *B = poses + 16 * (size_t)(t + 1);
            for (int k = 0; k < 16; ++k)
                if (!std::isfinite(A[k]) || !std::isfinite(B[k])) return fail(RELOC_ENUMERIC, "non-finite pose");
            double R[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    R[3 * i + j] = B[4 * i] * A[4 * j] + B[4 * i + 1] * A[4 * j + 1] + B[4 * i + 2] * A[4 * j + 2];
            for (int i = 0; i < 9; ++i) rel[12 * (size_t)t + i] = (float)R[i];
            for (int i = 0; i < 3; ++i)
                rel[12 * (size_t)t + 9 + i] =
                    (float)(B[4 * i + 3] - (R[3 * i] * A[3] + R[3 * i + 1] * A[7] + R[3 * i + 2] * A[11]));
        }
        CKS(ctx->trel.ensure(sizeof(float) * rel.size()));
        CK(cudaMemcpyAsync(ctx->trel.p, rel.data(), sizeof(float) * rel.size(), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        co.rel = ctx->trel.as<float>();
        co.rp_l1_scale = o.w_reproj * (1.0 - o.lambda_dssim) / ((double)(n_views - 1) * 3.0 * (double)HW);
        co.rp_ssim_scale = o.w_reproj * o.lambda_dssim / ((double)(n_views - 1) * 3.0 * (double)HW);
        co.rp_alpha_min = (float)o.reproj_alpha_min;
    }
    co.tgrad = grad;
    CKS(run_batch(ctx, qs, cam, st, co, false));
    CK(cudaMemcpyAsync(loss_host, ctx->tloss.p, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return RELOC_OK;
}

extern "C" reloc_status reloc_train_grad(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges,
                                         const double *poses, int n_views, const reloc_camera *cam,
                                         const float *targets_dev, const reloc_train_options *opt,
                                         double *loss_host, float *grad_dev, void *stream)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    if (!grad_dev) return fail(RELOC_EINVAL, "grad_dev is NULL");
    reloc_train_options o;
    if (opt) o = *opt; else reloc_default_train_options(&o);
    return train_loss_grad(ctx, ranges, n_ranges, poses, n_views, cam, targets_dev, o, grad_dev, loss_host,
                           (cudaStream_t)stream);
}

extern "C" reloc_status reloc_train_step(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges,
                                         const double *poses, int n_views, const reloc_camera *cam,
                                         const float *targets_dev, const reloc_train_options *opt,
                                         double *loss_host, void *stream)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    reloc_train_options o;
    if (opt) o = *opt; else reloc_default_train_options(&o);
    const double lrs[5] = {o.lr_mean, o.lr_scale, o.lr_quat, o.lr_opacity, o.lr_color};
    for (double l : lrs)
        if (!(l >= 0) || !std::isfinite(l)) return fail(RELOC_EINVAL, "bad learning rate");
    if (!(o.beta1 >= 0 && o.beta1 < 1) || !(o.beta2 >= 0 && o.beta2 < 1) || !(o.eps >= 0))
        return fail(RELOC_EINVAL, "bad Adam parameters");
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    const size_t pbytes = sizeof(float) * 14 * (size_t)ctx->n;
    CKS(ctx->tgrad.ensure(pbytes));
    CKS(train_loss_grad(ctx, ranges, n_ranges, poses, n_views, cam, targets_dev, o, ctx->tgrad.as<float>(),
                        loss_host, st));
    CKS(ctx->adam_m.ensure(pbytes));
    CKS(ctx->adam_v.ensure(pbytes));
    if (ctx->adam_t == 0) {
        CK(cudaMemsetAsync(ctx->adam_m.p, 0, pbytes, st));
        CK(cudaMemsetAsync(ctx->adam_v.p, 0, pbytes, st));
    }
    ctx->adam_t += 1;
    AdamParams P;
    for (int k = 0; k < 5; ++k) P.lr[k] = (float)lrs[k];
    P.beta1 = (float)o.beta1;
    P.beta2 = (float)o.beta2;
    P.eps = (float)o.eps;
    P.bc1 = (float)(1.0 / (1.0 - std::pow(o.beta1, (double)ctx->adam_t)));
    P.bc2 = (float)(1.0 / (1.0 - std::pow(o.beta2, (double)ctx->adam_t)));
    P.o_min = 1e-6f;
    CK(launch_adam(ctx->mean.as<float>(), ctx->attr.as<float>(), ctx->tgrad.as<float>(), ctx->adam_m.as<float>(),
                   ctx->adam_v.as<float>(), ctx->n, P, st));
    CK(cudaStreamSynchronize(st));
    return RELOC_OK;
}

extern "C" reloc_status reloc_train_reset(reloc_ctx *ctx)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    ctx->adam_t = 0;
    return RELOC_OK;
}

extern "C" reloc_status reloc_read_map(reloc_ctx *ctx, float *mean, float *scale, float *quat, float *opacity,
                                       float *sh)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    if (ctx->precision != RELOC_FP32) return fail(RELOC_EINVAL, "reading the map back needs FP32 attributes");
    const int64_t n = ctx->n;
    const int K = (ctx->sh_degree + 1) * (ctx->sh_degree + 1);
    const size_t nc = attr_components(ctx->sh_degree);
    CK(cudaSetDevice(ctx->device));
    std::vector<float> m((size_t)3 * n), a(nc * (size_t)n);
    CK(cudaMemcpy(m.data(), ctx->mean.p, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(a.data(), ctx->attr.p, sizeof(float) * nc * n, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            if (mean) mean[3 * i + k] = m[(size_t)k * n + i];
            if (scale) scale[3 * i + k] = a[(size_t)(ATTR_SCALE + k) * n + i];
        }
        for (int k = 0; k < 4; ++k)
            if (quat) quat[4 * i + k] = a[(size_t)(ATTR_QUAT + k) * n + i];
        if (opacity) opacity[i] = a[(size_t)ATTR_OPAC * n + i];
        if (sh)
            for (int k = 0; k < 3 * K; ++k) sh[(size_t)3 * K * i + k] = a[(size_t)(ATTR_SH + k) * n + i];
    }
    return RELOC_OK;
}
