// api.cu -- the C ABI of reloc.h: context, map load, block selection,
// candidate grid, and the per-call orchestration of the kernels
// (K1 gather -> K2 project -> depth sort -> K3 emit -> K4 tile sort ->
//  K5 ranges -> K6 blend + NCC partials -> K7 NCC -> K8 argmax -> export).
//
// All stages run on the caller's stream with device-resident counts, so a
// call needs one host synchronisation at its end (to return scores and to
// check workspace capacity).  If a view produced more tile instances than
// the workspace holds, the call grows the workspace to the size the device
// reported and re-runs from the emission stage.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "blockindex.h"
#include "internal.cuh"
#include "reloc.h"

using namespace reloc;

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

// pinned readback block written at the end of every call
struct Readback {
    int overflow;
    int best;
    unsigned long long need;
    double best_score;
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
    // workspace
    DevBuf gidx, runs, views, rec, rect, ntiles, dkey, k1a, v1a, k1b, v1b, nvis, hist1, chunk_sums;
    DevBuf ikA, ivA, ikB, ivB, ninst, hist2, ranges, partials, qpart, qstats, scores, degen, best, best_score, flags;
    DevBuf hq, hrgb, hdepth;
    PinBuf pin;
    int64_t inst_stride = 0;
    // last call
    int last_V = 0;
    int64_t last_S = 0;
    CamParams last_cam{};
    bool last_valid = false;
    bool last_final_b = false;      // final instance lists live in ikB/ivB
    std::vector<int64_t> last_ninst;
    reloc_counts counts{};
    // profiling
    bool prof = false;
    cudaEvent_t ev[RELOC_STAGE_COUNT + 1] = {};
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
    cfg->inst_capacity = 1 << 20;
    cfg->blend_rpl = 1;
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
        !(c.det_fp64 >= 0) || !(c.block_size > 0) || c.inst_capacity < 1 || c.blend_rpl < 1 || c.blend_rpl > 2)
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
    ctx->inst_stride = c.inst_capacity;
    for (auto &e : ctx->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            reloc_destroy(ctx);
            return fail(RELOC_ECUDA, "cudaEventCreate failed");
        }
    }
    *out = ctx;
    return RELOC_OK;
}

extern "C" reloc_status reloc_destroy(reloc_ctx *ctx)
{
    if (!ctx) return RELOC_OK;
    cudaSetDevice(ctx->device);
    DevBuf *bufs[] = {&ctx->mean, &ctx->attr, &ctx->gidx, &ctx->runs, &ctx->views, &ctx->rec, &ctx->rect,
                      &ctx->ntiles, &ctx->dkey, &ctx->k1a, &ctx->v1a, &ctx->k1b, &ctx->v1b, &ctx->nvis,
                      &ctx->hist1, &ctx->chunk_sums, &ctx->ikA, &ctx->ivA, &ctx->ikB, &ctx->ivB, &ctx->ninst,
                      &ctx->hist2, &ctx->ranges, &ctx->partials, &ctx->qpart, &ctx->qstats, &ctx->scores,
                      &ctx->degen, &ctx->best, &ctx->best_score, &ctx->flags, &ctx->hq, &ctx->hrgb, &ctx->hdepth};
    for (DevBuf *b : bufs) b->release();
    ctx->pin.release();
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
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
    return RELOC_OK;
}

static reloc_status make_views(const double *poses, int V, std::vector<ViewParams> &vp)
{
    vp.resize(V);
    for (int v = 0; v < V; ++v) {
        const double *W = poses + 16 * v;
        for (int k = 0; k < 16; ++k)
            if (!std::isfinite(W[k])) return fail(RELOC_ENUMERIC, "non-finite pose %d", v);
        ViewParams &P = vp[v];
        memset(&P, 0, sizeof P);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) P.R[3 * r + c] = (float)W[4 * r + c];
        for (int i = 0; i < 3; ++i) {
            const double C = -(W[i] * W[3] + W[4 + i] * W[7] + W[8 + i] * W[11]);
            P.c_hi[i] = (float)C;
            P.c_lo[i] = (float)(C - (double)P.c_hi[i]);
        }
    }
    return RELOC_OK;
}

struct CallOut {
    const float *query = nullptr;    // device; scores computed if non-null
    float *rgb = nullptr, *depth = nullptr, *alpha = nullptr;          // all views
    bool export_best = false;
    float *brgb = nullptr, *bdepth = nullptr, *balpha = nullptr;       // winner
    double *scores_host = nullptr;
    int *degen_host = nullptr;
    int best = -1;
    double best_score = 0;
};

static void stage_mark(reloc_ctx *ctx, int s, cudaStream_t st)
{
    if (ctx->prof) cudaEventRecord(ctx->ev[s], st);
}

static reloc_status run_views(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges, const double *poses, int V,
                              const reloc_camera *cam, cudaStream_t st, CallOut &o)
{
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    if (V < 1 || V > 4096) return fail(RELOC_EINVAL, "n_views %d not in 1..4096", V);
    if (!poses) return fail(RELOC_EINVAL, "poses is NULL");
    if (n_ranges < 0 || (n_ranges > 0 && !ranges)) return fail(RELOC_EINVAL, "bad ranges");
    int64_t S = 0;
    for (int r = 0; r < n_ranges; ++r) {
        if (ranges[r].begin < 0 || ranges[r].end < ranges[r].begin || ranges[r].end > ctx->n)
            return fail(RELOC_EINVAL, "range %d [%lld, %lld) outside the map", r, (long long)ranges[r].begin,
                        (long long)ranges[r].end);
        S += ranges[r].end - ranges[r].begin;
    }
    if (S > (int64_t)UINT32_MAX / 4) return fail(RELOC_EINVAL, "subset too large");
    CamParams cp;
    CKS(make_cam(ctx, cam, cp));
    std::vector<ViewParams> vp;
    CKS(make_views(poses, V, vp));
    CK(cudaSetDevice(ctx->device));
    ctx->last_valid = false;

    const int64_t HW = (int64_t)cp.width * cp.height;
    const int64_t S1 = S > 0 ? S : 1;
    // ---- workspace --------------------------------------------------------
    const size_t VS = (size_t)V * S1;
    CKS(ctx->gidx.ensure(4 * S1));
    CKS(ctx->runs.ensure(16 * (size_t)(n_ranges + 1)));
    CKS(ctx->views.ensure(sizeof(ViewParams) * V));
    CKS(ctx->rec.ensure(48 * VS));
    CKS(ctx->rect.ensure(8 * VS));
    CKS(ctx->ntiles.ensure(4 * VS));
    CKS(ctx->dkey.ensure(4 * VS));
    CKS(ctx->k1a.ensure(4 * VS));
    CKS(ctx->v1a.ensure(4 * VS));
    CKS(ctx->k1b.ensure(4 * VS));
    CKS(ctx->v1b.ensure(4 * VS));
    CKS(ctx->nvis.ensure(4 * (size_t)V));
    CKS(ctx->hist1.ensure(4 * (size_t)radix_hist_words(V, S1)));
    CKS(ctx->chunk_sums.ensure(4 * (size_t)emit_chunk_words(V, S1)));
    CKS(ctx->ninst.ensure(4 * (size_t)V));
    CKS(ctx->ranges.ensure(sizeof(int2) * (size_t)V * cp.n_tiles));
    CKS(ctx->partials.ensure(24 * (size_t)V * cp.n_tiles));
    CKS(ctx->qpart.ensure(16 * 256));
    CKS(ctx->qstats.ensure(16));
    CKS(ctx->scores.ensure(8 * (size_t)V));
    CKS(ctx->degen.ensure(4 * (size_t)V));
    CKS(ctx->best.ensure(16));
    CKS(ctx->best_score.ensure(16));
    CKS(ctx->flags.ensure(64));
    const size_t pin_need = sizeof(Readback) + 16 * (size_t)(n_ranges + 1) + sizeof(ViewParams) * V +
                            (8 + 4 + 4 + 4) * (size_t)V + 64;
    CKS(ctx->pin.ensure(pin_need));

    // ---- uploads (pinned staging) -----------------------------------------
    char *pin = (char *)ctx->pin.p;
    Readback *rb = (Readback *)pin;
    int64_t *h_runs = (int64_t *)(pin + sizeof(Readback));
    ViewParams *h_views = (ViewParams *)(h_runs + 2 * (n_ranges + 1));
    double *h_scores = (double *)(h_views + V);
    int *h_degen = (int *)(h_scores + V);
    uint32_t *h_nvis = (uint32_t *)(h_degen + V);
    uint32_t *h_ninst = h_nvis + V;
    {
        int64_t off = 0;
        for (int r = 0; r < n_ranges; ++r) {
            h_runs[r] = ranges[r].begin;
            h_runs[n_ranges + 1 + r] = off;
            off += ranges[r].end - ranges[r].begin;
        }
        h_runs[n_ranges] = 0;
        h_runs[n_ranges + 1 + n_ranges] = off;
    }
    memcpy(h_views, vp.data(), sizeof(ViewParams) * V);
    CK(cudaMemcpyAsync(ctx->runs.p, h_runs, 16 * (size_t)(n_ranges + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->views.p, h_views, sizeof(ViewParams) * V, cudaMemcpyHostToDevice, st));
    const int64_t *d_run_begin = ctx->runs.as<int64_t>();
    const int64_t *d_run_off = d_run_begin + n_ranges + 1;

    int *d_overflow = ctx->flags.as<int>();
    unsigned long long *d_need = (unsigned long long *)(ctx->flags.as<char>() + 8);

    // ---- K1 + K2 + depth sort (done once per call) ------------------------
    stage_mark(ctx, RELOC_STAGE_CULL, st);
    int launches = 0;
    if (S > 0) { CK(launch_gather_subset(d_run_begin, d_run_off, n_ranges, S, ctx->gidx.as<uint32_t>(), st)); launches += 1; }
    stage_mark(ctx, RELOC_STAGE_PROJECT, st);
    if (S > 0) launches += 1;
    if (S > 0)
        CK(launch_project(ctx->mean.as<float>(), ctx->mean.as<float>() + ctx->n, ctx->mean.as<float>() + 2 * ctx->n,
                          ctx->attr.p, ctx->precision, ctx->sh_degree, ctx->n, ctx->gidx.as<uint32_t>(), S,
                          ctx->views.as<ViewParams>(), V, cp, ctx->rec.as<float4>(), ctx->rect.as<uint2>(),
                          ctx->ntiles.as<uint32_t>(), ctx->dkey.as<uint32_t>(), st));
    stage_mark(ctx, RELOC_STAGE_DEPTH_SORT, st);
    CK(cudaMemsetAsync(ctx->nvis.p, 0, 4 * (size_t)V, st));
    if (S > 0) {
        RadixPass p{};
        p.V = V;
        p.stride = S;
        p.cps = (int)ceil_div(S, SORT_CHUNK);
        p.hist = ctx->hist1.as<uint32_t>();
        p.mask = 0xFF;
        uint32_t *ka = ctx->k1a.as<uint32_t>(), *va = ctx->v1a.as<uint32_t>();
        uint32_t *kb = ctx->k1b.as<uint32_t>(), *vb = ctx->v1b.as<uint32_t>();
        // pass 0: dense (view, Gaussian) arrays, invisible pairs dropped
        p.keys_in = ctx->dkey.as<uint32_t>();
        p.vals_in = nullptr;
        p.filt = ctx->ntiles.as<uint32_t>();
        p.len = nullptr;
        p.keys_out = ka;
        p.vals_out = va;
        p.len_out = ctx->nvis.as<uint32_t>();
        p.shift = 0;
        CK(launch_radix_pass(p, st));
        launches += 3;
        p.filt = nullptr;
        p.len = ctx->nvis.as<uint32_t>();
        p.len_out = nullptr;
        for (int pass = 1; pass < 4; ++pass) {
            p.shift = 8 * pass;
            p.keys_in = (pass & 1) ? ka : kb;
            p.vals_in = (pass & 1) ? va : vb;
            p.keys_out = (pass & 1) ? kb : ka;
            p.vals_out = (pass & 1) ? vb : va;
            CK(launch_radix_pass(p, st));
            launches += 3;
        }
    }
    const uint32_t *sorted_g = ctx->v1b.as<uint32_t>();   // after 4 passes

    // ---- instance stages (re-run if the instance workspace overflows) -----
    int retries = 0;
    for (;;) {
        const int64_t IS = ctx->inst_stride;
        const size_t VI = (size_t)V * IS;
        CKS(ctx->ikA.ensure(4 * VI));
        CKS(ctx->ivA.ensure(4 * VI));
        CKS(ctx->ikB.ensure(4 * VI));
        CKS(ctx->ivB.ensure(4 * VI));
        CKS(ctx->hist2.ensure(4 * (size_t)radix_hist_words(V, IS)));
        CK(cudaMemsetAsync(ctx->flags.p, 0, 64, st));
        CK(cudaMemsetAsync(ctx->ninst.p, 0, 4 * (size_t)V, st));
        stage_mark(ctx, RELOC_STAGE_EMIT, st);
        if (S > 0) launches += 3;
        if (S > 0)
            CK(launch_emit(sorted_g, ctx->nvis.as<uint32_t>(), ctx->ntiles.as<uint32_t>(), ctx->rect.as<uint2>(), S, V,
                           cp.ntx, IS, ctx->chunk_sums.as<uint32_t>(), ctx->ikA.as<uint32_t>(),
                           ctx->ivA.as<uint32_t>(), ctx->ninst.as<uint32_t>(), d_need, d_overflow, st));
        stage_mark(ctx, RELOC_STAGE_TILE_SORT, st);
        bool final_b = false;
        if (S > 0 && cp.tile_bits > 0) {
            RadixPass p{};
            p.V = V;
            p.stride = IS;
            p.cps = (int)ceil_div(IS, SORT_CHUNK);
            p.hist = ctx->hist2.as<uint32_t>();
            p.len = ctx->ninst.as<uint32_t>();
            const int b1 = cp.tile_bits <= 8 ? cp.tile_bits : (cp.tile_bits + 1) / 2;
            const int b2 = cp.tile_bits - b1;
            p.keys_in = ctx->ikA.as<uint32_t>();
            p.vals_in = ctx->ivA.as<uint32_t>();
            p.keys_out = ctx->ikB.as<uint32_t>();
            p.vals_out = ctx->ivB.as<uint32_t>();
            p.shift = 0;
            p.mask = (1u << b1) - 1;
            CK(launch_radix_pass(p, st));
            launches += 3;
            final_b = true;
            if (b2 > 0) {
                p.keys_in = ctx->ikB.as<uint32_t>();
                p.vals_in = ctx->ivB.as<uint32_t>();
                p.keys_out = ctx->ikA.as<uint32_t>();
                p.vals_out = ctx->ivA.as<uint32_t>();
                p.shift = b1;
                p.mask = (1u << b2) - 1;
                CK(launch_radix_pass(p, st));
                launches += 3;
                final_b = false;
            }
        }
        const uint32_t *ftile = final_b ? ctx->ikB.as<uint32_t>() : ctx->ikA.as<uint32_t>();
        const uint32_t *fgauss = final_b ? ctx->ivB.as<uint32_t>() : ctx->ivA.as<uint32_t>();
        ctx->last_final_b = final_b;
        stage_mark(ctx, RELOC_STAGE_RANGES, st);
        launches += 1;
        CK(launch_ranges(ftile, ctx->ninst.as<uint32_t>(), IS, V, cp.n_tiles, ctx->ranges.as<int2>(), d_overflow, st));
        stage_mark(ctx, RELOC_STAGE_BLEND, st);
        if (o.query) launches += 2;
        if (o.query) CK(launch_query_stats(o.query, 3 * HW, ctx->qpart.as<double>(), ctx->qstats.as<double>(), st));
        launches += 1;
        CK(launch_blend(ctx->rec.as<float4>(), S1, fgauss, IS, ctx->ranges.as<int2>(), V, cp, o.query,
                        o.query ? ctx->partials.as<double>() : nullptr, o.rgb, o.depth, o.alpha, nullptr, d_overflow,
                        st));
        stage_mark(ctx, RELOC_STAGE_SCORE, st);
        if (o.query) {
            launches += 1;
            CK(launch_ncc_finalize(ctx->partials.as<double>(), ctx->qstats.as<double>(), V, cp.n_tiles, 3 * HW,
                                   ctx->scores.as<double>(), ctx->degen.as<int>(), st));
            if (o.export_best) {
                launches += 1;
                CK(launch_argmax(ctx->scores.as<double>(), V, ctx->best.as<int>(), ctx->best_score.as<double>(), st));
                if (o.brgb || o.bdepth || o.balpha) launches += 1;
                if (o.brgb || o.bdepth || o.balpha)
                    CK(launch_blend(ctx->rec.as<float4>(), S1, fgauss, IS, ctx->ranges.as<int2>(), V, cp, nullptr,
                                    nullptr, o.brgb, o.bdepth, o.balpha, ctx->best.as<int>(), d_overflow, st));
            }
        }
        stage_mark(ctx, RELOC_STAGE_COUNT, st);
        // ---- readback -----------------------------------------------------
        CK(cudaMemcpyAsync(&rb->overflow, d_overflow, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&rb->need, d_need, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_nvis, ctx->nvis.p, 4 * (size_t)V, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_ninst, ctx->ninst.p, 4 * (size_t)V, cudaMemcpyDeviceToHost, st));
        if (o.query) {
            CK(cudaMemcpyAsync(h_scores, ctx->scores.p, 8 * (size_t)V, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(h_degen, ctx->degen.p, 4 * (size_t)V, cudaMemcpyDeviceToHost, st));
            if (o.export_best) {
                CK(cudaMemcpyAsync(&rb->best, ctx->best.p, 4, cudaMemcpyDeviceToHost, st));
                CK(cudaMemcpyAsync(&rb->best_score, ctx->best_score.p, 8, cudaMemcpyDeviceToHost, st));
            }
        }
        CK(cudaStreamSynchronize(st));
        CK(cudaGetLastError());
        if (ctx->prof) {
            for (int s = 0; s < RELOC_STAGE_COUNT; ++s) {
                float ms = 0;
                if (cudaEventElapsedTime(&ms, ctx->ev[s], ctx->ev[s + 1]) == cudaSuccess) {
                    ctx->stage_ms[s] += ms;
                    ctx->stage_calls[s] += 1;
                } else {
                    cudaGetLastError();
                }
            }
        }
        if (!rb->overflow) break;
        if (++retries > 3) return fail(RELOC_EOVERFLOW, "tile-instance workspace still too small after %d grows", retries);
        int64_t grow = (int64_t)rb->need + rb->need / 4 + 4096;
        ctx->inst_stride = ceil_div(grow, SORT_CHUNK) * SORT_CHUNK;
    }

    // ---- results ------------------------------------------------------------
    ctx->last_V = V;
    ctx->last_S = S;
    ctx->last_cam = cp;
    ctx->last_valid = true;
    ctx->last_ninst.assign(V, 0);
    reloc_counts &c = ctx->counts;
    memset(&c, 0, sizeof c);
    c.n_views = V;
    c.n_gauss = S;
    c.inst_stride = ctx->inst_stride;
    c.retries = retries;
    c.kernel_launches = launches;
    for (int v = 0; v < V; ++v) {
        c.n_visible += h_nvis[v];
        c.n_instances += h_ninst[v];
        ctx->last_ninst[v] = h_ninst[v];
    }
    if (o.query) {
        if (o.scores_host) memcpy(o.scores_host, h_scores, 8 * (size_t)V);
        if (o.degen_host) memcpy(o.degen_host, h_degen, 4 * (size_t)V);
        if (o.export_best) {
            o.best = rb->best;
            o.best_score = rb->best_score;
        }
    }
    return RELOC_OK;
}

// ============================================================== entry points ==

extern "C" reloc_status reloc_render(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges, const double *poses,
                                     int n_views, const reloc_camera *cam, float *rgb_dev, float *depth_dev,
                                     float *alpha_dev, void *stream)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    CallOut o;
    o.rgb = rgb_dev;
    o.depth = depth_dev;
    o.alpha = alpha_dev;
    return run_views(ctx, ranges, n_ranges, poses, n_views, cam, (cudaStream_t)stream, o);
}

extern "C" reloc_status reloc_score(reloc_ctx *ctx, const reloc_range *ranges, int n_ranges, const double *poses,
                                    int n_views, const reloc_camera *cam, const float *query_dev, double *scores_host,
                                    int *degenerate_host, void *stream)
{
    if (!ctx) return fail(RELOC_EINVAL, "NULL context");
    if (!query_dev || !scores_host) return fail(RELOC_EINVAL, "query_dev and scores_host are required");
    CallOut o;
    o.query = query_dev;
    o.scores_host = scores_host;
    o.degen_host = degenerate_host;
    return run_views(ctx, ranges, n_ranges, poses, n_views, cam, (cudaStream_t)stream, o);
}

static reloc_status localize_impl(reloc_ctx *ctx, const float *query_dev, const double *coarse_pose, double radius,
                                  const reloc_grid *grid, const reloc_camera *cam, reloc_result *out,
                                  double *scores_host, float *brgb, float *bdepth, float *balpha, cudaStream_t st)
{
    if (!ctx || !query_dev || !coarse_pose || !grid || !cam || !out) return fail(RELOC_EINVAL, "NULL argument");
    if (ctx->n == 0) return fail(RELOC_ENOMAP, "no map loaded");
    if (grid->nx < 1 || grid->ny < 1 || grid->nyaw < 1 || (int64_t)grid->nx * grid->ny * grid->nyaw > 4096)
        return fail(RELOC_EINVAL, "grid %dx%dx%d not in 1..4096 candidates", grid->nx, grid->ny, grid->nyaw);
    if (!std::isfinite(grid->step_xy) || !std::isfinite(grid->step_yaw_deg))
        return fail(RELOC_ENUMERIC, "non-finite grid step");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(coarse_pose[k])) return fail(RELOC_ENUMERIC, "non-finite coarse pose");
    const double *W = coarse_pose;
    const double Cx = -(W[0] * W[3] + W[4] * W[7] + W[8] * W[11]);
    const double Cy = -(W[1] * W[3] + W[5] * W[7] + W[9] * W[11]);
    std::vector<int> ids;
    ctx->blocks.range(Cx, Cy, radius, ids);
    std::vector<reloc_range> runs;
    merge_runs(ctx->blocks, ids, runs);
    std::vector<double> poses;
    grid_poses(coarse_pose, *grid, poses);
    const int V = grid->nx * grid->ny * grid->nyaw;
    std::vector<int> degen(V);
    std::vector<double> sc(V);
    CallOut o;
    o.query = query_dev;
    o.export_best = true;
    o.brgb = brgb;
    o.bdepth = bdepth;
    o.balpha = balpha;
    o.scores_host = sc.data();
    o.degen_host = degen.data();
    CKS(run_views(ctx, runs.data(), (int)runs.size(), poses.data(), V, cam, st, o));
    memset(out, 0, sizeof *out);
    out->best_index = o.best;
    out->n_candidates = V;
    out->best_score = o.best_score;
    if (o.best >= 0 && o.best < V) {
        memcpy(out->best_pose, poses.data() + 16 * o.best, sizeof(double) * 16);
        out->degenerate = degen[o.best];
    }
    out->n_gauss = ctx->counts.n_gauss;
    out->n_blocks = (int)ids.size();
    if (scores_host) memcpy(scores_host, sc.data(), sizeof(double) * V);
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

__global__ void k_unpack_rect(const uint2 *__restrict__ rc, int64_t n, int32_t *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint2 r = rc[i];
    if (r.x == 0xFFFFFFFFu) {
        out[4 * i] = out[4 * i + 1] = out[4 * i + 2] = out[4 * i + 3] = -1;
    } else {
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
    if (!ctx->last_valid) return fail(RELOC_EINVAL, "no completed call to export");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    const int64_t VS = (int64_t)ctx->last_V * ctx->last_S;
    const size_t VI = (size_t)ctx->last_V * ctx->inst_stride;
    if (records_dev && VS > 0)
        CK(cudaMemcpyAsync(records_dev, ctx->rec.p, 48 * (size_t)VS, cudaMemcpyDeviceToDevice, st));
    if (rects_dev && VS > 0) {
        k_unpack_rect<<<(unsigned)ceil_div(VS, 256), 256, 0, st>>>(ctx->rect.as<uint2>(), VS, rects_dev);
        CK(cudaGetLastError());
    }
    if (inst_tiles_dev)
        CK(cudaMemcpyAsync(inst_tiles_dev, ctx->last_final_b ? ctx->ikB.p : ctx->ikA.p, 4 * VI,
                           cudaMemcpyDeviceToDevice, st));
    if (inst_gauss_dev)
        CK(cudaMemcpyAsync(inst_gauss_dev, ctx->last_final_b ? ctx->ivB.p : ctx->ivA.p, 4 * VI,
                           cudaMemcpyDeviceToDevice, st));
    if (ranges_dev)
        CK(cudaMemcpyAsync(ranges_dev, ctx->ranges.p, sizeof(int2) * (size_t)ctx->last_V * ctx->last_cam.n_tiles,
                           cudaMemcpyDeviceToDevice, st));
    if (inst_count_host)
        for (int v = 0; v < ctx->last_V; ++v) inst_count_host[v] = ctx->last_ninst[v];
    CK(cudaStreamSynchronize(st));
    return RELOC_OK;
}
