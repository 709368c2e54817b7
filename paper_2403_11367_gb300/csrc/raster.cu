// raster.cu -- K6 per-tile front-to-back blending of RGB and depth, with the
// NCC sums of each tile fused into its epilogue (K7 partials), the NCC
// finalisation per view (K7) and the argmax over candidates (K8).
//
// Blending follows Sec. III-A of 3DGS-ReLoc: C(x) = sum_i c_i q_i(x) T_i and
// D(x) = sum_i z_i q_i(x) T_i with T_i = prod_{j<i} (1 - q_j(x)), footprint
// q_i(x) = o_i exp(-1/2 d^T Sigma'^-1 d) (Eq. footprint without the Jacobian
// normalisation), d = x - mu_hat.  NCC is Eq. ncc over all 3*H*W samples.
#include "internal.cuh"

namespace reloc {

// ------------------------------------------------------ query statistics ---

constexpr int QS_BLOCKS = 152;
constexpr int QS_THREADS = 256;

__device__ __forceinline__ double warp_sum_d(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ float warp_sum_f(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// Fixed grid and fixed reduction order: the sums are deterministic.
__global__ void __launch_bounds__(QS_THREADS) k_query_stats(const float *__restrict__ q, int64_t n, double *part)
{
    __shared__ double s[2][QS_THREADS / 32];
    double a = 0, b = 0;
    for (int64_t j = (int64_t)blockIdx.x * QS_THREADS + threadIdx.x; j < n; j += (int64_t)QS_BLOCKS * QS_THREADS) {
        double x = q[j];
        a += x;
        b += x * x;
    }
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if ((threadIdx.x & 31) == 0) { s[0][threadIdx.x >> 5] = a; s[1][threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0, B = 0;
        for (int w = 0; w < QS_THREADS / 32; ++w) { A += s[0][w]; B += s[1][w]; }
        part[2 * blockIdx.x] = A;
        part[2 * blockIdx.x + 1] = B;
    }
}

__global__ void k_query_stats_final(const double *part, double *qstats)
{
    double A = 0, B = 0;
    for (int k = 0; k < QS_BLOCKS; ++k) { A += part[2 * k]; B += part[2 * k + 1]; }
    qstats[0] = A;
    qstats[1] = B;
}

cudaError_t launch_query_stats(const float *query, int64_t n, double *block_scratch, double *qstats, cudaStream_t st)
{
    k_query_stats<<<QS_BLOCKS, QS_THREADS, 0, st>>>(query, n, block_scratch);
    k_query_stats_final<<<1, 1, 0, st>>>(block_scratch, qstats);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ K6 -----
// One CTA per (view, tile), one thread per pixel.  Records of the tile's
// sorted list are staged through shared memory in batches of one record per
// thread; the CTA stops early once every pixel's transmittance has run out.

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH)
k_blend(const float4 *__restrict__ rec, int64_t S, const uint32_t *__restrict__ inst_gauss, int64_t inst_stride,
        const int2 *__restrict__ ranges, CamParams cam, const float *__restrict__ query, double *__restrict__ partials,
        float *__restrict__ rgb, float *__restrict__ depth, float *__restrict__ alpha, const int *__restrict__ view_sel,
        const int *__restrict__ overflow)
{
    constexpr int NT = TW * TH;
    constexpr int NW = NT / 32;
    __shared__ float4 s_a[NT];   // u, v, depth, opacity
    __shared__ float4 s_b[NT];   // conic a, b, c
    __shared__ float4 s_c[NT];   // red, green, blue
    __shared__ double s_red[3][NW];

    const int tile = blockIdx.x;
    const int v = view_sel ? *view_sel : (int)blockIdx.y;
    const int out_v = view_sel ? 0 : (int)blockIdx.y;
    const int tx = tile % cam.ntx, ty = tile / cam.ntx;
    const int px = tx * TW + (int)(threadIdx.x % TW);
    const int py = ty * TH + (int)(threadIdx.x / TW);
    const bool inside = px < cam.width && py < cam.height;
    const float fxp = (float)px + 0.5f, fyp = (float)py + 0.5f;

    int2 r = make_int2(0, 0);
    if (!*overflow && v >= 0) r = ranges[(int64_t)v * cam.n_tiles + tile];
    const uint32_t *list = inst_gauss + (int64_t)v * inst_stride;
    const float4 *vrec = rec + (int64_t)v * S * 3;
    const float lim = -0.5f * cam.cut * cam.cut;

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    bool done = !inside;
    for (int b = r.x; b < r.y; b += NT) {
        if (__syncthreads_count(done) == NT) break;
        const int j = b + (int)threadIdx.x;
        if (j < r.y) {
            const float4 *p = vrec + 3 * (int64_t)list[j];
            s_a[threadIdx.x] = p[0];
            s_b[threadIdx.x] = p[1];
            s_c[threadIdx.x] = p[2];
        }
        __syncthreads();
        const int cnt = min(NT, r.y - b);
        if (!done) {
            for (int k = 0; k < cnt; ++k) {
                const float4 a = s_a[k];
                const float4 cb = s_b[k];
                const float dx = fxp - a.x, dy = fyp - a.y;
                const float power = -0.5f * (cb.x * dx * dx + cb.z * dy * dy) - cb.y * dx * dy;
                if (power < lim) continue;
                const float al = fminf(cam.alpha_max, a.w * __expf(power));
                if (al < cam.alpha_min) continue;
                const float tn = T * (1.f - al);
                if (tn < cam.t_min) { done = true; break; }
                const float w = al * T;
                const float4 c = s_c[k];
                C0 += c.x * w;
                C1 += c.y * w;
                C2 += c.z * w;
                D += a.z * w;
                T = tn;
            }
        }
        __syncthreads();
    }

    const int64_t HW = (int64_t)cam.width * cam.height;
    const int64_t pix = (int64_t)py * cam.width + px;
    if (inside) {
        if (rgb) {
            float *o = rgb + (int64_t)out_v * 3 * HW;
            o[pix] = C0;
            o[HW + pix] = C1;
            o[2 * HW + pix] = C2;
        }
        if (depth) depth[(int64_t)out_v * HW + pix] = D;
        if (alpha) alpha[(int64_t)out_v * HW + pix] = 1.f - T;
    }
    if (partials) {
        float sr = C0 + C1 + C2;
        float srr = C0 * C0 + C1 * C1 + C2 * C2;
        float srq = 0.f;
        if (inside) srq = C0 * __ldg(query + pix) + C1 * __ldg(query + HW + pix) + C2 * __ldg(query + 2 * HW + pix);
        sr = warp_sum_f(sr);
        srr = warp_sum_f(srr);
        srq = warp_sum_f(srq);
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) { s_red[0][w] = sr; s_red[1][w] = srr; s_red[2][w] = srq; }
        __syncthreads();
        if (threadIdx.x < 3) {
            double acc = 0;
#pragma unroll
            for (int k = 0; k < NW; ++k) acc += s_red[threadIdx.x][k];
            partials[((int64_t)blockIdx.y * cam.n_tiles + tile) * 3 + threadIdx.x] = acc;
        }
    }
}

template <int TW, int TH>
static cudaError_t blend_t(const float4 *rec, int64_t S, const uint32_t *inst_gauss, int64_t inst_stride,
                           const int2 *ranges, int V, const CamParams &cam, const float *query, double *partials,
                           float *rgb, float *depth, float *alpha, const int *view_sel, const int *overflow,
                           cudaStream_t st)
{
    dim3 grid(cam.n_tiles, view_sel ? 1 : V);
    k_blend<TW, TH><<<grid, TW * TH, 0, st>>>(rec, S, inst_gauss, inst_stride, ranges, cam, query, partials, rgb,
                                              depth, alpha, view_sel, overflow);
    return cudaGetLastError();
}

cudaError_t launch_blend(const float4 *rec, int64_t S, const uint32_t *inst_gauss, int64_t inst_stride,
                         const int2 *ranges, int V, const CamParams &cam, const float *query, double *partials,
                         float *rgb, float *depth, float *alpha, const int *view_sel, const int *overflow,
                         cudaStream_t st)
{
#define RELOC_BLEND_CASE(W_, H_)                                                                                 \
    if (cam.tile_w == W_ && cam.tile_h == H_)                                                                   \
        return blend_t<W_, H_>(rec, S, inst_gauss, inst_stride, ranges, V, cam, query, partials, rgb, depth, alpha, \
                               view_sel, overflow, st);
    RELOC_BLEND_CASE(16, 16)
    RELOC_BLEND_CASE(8, 8)
    RELOC_BLEND_CASE(32, 8)
    RELOC_BLEND_CASE(16, 8)
    RELOC_BLEND_CASE(8, 16)
    RELOC_BLEND_CASE(32, 16)
#undef RELOC_BLEND_CASE
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ K7 -----
// NCC = (S_rq - S_r S_q / n) / sqrt((S_rr - S_r^2 / n)(S_qq - S_q^2 / n)),
// the one-pass form of Eq. ncc, summed in FP64 in a fixed order.

constexpr int NCC_THREADS = 256;

__global__ void __launch_bounds__(NCC_THREADS)
k_ncc_finalize(const double *__restrict__ partials, const double *__restrict__ qstats, int n_tiles, int64_t n,
               double *__restrict__ scores, int *__restrict__ degenerate)
{
    __shared__ double s[3][NCC_THREADS / 32];
    const int v = blockIdx.x;
    const double *p = partials + (int64_t)v * n_tiles * 3;
    double a = 0, b = 0, c = 0;
    for (int t = threadIdx.x; t < n_tiles; t += NCC_THREADS) {
        a += p[3 * t];
        b += p[3 * t + 1];
        c += p[3 * t + 2];
    }
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    c = warp_sum_d(c);
    if ((threadIdx.x & 31) == 0) { s[0][threadIdx.x >> 5] = a; s[1][threadIdx.x >> 5] = b; s[2][threadIdx.x >> 5] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double Sr = 0, Srr = 0, Srq = 0;
        for (int w = 0; w < NCC_THREADS / 32; ++w) { Sr += s[0][w]; Srr += s[1][w]; Srq += s[2][w]; }
        const double nn = (double)n;
        const double Sq = qstats[0], Sqq = qstats[1];
        const double cov = Srq - Sr * Sq / nn;
        const double vr = Srr - Sr * Sr / nn;
        const double vq = Sqq - Sq * Sq / nn;
        const bool dg = !(vr > 1e-12 * nn) || !(vq > 1e-12 * nn);
        scores[v] = dg ? 0.0 : cov / (sqrt(vr) * sqrt(vq));
        if (degenerate) degenerate[v] = dg ? 1 : 0;
    }
}

cudaError_t launch_ncc_finalize(const double *partials, const double *qstats, int V, int n_tiles, int64_t n_samples,
                                double *scores, int *degenerate, cudaStream_t st)
{
    k_ncc_finalize<<<V, NCC_THREADS, 0, st>>>(partials, qstats, n_tiles, n_samples, scores, degenerate);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ K8 -----

__device__ __forceinline__ bool better(double sa, int ia, double sb, int ib)
{
    return sa > sb || (sa == sb && ia < ib);
}

__global__ void __launch_bounds__(256) k_argmax(const double *__restrict__ scores, int V, int *best, double *best_score)
{
    __shared__ double s_s[256];
    __shared__ int s_i[256];
    double bs = -INFINITY;
    int bi = 0x7fffffff;
    for (int v = threadIdx.x; v < V; v += 256)
        if (better(scores[v], v, bs, bi)) { bs = scores[v]; bi = v; }
    s_s[threadIdx.x] = bs;
    s_i[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o && better(s_s[threadIdx.x + o], s_i[threadIdx.x + o], s_s[threadIdx.x], s_i[threadIdx.x])) {
            s_s[threadIdx.x] = s_s[threadIdx.x + o];
            s_i[threadIdx.x] = s_i[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        best[0] = s_i[0] < V ? s_i[0] : 0;
        best_score[0] = s_s[0];
    }
}

cudaError_t launch_argmax(const double *scores, int V, int *best, double *best_score, cudaStream_t st)
{
    k_argmax<<<1, 256, 0, st>>>(scores, V, best, best_score);
    return cudaGetLastError();
}

}  // namespace reloc
