// cnn.cu -- elementwise and layout kernels of the learned candidate proposal
// (the dense contractions run in gemm.cu).
//
// The proposal network ranks the candidates of the relocalization grid from a
// low-resolution view of the query and of the coarse-pose render, so that only
// the most likely candidates are rendered and scored (the full sweep of
// Sec. III-C.1 stays as the fallback).  Activations are NHWC BF16; every
// convolution is 3x3, stride 2, padding 1, lowered to a GEMM by im2col with
// column index k = (ky * 3 + kx) * C_in + c_in (zero-padded to a multiple of 64).
#include "internal.cuh"

namespace reloc {

// 8x box average of the RGB mean (gray) of a planar [3][H][W] image into
// channel `ch` of an NHWC [Ho][Wo][2] BF16 input, Ho = H / f, Wo = W / f.
__global__ void k_downsample_gray(const float *__restrict__ img, int H, int W, int f, int ch,
                                  __nv_bfloat16 *__restrict__ out)
{
    const int Ho = H / f, Wo = W / f;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ho * Wo) return;
    const int oy = i / Wo, ox = i % Wo;
    const int64_t HW = (int64_t)H * W;
    float s = 0.f;
    for (int y = oy * f; y < oy * f + f; ++y)
        for (int x = ox * f; x < ox * f + f; ++x) {
            const int64_t p = (int64_t)y * W + x;
            s += img[p] + img[HW + p] + img[2 * HW + p];
        }
    out[(int64_t)i * 2 + ch] = __float2bfloat16_rn(s / (3.f * f * f));
}

cudaError_t launch_downsample_gray(const float *img, int H, int W, int f, int ch, __nv_bfloat16 *out, cudaStream_t st)
{
    const int n = (H / f) * (W / f);
    k_downsample_gray<<<(n + 255) / 256, 256, 0, st>>>(img, H, W, f, ch, out);
    return cudaGetLastError();
}

// im2col for a 3x3 / stride 2 / pad 1 convolution: X [B][H][W][C] ->
// col [B*Ho*Wo][Kp], zero beyond K = 9 C.
__global__ void k_im2col(const __nv_bfloat16 *__restrict__ x, int B, int H, int W, int C, int Ho, int Wo, int Kp,
                         __nv_bfloat16 *__restrict__ col)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)B * Ho * Wo * Kp;
    if (i >= total) return;
    const int k = (int)(i % Kp);
    const int64_t row = i / Kp;
    const int ox = (int)(row % Wo), oy = (int)((row / Wo) % Ho), b = (int)(row / ((int64_t)Wo * Ho));
    __nv_bfloat16 v = __float2bfloat16_rn(0.f);
    if (k < 9 * C) {
        const int ci = k % C, kk = k / C, ky = kk / 3, kx = kk % 3;
        const int y = 2 * oy - 1 + ky, xx = 2 * ox - 1 + kx;
        if (y >= 0 && y < H && xx >= 0 && xx < W) v = x[(((int64_t)b * H + y) * W + xx) * C + ci];
    }
    col[i] = v;
}

cudaError_t launch_im2col(const __nv_bfloat16 *x, int B, int H, int W, int C, int Ho, int Wo, int Kp,
                          __nv_bfloat16 *col, cudaStream_t st)
{
    const int64_t n = (int64_t)B * Ho * Wo * Kp;
    k_im2col<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(x, B, H, W, C, Ho, Wo, Kp, col);
    return cudaGetLastError();
}

// col2im (gather form, fixed summation order): dX[b][y][x][c] = sum over the
// (ky, kx) whose output position (oy, ox) with y = 2 oy - 1 + ky,
// x = 2 ox - 1 + kx lies in the output, of dcol[(b, oy, ox)][(ky, kx, c)].
__global__ void k_col2im(const float *__restrict__ dcol, int B, int H, int W, int C, int Ho, int Wo, int Kp,
                         __nv_bfloat16 *__restrict__ dx_bf, float *__restrict__ dx_f)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)B * H * W * C;
    if (i >= total) return;
    const int c = (int)(i % C);
    const int64_t p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H), b = (int)(p / ((int64_t)W * H));
    float s = 0.f;
    for (int ky = 0; ky < 3; ++ky) {
        const int ty = y + 1 - ky;
        if (ty < 0 || (ty & 1)) continue;
        const int oy = ty >> 1;
        if (oy >= Ho) continue;
        for (int kx = 0; kx < 3; ++kx) {
            const int tx = x + 1 - kx;
            if (tx < 0 || (tx & 1)) continue;
            const int ox = tx >> 1;
            if (ox >= Wo) continue;
            s += dcol[(((int64_t)b * Ho + oy) * Wo + ox) * Kp + (ky * 3 + kx) * C + c];
        }
    }
    if (dx_bf) dx_bf[i] = __float2bfloat16_rn(s);
    if (dx_f) dx_f[i] = s;
}

cudaError_t launch_col2im(const float *dcol, int B, int H, int W, int C, int Ho, int Wo, int Kp, __nv_bfloat16 *dx_bf,
                          float *dx_f, cudaStream_t st)
{
    const int64_t n = (int64_t)B * H * W * C;
    k_col2im<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(dcol, B, H, W, C, Ho, Wo, Kp, dx_bf, dx_f);
    return cudaGetLastError();
}

// out[c][r] = in[r][c] for r < R, c < Cc; out is Cp rows of Rp values (zero
// padding, Rp >= R, Cp >= Cc) with row stride ldo >= Rp.  in: BF16 or FP32
// (converted).
template <typename T>
__global__ void k_transpose(const T *__restrict__ in, int R, int Cc, int ld_in, __nv_bfloat16 *__restrict__ out, int Rp,
                            int Cp, int ldo)
{
    __shared__ float t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        float v = 0.f;
        if (r < R && c < Cc) v = (float)in[(int64_t)r * ld_in + c];
        t[j][threadIdx.x] = v;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int c = c0 + j, r = r0 + threadIdx.x;
        if (c < Cp && r < Rp) out[(int64_t)c * ldo + r] = __float2bfloat16_rn(t[threadIdx.x][j]);
    }
}

cudaError_t launch_transpose_bf16(const __nv_bfloat16 *in, int R, int Cc, int ld_in, __nv_bfloat16 *out, int Rp, int Cp,
                                  cudaStream_t st, int ldo)
{
    dim3 grid((unsigned)ceil_div(Cp, 32), (unsigned)ceil_div(Rp, 32));
    k_transpose<__nv_bfloat16><<<grid, dim3(32, 8), 0, st>>>(in, R, Cc, ld_in, out, Rp, Cp, ldo > 0 ? ldo : Rp);
    return cudaGetLastError();
}

cudaError_t launch_transpose_f32(const float *in, int R, int Cc, int ld_in, __nv_bfloat16 *out, int Rp, int Cp,
                                 cudaStream_t st)
{
    dim3 grid((unsigned)ceil_div(Cp, 32), (unsigned)ceil_div(Rp, 32));
    k_transpose<float><<<grid, dim3(32, 8), 0, st>>>(in, R, Cc, ld_in, out, Rp, Cp, Rp);
    return cudaGetLastError();
}

// d (FP32) *= (y > 0), written as BF16 (the gradient through a ReLU).
// A backward signal carried as two BF16 terms: out [M][2N] holds hi =
// bf16(x) in columns 0..N-1 and lo = bf16(x - hi) in N..2N-1, so hi + lo
// keeps ~16 significant bits of x and the GEMMs that contract it (over 2N
// columns, or 2M rows stacked) accumulate both in FP32.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// ReLU backward of d [M][N] at the stored activations y, split into hi | lo.
__global__ void k_relu_back(const float *__restrict__ d, const __nv_bfloat16 *__restrict__ y, int64_t M, int N,
                            __nv_bfloat16 *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * N) return;
    const int64_t r = i / N;
    const int c = (int)(i - r * N);
    __nv_bfloat16 hi, lo;
    split_bf16((float)y[i] > 0.f ? d[i] : 0.f, hi, lo);
    out[r * 2 * N + c] = hi;
    out[r * 2 * N + N + c] = lo;
}

cudaError_t launch_relu_back(const float *d, const __nv_bfloat16 *y, int64_t M, int N, __nv_bfloat16 *out,
                             cudaStream_t st)
{
    const int64_t n = M * N;
    k_relu_back<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(d, y, M, N, out);
    return cudaGetLastError();
}

// db[c] = sum over the R rows of the split signal d [R][2 Cc] (hi + lo), FP32.
__global__ void k_colsum(const __nv_bfloat16 *__restrict__ d, int R, int Cc, float *__restrict__ db)
{
    __shared__ float s[256];
    const int c = blockIdx.x;
    float a = 0.f;
    for (int r = threadIdx.x; r < R; r += 256)
        a += (float)d[(int64_t)r * 2 * Cc + c] + (float)d[(int64_t)r * 2 * Cc + Cc + c];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = s[0];
}

cudaError_t launch_colsum(const __nv_bfloat16 *d, int R, int Cc, float *db, cudaStream_t st)
{
    k_colsum<<<Cc, 256, 0, st>>>(d, R, Cc, db);
    return cudaGetLastError();
}

// Softmax cross-entropy rows: loss_rows[b], dl = (softmax - onehot) / B in
// FP32 and split into hi | lo BF16 terms (dlb [B][2C]).
__global__ void k_softmax_ce(const float *__restrict__ logits, const int32_t *__restrict__ labels, int B, int C,
                             float *__restrict__ loss_rows, float *__restrict__ dl, __nv_bfloat16 *__restrict__ dlb)
{
    const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    const float *z = logits + (int64_t)b * C;
    float mx = -INFINITY;
    for (int c = lane; c < C; c += 32) mx = fmaxf(mx, z[c]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float se = 0.f;
    for (int c = lane; c < C; c += 32) se += expf(z[c] - mx);
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    const int y = labels[b];
    for (int c = lane; c < C; c += 32) {
        const float p = expf(z[c] - mx) / se;
        const float g = (p - (c == y ? 1.f : 0.f)) / (float)B;
        dl[(int64_t)b * C + c] = g;
        split_bf16(g, dlb[(int64_t)b * 2 * C + c], dlb[(int64_t)b * 2 * C + C + c]);
    }
    if (lane == 0) loss_rows[b] = logf(se) + mx - z[y];
}

cudaError_t launch_softmax_ce(const float *logits, const int32_t *labels, int B, int C, float *loss_rows, float *dl,
                              __nv_bfloat16 *dlb, cudaStream_t st)
{
    k_softmax_ce<<<(unsigned)ceil_div(B, 8), 256, 0, st>>>(logits, labels, B, C, loss_rows, dl, dlb);
    return cudaGetLastError();
}

// Adam (Kingma and Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  Also refreshes
// the BF16 copy of the weight (w_bf may be null for biases).
__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16 *__restrict__ w_bf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (w_bf) w_bf[i] = __float2bfloat16_rn(wi);
}

cudaError_t launch_adam(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2, float eps,
                        float c1, float c2, __nv_bfloat16 *w_bf, cudaStream_t st)
{
    k_adam<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(w, m, v, g, n, lr, b1, b2, eps, c1, c2, w_bf);
    return cudaGetLastError();
}

// FP32 -> BF16 copy.
__global__ void k_to_bf16(const float *__restrict__ a, int64_t n, __nv_bfloat16 *__restrict__ b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

cudaError_t launch_to_bf16(const float *a, int64_t n, __nv_bfloat16 *b, cudaStream_t st)
{
    k_to_bf16<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(a, n, b);
    return cudaGetLastError();
}

// Top-k of each row of C logits (k <= 32), descending, ties by lower index;
// also the softmax margin p1 - p2.  One warp per row.
__global__ void k_topk(const float *__restrict__ logits, int B, int C, int k, int32_t *__restrict__ idx,
                       float *__restrict__ margin)
{
    const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    const float *z = logits + (int64_t)b * C;
    float mx = -INFINITY;
    for (int c = lane; c < C; c += 32) mx = fmaxf(mx, z[c]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float se = 0.f;
    for (int c = lane; c < C; c += 32) se += expf(z[c] - mx);
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    uint32_t taken[4] = {0, 0, 0, 0};     // up to 128 classes
    float p1 = 0.f, p2 = 0.f;
    for (int r = 0; r < k; ++r) {
        float best = -INFINITY;
        int bi = 0x7fffffff;
        for (int c = lane; c < C; c += 32)
            if (!((taken[c >> 5] >> (c & 31)) & 1u) && (z[c] > best || (z[c] == best && c < bi))) { best = z[c]; bi = c; }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (bi >= C) break;
        taken[bi >> 5] |= 1u << (bi & 31);
        if (lane == 0) idx[(int64_t)b * k + r] = bi;
        if (r == 0) p1 = expf(best - mx) / se;
        if (r == 1) p2 = expf(best - mx) / se;
    }
    if (lane == 0) margin[b] = p1 - p2;
}

cudaError_t launch_topk(const float *logits, int B, int C, int k, int32_t *idx, float *margin, cudaStream_t st)
{
    if (C > 128 || k > 32 || k < 2) return cudaErrorInvalidValue;
    k_topk<<<(unsigned)ceil_div(B, 8), 256, 0, st>>>(logits, B, C, k, idx, margin);
    return cudaGetLastError();
}

}  // namespace reloc
