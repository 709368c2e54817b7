// train.cu -- map training (Sec. III-B.3): the image loss and its gradient per
// pixel, the chain rule from per-(view, Gaussian) screen-space gradients to the
// Gaussians' parameters, and the Adam step on the map.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace reloc {

// ------------------------------------------------------------------ L1 -----
// L1 part of L_rgb (Eq. 3) over n samples: loss += scale * sum |C - I| and
// dL/dC = scale * sign(C - I) (sign(0) = +1, the right derivative), written
// or added (accumulate) to gimg.  One FP64 atomic per block.
__global__ void __launch_bounds__(256)
k_photo_l1(const float *__restrict__ rgb, const float *__restrict__ target, int64_t n, float scale, double dscale,
           float *__restrict__ gimg, int accumulate, double *__restrict__ loss)
{
    __shared__ double s_red[8];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const float d = rgb[i] - target[i];
        acc += (double)fabsf(d);
        const float g = d >= 0.f ? scale : -scale;
        gimg[i] = accumulate ? gimg[i] + g : g;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += s_red[w];
        atomicAdd(loss, s * dscale);
    }
}

cudaError_t launch_photo_l1(const float *rgb, const float *target, int64_t n, double scale, float *gimg,
                            bool accumulate, double *loss, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>(ceil_div(n, 256 * 8), 152 * 16);
    k_photo_l1<<<(int)blocks, 256, 0, st>>>(rgb, target, n, (float)scale, scale, gimg, accumulate ? 1 : 0, loss);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- D-SSIM --
// D-SSIM term of L_rgb (Eq. 3): SSIM of Wang, Bovik, Sheikh and Simoncelli
// (2004) per channel plane, with local statistics under an 11 x 11 Gaussian
// window (standard deviation 1.5 px, unit sum; separable, so two 11-tap
// passes) and samples outside the image counting as 0; C1 = 0.01^2, C2 =
// 0.03^2.  The loss adds scale * sum over pixels of (1 - SSIM).  A 256-thread
// block covers a 32 x 32 tile of one plane; its inputs with a 5-pixel halo
// sit in shared memory, and each thread slides the window over four
// neighbouring outputs from registers (14 loads per source for 4 outputs)
// in both passes.
constexpr int SS_T = 32, SS_R = 5, SS_N = 2 * SS_R + 1, SS_H = SS_T + 2 * SS_R;
constexpr int SS_THREADS = 256, SS_OUT = 4, SS_WIN = SS_OUT + 2 * SS_R;
constexpr int SS_IN_STRIDE = 45;     // input rows: 8 lanes at stride 4 per row, rows 45 apart: no bank conflict
constexpr int SS_H_STRIDE = 33;      // pass-1 rows: (row + column) spreads the lanes over the banks
constexpr float SS_C1 = 0.01f * 0.01f, SS_C2 = 0.03f * 0.03f;

struct SsimWin {
    float w[SS_N];   // one-dimensional factor of the window (sums to 1)
};

static SsimWin ssim_window()
{
    double g[SS_N], s = 0.0;
    for (int k = 0; k < SS_N; ++k) {
        const double d = k - SS_R;
        g[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    SsimWin w;
    for (int k = 0; k < SS_N; ++k) w.w[k] = (float)(g[k] / s);
    return w;
}

// Load a (SS_H x SS_H) halo tile of NQ planes (src[m] + plane offset) into
// dst[m][row * SS_IN_STRIDE + col], 0 outside the image.
template <int NQ>
__device__ __forceinline__ void ssim_load(float (*dst)[SS_H * SS_IN_STRIDE], const float *const (&src)[NQ], int H,
                                          int W, int x0, int y0)
{
    // every load of the thread first (all in flight together), then the stores
    constexpr int PER = (SS_H * SS_H + SS_THREADS - 1) / SS_THREADS;
    float v[PER][NQ];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int k = u * SS_THREADS + threadIdx.x;
        const int r = k / SS_H, c = k - r * SS_H;
        const int gy = y0 + r - SS_R, gx = x0 + c - SS_R;
        const bool in = k < SS_H * SS_H && gy >= 0 && gy < H && gx >= 0 && gx < W;
#pragma unroll
        for (int m = 0; m < NQ; ++m) v[u][m] = in ? src[m][(int64_t)gy * W + gx] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int k = u * SS_THREADS + threadIdx.x;
        if (k < SS_H * SS_H) {
            const int r = k / SS_H, c = k - r * SS_H;
#pragma unroll
            for (int m = 0; m < NQ; ++m) dst[m][r * SS_IN_STRIDE + c] = v[u][m];
        }
    }
}

// Forward: per pixel SSIM s and, with dL/ds = -scale, the products of dL/ds
// with the partial derivatives of s with respect to the local mean of x, the
// local mean of x^2 and the local mean of x y (A1 = 2 mx my + C1, A2 = 2 sxy +
// C2, B1 = mx^2 + my^2 + C1, B2 = sx^2 + sy^2 + C2, s = A1 A2 / (B1 B2)):
//   ds/dmx   = (2 my (A2 - A1) - 2 mx s (B2 - B1)) / (B1 B2)
//   ds/dE[xx] = -s / B2,  ds/dE[xy] = 2 A1 / (B1 B2),
// into abc [plane][3][H][W].
__global__ void __launch_bounds__(SS_THREADS)
k_ssim_fwd(const float *__restrict__ x_img, const float *__restrict__ y_img, int H, int W, SsimWin win,
           float scale, double dscale, float *__restrict__ abc, double *__restrict__ loss)
{
    __shared__ float sin_[2][SS_H * SS_IN_STRIDE];
    __shared__ float hsum[5][SS_H * SS_H_STRIDE];
    __shared__ double s_red[SS_THREADS / 32];
    const int64_t HW = (int64_t)H * W;
    const int plane = blockIdx.z;
    const int x0 = blockIdx.x * SS_T, y0 = blockIdx.y * SS_T;
    const float *const src[2] = {x_img + plane * HW, y_img + plane * HW};
    ssim_load<2>(sin_, src, H, W, x0, y0);
    __syncthreads();
    // pass 1 (along x): item = (row, group of 4 output columns)
    for (int it = threadIdx.x; it < SS_H * (SS_T / SS_OUT); it += SS_THREADS) {
        const int r = it / (SS_T / SS_OUT), c0 = (it - r * (SS_T / SS_OUT)) * SS_OUT;
        float a[SS_WIN], b[SS_WIN];
#pragma unroll
        for (int i = 0; i < SS_WIN; ++i) {
            a[i] = sin_[0][r * SS_IN_STRIDE + c0 + i];
            b[i] = sin_[1][r * SS_IN_STRIDE + c0 + i];
        }
#pragma unroll
        for (int o = 0; o < SS_OUT; ++o) {
            float m1 = 0.f, m2 = 0.f, e11 = 0.f, e22 = 0.f, e12 = 0.f;
#pragma unroll
            for (int t = 0; t < SS_N; ++t) {
                const float w = win.w[t], xa = a[o + t], yb = b[o + t];
                const float wx = w * xa, wy = w * yb;
                m1 += wx;
                m2 += wy;
                e11 = fmaf(wx, xa, e11);
                e22 = fmaf(wy, yb, e22);
                e12 = fmaf(wx, yb, e12);
            }
            const int h = r * SS_H_STRIDE + c0 + o;
            hsum[0][h] = m1; hsum[1][h] = m2; hsum[2][h] = e11; hsum[3][h] = e22; hsum[4][h] = e12;
        }
    }
    __syncthreads();
    // pass 2 (along y): thread = (column, group of 4 output rows)
    const int col = threadIdx.x % SS_T, r0 = (threadIdx.x / SS_T) * SS_OUT;
    float q[5][SS_OUT];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        float v[SS_WIN];
#pragma unroll
        for (int i = 0; i < SS_WIN; ++i) v[i] = hsum[m][(r0 + i) * SS_H_STRIDE + col];
#pragma unroll
        for (int o = 0; o < SS_OUT; ++o) {
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t < SS_N; ++t) acc = fmaf(win.w[t], v[o + t], acc);
            q[m][o] = acc;
        }
    }
    double contrib = 0.0;
    const int gx = x0 + col;
#pragma unroll
    for (int o = 0; o < SS_OUT; ++o) {
        const int gy = y0 + r0 + o;
        if (gx < W && gy < H) {
            const float mx = q[0][o], my = q[1][o];
            const float vx = q[2][o] - mx * mx, vy = q[3][o] - my * my, cxy = q[4][o] - mx * my;
            const float A1 = 2.f * mx * my + SS_C1, A2 = 2.f * cxy + SS_C2;
            const float B1 = mx * mx + my * my + SS_C1, B2 = vx + vy + SS_C2;
            const float iB = 1.f / (B1 * B2);
            const float s = A1 * A2 * iB;
            const float d_m = (2.f * my * (A2 - A1) - 2.f * mx * s * (B2 - B1)) * iB;
            const float d_xx = -s / B2, d_xy = 2.f * A1 * iB;
            float *po = abc + (int64_t)plane * 3 * HW + (int64_t)gy * W + gx;
            po[0] = -scale * d_m;
            po[HW] = -scale * d_xx;
            po[2 * HW] = -scale * d_xy;
            contrib += 1.0 - (double)s;
        }
    }
    for (int off = 16; off > 0; off >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = contrib;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < SS_THREADS / 32; ++w) t += s_red[w];
        atomicAdd(loss, t * dscale);
    }
}

// Backward: dL/dx(q) = sum_p w(p - q) (a(p) + 2 x(q) b(p) + y(q) c(p)) over
// the image's pixels p (the window is symmetric, so the same separable
// passes), added to gimg.
__global__ void __launch_bounds__(SS_THREADS)
k_ssim_bwd(const float *__restrict__ abc, const float *__restrict__ x_img, const float *__restrict__ y_img, int H,
           int W, SsimWin win, float *__restrict__ gimg)
{
    __shared__ float sin_[3][SS_H * SS_IN_STRIDE];
    __shared__ float hsum[3][SS_H * SS_H_STRIDE];
    const int64_t HW = (int64_t)H * W;
    const int plane = blockIdx.z;
    const int x0 = blockIdx.x * SS_T, y0 = blockIdx.y * SS_T;
    const float *P = abc + (int64_t)plane * 3 * HW;
    const float *const src[3] = {P, P + HW, P + 2 * HW};
    ssim_load<3>(sin_, src, H, W, x0, y0);
    __syncthreads();
    for (int it = threadIdx.x; it < SS_H * (SS_T / SS_OUT); it += SS_THREADS) {
        const int r = it / (SS_T / SS_OUT), c0 = (it - r * (SS_T / SS_OUT)) * SS_OUT;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            float a[SS_WIN];
#pragma unroll
            for (int i = 0; i < SS_WIN; ++i) a[i] = sin_[m][r * SS_IN_STRIDE + c0 + i];
#pragma unroll
            for (int o = 0; o < SS_OUT; ++o) {
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < SS_N; ++t) acc = fmaf(win.w[t], a[o + t], acc);
                hsum[m][r * SS_H_STRIDE + c0 + o] = acc;
            }
        }
    }
    __syncthreads();
    const int col = threadIdx.x % SS_T, r0 = (threadIdx.x / SS_T) * SS_OUT;
    float q[3][SS_OUT];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        float v[SS_WIN];
#pragma unroll
        for (int i = 0; i < SS_WIN; ++i) v[i] = hsum[m][(r0 + i) * SS_H_STRIDE + col];
#pragma unroll
        for (int o = 0; o < SS_OUT; ++o) {
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t < SS_N; ++t) acc = fmaf(win.w[t], v[o + t], acc);
            q[m][o] = acc;
        }
    }
    const int gx = x0 + col;
#pragma unroll
    for (int o = 0; o < SS_OUT; ++o) {
        const int gy = y0 + r0 + o;
        if (gx < W && gy < H) {
            const int64_t pix = plane * HW + (int64_t)gy * W + gx;
            gimg[pix] += q[0][o] + 2.f * x_img[pix] * q[1][o] + y_img[pix] * q[2][o];
        }
    }
}

cudaError_t launch_ssim(const float *rgb, const float *target, int planes, int H, int W, double scale, float *abc,
                        float *gimg, double *loss, cudaStream_t st)
{
    if (planes <= 0) return cudaSuccess;
    const SsimWin win = ssim_window();
    dim3 grid((unsigned)ceil_div(W, SS_T), (unsigned)ceil_div(H, SS_T), (unsigned)planes);
    k_ssim_fwd<<<grid, SS_THREADS, 0, st>>>(rgb, target, H, W, win, (float)scale, scale, abc, loss);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ssim_bwd<<<grid, SS_THREADS, 0, st>>>(abc, rgb, target, H, W, win, gimg);
    return cudaGetLastError();
}

// ----------------------------------------------------------- re-projection --
// The P of Eq. 5 for the consecutive training views (t, t+1): a pixel p of
// view t whose rendered alpha A reaches alpha_min takes the depth d = D / A,
// is lifted to d * ray(p) (ray = ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1))
// and carried into view t+1 by the relative pose (rel[12] = R_rel row-major,
// t_rel: P = R_rel d ray + t_rel); in front of the near plane, with the four
// bilinear neighbours of q = (fx P_x / P_z + cx, fy P_y / P_z + cy) (pixel
// centres at +0.5) inside the image, the re-projected image takes I_{t+1}
// sampled there and jac the derivative of that sample with respect to d;
// otherwise it keeps I_t(p) and jac = 0.  A thread per pixel.
__global__ void __launch_bounds__(256)
k_reproj_warp(const float *__restrict__ dep, const float *__restrict__ alp, const float *__restrict__ targets,
              const float *__restrict__ rel, int n_views, int H, int W, float fx, float fy, float cx, float cy,
              float near_plane, float alpha_min, float *__restrict__ warped, float *__restrict__ jac)
{
    const int64_t HW = (int64_t)H * W;
    const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (idx >= (int64_t)n_views * HW) return;
    const int v = (int)(idx / HW);
    const int64_t pix = idx - (int64_t)v * HW;
    const int py = (int)(pix / W), px = (int)(pix - (int64_t)py * W);
    const float *It = targets + (int64_t)v * 3 * HW, *In = It + 3 * HW;
    float *wo = warped + (int64_t)v * 3 * HW + pix, *jo = jac + (int64_t)v * 3 * HW + pix;
    const float A = alp[idx];
    bool ok = A >= alpha_min;
    float out[3] = {It[pix], It[HW + pix], It[2 * HW + pix]}, dj[3] = {0.f, 0.f, 0.f};
    if (ok) {
        const float d = dep[idx] / A;
        const float r0 = ((float)px + 0.5f - cx) / fx, r1 = ((float)py + 0.5f - cy) / fy;
        const float *M = rel + 12 * v;
        const float m0 = M[0] * r0 + M[1] * r1 + M[2], m1 = M[3] * r0 + M[4] * r1 + M[5];
        const float m2 = M[6] * r0 + M[7] * r1 + M[8];
        const float P0 = fmaf(d, m0, M[9]), P1 = fmaf(d, m1, M[10]), P2 = fmaf(d, m2, M[11]);
        ok = P2 > near_plane;
        if (ok) {
            const float iz = 1.f / P2;
            const float sx = fx * P0 * iz + (cx - 0.5f), sy = fy * P1 * iz + (cy - 0.5f);
            const float x0 = floorf(sx), y0 = floorf(sy);
            ok = x0 >= 0.f && x0 <= (float)(W - 2) && y0 >= 0.f && y0 <= (float)(H - 2);
            if (ok) {
                const float ax = sx - x0, ay = sy - y0;
                const float dsx = fx * (m0 * P2 - P0 * m2) * iz * iz, dsy = fy * (m1 * P2 - P1 * m2) * iz * iz;
                const int64_t k00 = (int64_t)y0 * W + (int64_t)x0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float *I = In + c * HW;
                    const float i00 = I[k00], i01 = I[k00 + 1], i10 = I[k00 + W], i11 = I[k00 + W + 1];
                    out[c] = (1.f - ax) * (1.f - ay) * i00 + ax * (1.f - ay) * i01 + (1.f - ax) * ay * i10 +
                             ax * ay * i11;
                    const float gx = (1.f - ay) * (i01 - i00) + ay * (i11 - i10);
                    const float gy = (1.f - ax) * (i10 - i00) + ax * (i11 - i01);
                    dj[c] = gx * dsx + gy * dsy;
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        wo[c * HW] = out[c];
        jo[c * HW] = dj[c];
    }
}

// dL/dD = g_d / A and dL/dA = -g_d D / A^2 with g_d = sum_c dL/dwarped_c *
// jac_c (d = D / A), into gda [v][2][H][W]; 0 where the pixel had no sample.
__global__ void __launch_bounds__(256)
k_reproj_back(const float *__restrict__ gw, const float *__restrict__ jac, const float *__restrict__ dep,
              const float *__restrict__ alp, int n_views, int64_t HW, float alpha_min, float *__restrict__ gda)
{
    const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (idx >= (int64_t)n_views * HW) return;
    const int v = (int)(idx / HW);
    const int64_t pix = idx - (int64_t)v * HW;
    const float *g = gw + (int64_t)v * 3 * HW + pix, *j = jac + (int64_t)v * 3 * HW + pix;
    const float gd = g[0] * j[0] + g[HW] * j[HW] + g[2 * HW] * j[2 * HW];
    const float A = alp[idx];
    float gD = 0.f, gA = 0.f;
    if (A >= alpha_min && gd != 0.f) {
        gD = gd / A;
        gA = -gd * dep[idx] / (A * A);
    }
    gda[(int64_t)v * 2 * HW + pix] = gD;
    gda[(int64_t)v * 2 * HW + HW + pix] = gA;
}

cudaError_t launch_reproj_warp(const float *dep, const float *alp, const float *targets, const float *rel,
                               int n_views, const CamParams &cam, float alpha_min, float *warped, float *jac,
                               cudaStream_t st)
{
    const int64_t n = (int64_t)n_views * cam.width * cam.height;
    if (n <= 0) return cudaSuccess;
    k_reproj_warp<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(dep, alp, targets, rel, n_views, cam.height, cam.width,
                                                              cam.fx, cam.fy, cam.cx, cam.cy, cam.near_plane,
                                                              alpha_min, warped, jac);
    return cudaGetLastError();
}

cudaError_t launch_reproj_back(const float *gw, const float *jac, const float *dep, const float *alp, int n_views,
                               int64_t HW, float alpha_min, float *gda, cudaStream_t st)
{
    const int64_t n = (int64_t)n_views * HW;
    if (n <= 0) return cudaSuccess;
    k_reproj_back<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(gw, jac, dep, alp, n_views, HW, alpha_min, gda);
    return cudaGetLastError();
}

// --------------------------------------------------------- parameter chain --
// gin holds, per (view, subset Gaussian), the gradients of the loss with
// respect to the projected mean (u, v), the conic (a, b, c), the colour, the
// opacity and the camera depth z = t_z (k_blend_grad, image mode).  A thread per subset Gaussian walks
// its query's views and carries them back through the projection (Sec. III-A:
// Sigma' = J W Sigma W^T J^T + 0.3 I, conic = Sigma'^-1, t = W mu):
//   dL/dSigma' = -A G_A A                       (G_A = [[ga, gb/2], [gb/2, gc]])
//   dL/dSigma += T^T dL/dSigma' T, dL/dT = 2 dL/dSigma' T Sigma    (T = J W)
//   dL/dt from (u, v) and from J(t) (frustum clamp: no term through a clamped
//   coordinate), dL/dmu += W^T dL/dt;
// then once: Sigma = M M^T with M = R(q / |q|) diag(s): dL/dM = 2 dL/dSigma M,
// dL/ds_j = sum_i dL/dM_ij R_ij, dL/dR_ij = dL/dM_ij s_j, through the rotation
// entries to the unit quaternion and across its normalisation
// (g_q = (g_qhat - qhat (qhat . g_qhat)) / |q|).  The 14 sums are added to
// gmap [14][n_map] (mean xyz, scale xyz, quat wxyz, opacity, rgb).
__global__ void __launch_bounds__(PROJ_THREADS)
k_param_chain(const float *__restrict__ mx, const float *__restrict__ my, const float *__restrict__ mz,
              const float *__restrict__ attr, int64_t n_map, const uint32_t *__restrict__ gidx, Layout L,
              const ViewParams *__restrict__ views, CamParams cam, const float *__restrict__ gin,
              float *__restrict__ gmap)
{
    const int qi = find_segment(L.q_pblk, L.Q, (int)blockIdx.x);
    const int64_t S = L.q_gsub[qi + 1] - L.q_gsub[qi];
    const int64_t i = (int64_t)(blockIdx.x - L.q_pblk[qi]) * PROJ_THREADS + threadIdx.x;
    if (i >= S) return;
    const int v_begin = L.q_view[qi], V = L.q_view[qi + 1] - v_begin;
    const int64_t g = gidx[L.q_gsub[qi] + i];
    const float mu0 = __ldg(mx + g), mu1 = __ldg(my + g), mu2 = __ldg(mz + g);
    const float sc[3] = {__ldg(attr + (ATTR_SCALE + 0) * n_map + g), __ldg(attr + (ATTR_SCALE + 1) * n_map + g),
                         __ldg(attr + (ATTR_SCALE + 2) * n_map + g)};
    const float q0 = __ldg(attr + (ATTR_QUAT + 0) * n_map + g), q1 = __ldg(attr + (ATTR_QUAT + 1) * n_map + g);
    const float q2 = __ldg(attr + (ATTR_QUAT + 2) * n_map + g), q3 = __ldg(attr + (ATTR_QUAT + 3) * n_map + g);
    const float qn = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float qw = q0 / qn, qx = q1 / qn, qy = q2 / qn, qz = q3 / qn;
    const float r[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                        2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                        2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    float m[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) m[3 * a + b] = r[3 * a + b] * sc[b];
    float Sm[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Sm[3 * a + b] = m[3 * a] * m[3 * b] + m[3 * a + 1] * m[3 * b + 1] + m[3 * a + 2] * m[3 * b + 2];

    float gmu[3] = {0, 0, 0}, gS[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gcol[3] = {0, 0, 0}, gop = 0.f;
    bool any = false;
    for (int vv = 0; vv < V; ++vv) {
        const int v = v_begin + vv;
        const float *g10 = gin + 10 * (L.vd_off[v] + i);
        const float gu = g10[0], gv = g10[1], ga = g10[2], gb = g10[3], gc = g10[4];
        const float gr = g10[5], gg = g10[6], gbl = g10[7], go = g10[8], gz = g10[9];
        if (gu == 0.f && gv == 0.f && ga == 0.f && gb == 0.f && gc == 0.f && gr == 0.f && gg == 0.f &&
            gbl == 0.f && go == 0.f && gz == 0.f)
            continue;
        any = true;
        gcol[0] += gr; gcol[1] += gg; gcol[2] += gbl;
        gop += go;
        const ViewParams &P = views[v];
        const float d0 = (mu0 - P.c_hi[0]) - P.c_lo[0], d1 = (mu1 - P.c_hi[1]) - P.c_lo[1];
        const float d2 = (mu2 - P.c_hi[2]) - P.c_lo[2];
        const float t[3] = {P.R[0] * d0 + P.R[1] * d1 + P.R[2] * d2, P.R[3] * d0 + P.R[4] * d1 + P.R[5] * d2,
                            P.R[6] * d0 + P.R[7] * d1 + P.R[8] * d2};
        const float iz = 1.f / t[2];
        const float rx = t[0] * iz, ry = t[1] * iz;
        const bool cx_ = rx < -cam.limx || rx > cam.limx, cy_ = ry < -cam.limy || ry > cam.limy;
        const float xz = fminf(fmaxf(rx, -cam.limx), cam.limx), yz = fminf(fmaxf(ry, -cam.limy), cam.limy);
        const float J00 = cam.fx * iz, J02 = -cam.fx * xz * iz, J11 = cam.fy * iz, J12 = -cam.fy * yz * iz;
        float Tm[6];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            Tm[b] = J00 * P.R[b] + J02 * P.R[6 + b];
            Tm[3 + b] = J11 * P.R[3 + b] + J12 * P.R[6 + b];
        }
        float TS[6];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                TS[3 * a + b] = Tm[3 * a] * Sm[b] + Tm[3 * a + 1] * Sm[3 + b] + Tm[3 * a + 2] * Sm[6 + b];
        const float sa = TS[0] * Tm[0] + TS[1] * Tm[1] + TS[2] * Tm[2] + cam.eps2d;
        const float sb = TS[0] * Tm[3] + TS[1] * Tm[4] + TS[2] * Tm[5];
        const float scc = TS[3] * Tm[3] + TS[4] * Tm[4] + TS[5] * Tm[5] + cam.eps2d;
        const float idet = 1.f / (sa * scc - sb * sb);
        const float A00 = scc * idet, A01 = -sb * idet, A11 = sa * idet;
        const float h = 0.5f * gb;
        const float M00 = A00 * ga + A01 * h, M01 = A00 * h + A01 * gc;
        const float M10 = A01 * ga + A11 * h, M11 = A01 * h + A11 * gc;
        const float GS00 = -(M00 * A00 + M01 * A01), GS01 = -(M00 * A01 + M01 * A11);
        const float GS11 = -(M10 * A01 + M11 * A11);
        // dL/dSigma += T^T GS T
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float ua = GS00 * Tm[a] + GS01 * Tm[3 + a], wa = GS01 * Tm[a] + GS11 * Tm[3 + a];
#pragma unroll
            for (int b = 0; b < 3; ++b) gS[3 * a + b] += ua * Tm[b] + wa * Tm[3 + b];
        }
        float dT[6];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            dT[b] = 2.f * (GS00 * TS[b] + GS01 * TS[3 + b]);
            dT[3 + b] = 2.f * (GS01 * TS[b] + GS11 * TS[3 + b]);
        }
        const float dJ00 = dT[0] * P.R[0] + dT[1] * P.R[1] + dT[2] * P.R[2];
        const float dJ02 = dT[0] * P.R[6] + dT[1] * P.R[7] + dT[2] * P.R[8];
        const float dJ11 = dT[3] * P.R[3] + dT[4] * P.R[4] + dT[5] * P.R[5];
        const float dJ12 = dT[3] * P.R[6] + dT[4] * P.R[7] + dT[5] * P.R[8];
        float gt0 = gu * cam.fx * iz, gt1 = gv * cam.fy * iz;
        float gt2 = gz - (gu * cam.fx * t[0] + gv * cam.fy * t[1]) * iz * iz;
        gt2 += -(dJ00 * cam.fx + dJ11 * cam.fy) * iz * iz;
        gt2 += dJ02 * cam.fx * xz * iz * iz;
        gt2 += dJ12 * cam.fy * yz * iz * iz;
        if (!cx_) {
            gt0 += dJ02 * (-cam.fx * iz * iz);
            gt2 += dJ02 * (cam.fx * t[0] * iz * iz * iz);
        }
        if (!cy_) {
            gt1 += dJ12 * (-cam.fy * iz * iz);
            gt2 += dJ12 * (cam.fy * t[1] * iz * iz * iz);
        }
#pragma unroll
        for (int b = 0; b < 3; ++b) gmu[b] += P.R[b] * gt0 + P.R[3 + b] * gt1 + P.R[6 + b] * gt2;
    }
    if (!any) return;
    // dL/dM = 2 dL/dSigma M (dL/dSigma symmetric)
    float gM[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            gM[3 * a + b] = 2.f * (gS[3 * a] * m[b] + gS[3 * a + 1] * m[3 + b] + gS[3 * a + 2] * m[6 + b]);
    float gs[3], gR[9];
#pragma unroll
    for (int b = 0; b < 3; ++b) gs[b] = gM[b] * r[b] + gM[3 + b] * r[3 + b] + gM[6 + b] * r[6 + b];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) gR[3 * a + b] = gM[3 * a + b] * sc[b];
    // rotation entries -> unit quaternion (w, x, y, z)
    const float hw = 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
    const float hx = 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - qw * gR[5] + qz * gR[6] +
                            qw * gR[7] - 2.f * qx * gR[8]);
    const float hy = 2.f * (-2.f * qy * gR[0] + qx * gR[1] + qw * gR[2] + qx * gR[3] + qz * gR[5] - qw * gR[6] +
                            qz * gR[7] - 2.f * qy * gR[8]);
    const float hz = 2.f * (-2.f * qz * gR[0] - qw * gR[1] + qx * gR[2] + qw * gR[3] - 2.f * qz * gR[4] +
                            qy * gR[5] + qx * gR[6] + qy * gR[7]);
    const float dot = qw * hw + qx * hx + qy * hy + qz * hz;
    const float gq[4] = {(hw - qw * dot) / qn, (hx - qx * dot) / qn, (hy - qy * dot) / qn, (hz - qz * dot) / qn};
    const float out[14] = {gmu[0], gmu[1], gmu[2], gs[0], gs[1], gs[2], gq[0], gq[1], gq[2], gq[3],
                           gop, gcol[0], gcol[1], gcol[2]};
#pragma unroll
    for (int k = 0; k < 14; ++k)
        if (out[k] != 0.f) atomicAdd(gmap + k * n_map + g, out[k]);
}

cudaError_t launch_param_chain(const float *mx, const float *my, const float *mz, const float *attr, int64_t n_map,
                               const uint32_t *gidx, const Layout &L, int n_blocks, const ViewParams *views,
                               const CamParams &cam, const float *gin, float *gmap, cudaStream_t st)
{
    if (n_blocks <= 0 || L.V <= 0) return cudaSuccess;
    k_param_chain<<<n_blocks, PROJ_THREADS, 0, st>>>(mx, my, mz, attr, n_map, gidx, L, views, cam, gin, gmap);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Adam ---
// One Adam step (Kingma and Ba 2015) over the 14 parameter rows of the map,
// on 3D Gaussian Splatting's latent parameters: log scale (s = exp(l), so
// dL/dl = s dL/ds and s' = s exp(-step)), logit opacity (o = sigmoid(z),
// dL/dz = o (1 - o) dL/do), the rest as stored.  Group k in {mean, scale,
// quaternion, opacity, colour} has learning rate lr[k]; bc1, bc2 are the bias
// corrections 1 / (1 - beta^t).
__global__ void __launch_bounds__(256)
k_adam(float *__restrict__ mean, float *__restrict__ attr, const float *__restrict__ grad, float *__restrict__ m1,
       float *__restrict__ m2, int64_t n, AdamParams P)
{
    const int64_t total = 14 * n;
    for (int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * 256) {
        const int c = (int)(idx / n);
        const int64_t i = idx - (int64_t)c * n;
        float *p;
        int grp;
        if (c < 3) { p = mean + c * n + i; grp = 0; }
        else if (c < 6) { p = attr + (ATTR_SCALE + c - 3) * n + i; grp = 1; }
        else if (c < 10) { p = attr + (ATTR_QUAT + c - 6) * n + i; grp = 2; }
        else if (c == 10) { p = attr + ATTR_OPAC * n + i; grp = 3; }
        else { p = attr + (ATTR_SH + c - 11) * n + i; grp = 4; }
        const float x = *p;
        float gr = grad[idx];
        float o = 0.f;
        if (grp == 1) gr *= x;
        if (grp == 3) {
            o = fminf(fmaxf(x, P.o_min), 1.f - P.o_min);
            gr *= o * (1.f - o);
        }
        const float a = P.beta1 * m1[idx] + (1.f - P.beta1) * gr;
        const float b = P.beta2 * m2[idx] + (1.f - P.beta2) * gr * gr;
        m1[idx] = a;
        m2[idx] = b;
        const float step = P.lr[grp] * (a * P.bc1) / (sqrtf(b * P.bc2) + P.eps);
        if (grp == 1) {
            *p = x * expf(-step);
        } else if (grp == 3) {
            const float z = logf(o / (1.f - o)) - step;
            *p = 1.f / (1.f + expf(-z));
        } else {
            *p = x - step;
        }
    }
}

cudaError_t launch_adam(float *mean, float *attr, const float *grad, float *m1, float *m2, int64_t n,
                        const AdamParams &P, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>(ceil_div(14 * n, 256 * 4), 152 * 16);
    k_adam<<<(int)blocks, 256, 0, st>>>(mean, attr, grad, m1, m2, n, P);
    return cudaGetLastError();
}

}  // namespace reloc
