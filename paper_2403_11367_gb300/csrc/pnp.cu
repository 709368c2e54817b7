// pnp.cu -- pose refinement by Perspective-n-Point (Sec. III-C.2).
//
// The rendered view at pose_render supplies depth: each matched render pixel
// is back-projected with the view's normalised depth D / A (Eq. depth over
// 1 - T) into a world point X_i; the query's pose W = [R | t] then minimises
// the Huber cost of the reprojection errors pi(W X_i) - q_i.  The solve is
// iteratively reweighted Gauss-Newton in FP64 with the update applied on the
// left, W <- [Exp(phi) R | Exp(phi) t + rho], so the Jacobian of a camera
// point P = R X + t is [I | -[P]x] and of its pixel
// J_pi = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]].
//
// The problem is small (thousands of pairs, a 6 x 6 system per iteration)
// but FP64, whose rate per SM is low on this GPU, so the pairs are spread
// over up to one block per SM in one cooperative launch: every pass over the
// pairs writes one partial sum per block, block 0 adds them in block order
// (the result does not depend on timing) and factors the system, and grid
// barriers separate the phases.  The solver state (pose, trial pose, step,
// decision) lives in global memory and is read past L1 after each barrier.
#include <algorithm>

#include <cooperative_groups.h>

#include "internal.cuh"

namespace reloc {

constexpr int PNP_THREADS = 256;
constexpr int PNP_ACC = 28;              // 21 (upper H) + 6 (g) + cost

struct PnpArgs {
    double Rr[9], tr[3];                 // render pose (world -> camera)
    double W0[12];                       // initial pose: R row-major, then t
    double fx, fy, cx, cy;
    int width, height, n, max_iters;
    double huber, alpha_min, tol;
    const float *depth, *alpha;
    const float4 *pairs;
    double4 *X;                          // scratch [n]: world point, w = 1 if used
    double *part;                        // scratch [gridDim.x][PNP_ACC]: per-block sums
    double *st;                          // scratch [PNP_STATE]: solver state
    double *out;                         // [16 pose, rms, cost, n_used, iters, status]
};

// solver state in global memory
enum { PS_POSE = 0, PS_TRIAL = 12, PS_DELTA = 24, PS_COST = 30, PS_STEP = 31, PS_FLAG = 32, PS_NUSED = 33,
       PNP_STATE = 34 };

__device__ __forceinline__ double warp_sum_dbl(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block sum of v[0..m) (every thread); the results land in s_out[0..m).
__device__ void block_sum(const double *v, int m, double (*s_red)[PNP_ACC], double *s_out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < m; ++j) {
        const double s = warp_sum_dbl(v[j]);
        if (lane == 0) s_red[warp][j] = s;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double s = 0.0;
        for (int w = 0; w < PNP_THREADS / 32; ++w) s += s_red[w][threadIdx.x];
        s_out[threadIdx.x] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double huber_rho(double e, double k) { return e <= k ? 0.5 * e * e : k * (e - 0.5 * k); }

// Huber cost (acc[27]) and, with GRAD, the weighted normal equations of pose
// (R, t) over this thread's pairs.  Also the plain squared error and count
// (acc[0], acc[1]) when RMS is set (no gradient then).
template <bool GRAD, bool RMS>
__device__ void pnp_accumulate(const PnpArgs &a, const double *R, const double *t, double *acc)
{
    for (int j = 0; j < PNP_ACC; ++j) acc[j] = 0.0;
    for (int i = blockIdx.x * PNP_THREADS + threadIdx.x; i < a.n; i += gridDim.x * PNP_THREADS) {
        const double4 X = a.X[i];
        if (X.w == 0.0) continue;
        const float4 q = a.pairs[i];
        const double px = R[0] * X.x + R[1] * X.y + R[2] * X.z + t[0];
        const double py = R[3] * X.x + R[4] * X.y + R[5] * X.z + t[1];
        const double pz = R[6] * X.x + R[7] * X.y + R[8] * X.z + t[2];
        if (pz <= 1e-6) continue;
        const double iz = 1.0 / pz;
        const double ru = a.fx * px * iz + a.cx - (double)q.z;
        const double rv = a.fy * py * iz + a.cy - (double)q.w;
        const double e = sqrt(ru * ru + rv * rv);
        acc[27] += huber_rho(e, a.huber);
        if (RMS) {
            acc[0] += e * e;
            acc[1] += 1.0;
        }
        if (GRAD) {
            const double w = e <= a.huber ? 1.0 : a.huber / e;
            const double a0 = a.fx * iz, a2 = -a.fx * px * iz * iz;
            const double b1 = a.fy * iz, b2 = -a.fy * py * iz * iz;
            const double Ju[6] = {a0, 0.0, a2, a2 * py, a0 * pz - a2 * px, -a0 * py};
            const double Jv[6] = {0.0, b1, b2, -b1 * pz + b2 * py, -b2 * px, b1 * px};
            int k = 0;
            for (int r = 0; r < 6; ++r)
                for (int c = r; c < 6; ++c) acc[k++] += w * (Ju[r] * Ju[c] + Jv[r] * Jv[c]);
            for (int r = 0; r < 6; ++r) acc[21 + r] += w * (Ju[r] * ru + Jv[r] * rv);
        }
    }
}

// W' = [Exp(phi) R | Exp(phi) t + rho] for delta = (rho, phi) scaled by s.
__device__ void apply_update(const double *W, const double *delta, double s, double *Wn)
{
    const double rho[3] = {s * delta[0], s * delta[1], s * delta[2]};
    const double ph[3] = {s * delta[3], s * delta[4], s * delta[5]};
    const double th2 = ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2], th = sqrt(th2);
    double A, B;                                   // Exp = I + A K + B K^2, K = [phi]x
    if (th < 1e-8) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
    }
    const double K[9] = {0.0, -ph[2], ph[1], ph[2], 0.0, -ph[0], -ph[1], ph[0], 0.0};
    double E[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double k2 = 0.0;
            for (int m = 0; m < 3; ++m) k2 += K[3 * r + m] * K[3 * m + c];
            E[3 * r + c] = (r == c ? 1.0 : 0.0) + A * K[3 * r + c] + B * k2;
        }
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
            Wn[3 * r + c] = E[3 * r] * W[c] + E[3 * r + 1] * W[3 + c] + E[3 * r + 2] * W[6 + c];
        Wn[9 + r] = E[3 * r] * W[9] + E[3 * r + 1] * W[10] + E[3 * r + 2] * W[11] + rho[r];
    }
}

// Solve (H + 1e-9 tr(H)/6 I) x = -g by Cholesky; H given as 21 upper entries.
__device__ bool solve6(const double *Hu, const double *g, double *x)
{
    double H[36];
    int k = 0;
    for (int r = 0; r < 6; ++r)
        for (int c = r; c < 6; ++c) H[6 * r + c] = H[6 * c + r] = Hu[k++];
    const double tr = H[0] + H[7] + H[14] + H[21] + H[28] + H[35];
    for (int r = 0; r < 6; ++r) H[7 * r] += 1e-9 * tr / 6.0;
    double L[36] = {0};
    for (int j = 0; j < 6; ++j) {
        double d = H[7 * j];
        for (int m = 0; m < j; ++m) d -= L[6 * j + m] * L[6 * j + m];
        if (!(d > 0.0)) return false;
        L[7 * j] = sqrt(d);
        for (int i = j + 1; i < 6; ++i) {
            double s = H[6 * i + j];
            for (int m = 0; m < j; ++m) s -= L[6 * i + m] * L[6 * j + m];
            L[6 * i + j] = s / L[7 * j];
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = -g[i];
        for (int m = 0; m < i; ++m) s -= L[6 * i + m] * y[m];
        y[i] = s / L[7 * i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int m = i + 1; m < 6; ++m) s -= L[6 * m + i] * x[m];
        x[i] = s / L[7 * i];
    }
    return true;
}

// This block's sums of v[0..m) into part[blockIdx.x][0..m).
__device__ void block_partial(const PnpArgs &a, const double *v, int m, double (*s_red)[PNP_ACC], double *s_sum)
{
    block_sum(v, m, s_red, s_sum);
    if (threadIdx.x < m) a.part[(int64_t)blockIdx.x * PNP_ACC + threadIdx.x] = s_sum[threadIdx.x];
}

// Block 0: totals of the per-block sums of entries [j0, j0 + m), in block order.
__device__ void grid_total(const PnpArgs &a, int j0, int m, double *out)
{
    if (threadIdx.x < m) {
        double t = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(a.part + (int64_t)b * PNP_ACC + j0 + threadIdx.x);
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(PNP_THREADS) k_refine_pnp(PnpArgs a)
{
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    __shared__ double s_red[PNP_THREADS / 32][PNP_ACC];
    __shared__ double s_sum[PNP_ACC];
    __shared__ double s_tot[PNP_ACC];
    __shared__ double s_pose[12];
    double acc[PNP_ACC];
    double *st = a.st;
    const bool lead = blockIdx.x == 0;

    // back-projection of every pair with the rendered depth
    double used = 0.0;
    for (int i = blockIdx.x * PNP_THREADS + threadIdx.x; i < a.n; i += gridDim.x * PNP_THREADS) {
        const float4 p = a.pairs[i];
        double4 X = make_double4(0.0, 0.0, 0.0, 0.0);
        const double sx = (double)p.x - 0.5, sy = (double)p.y - 0.5;
        if (isfinite(sx) && isfinite(sy) && isfinite((double)p.z) && isfinite((double)p.w)) {
            const double fx0 = floor(sx), fy0 = floor(sy);
            if (fx0 >= 0.0 && fy0 >= 0.0 && fx0 + 1.0 < (double)a.width && fy0 + 1.0 < (double)a.height) {
                const int x0 = (int)fx0, y0 = (int)fy0;
                const double wx = sx - fx0, wy = sy - fy0;
                const int64_t o = (int64_t)y0 * a.width + x0;
                const double D = (1 - wy) * ((1 - wx) * a.depth[o] + wx * a.depth[o + 1]) +
                                 wy * ((1 - wx) * a.depth[o + a.width] + wx * a.depth[o + a.width + 1]);
                const double A = (1 - wy) * ((1 - wx) * a.alpha[o] + wx * a.alpha[o + 1]) +
                                 wy * ((1 - wx) * a.alpha[o + a.width] + wx * a.alpha[o + a.width + 1]);
                if (A >= a.alpha_min) {
                    const double z = D / A;
                    const double c[3] = {z * ((double)p.x - a.cx) / a.fx - a.tr[0],
                                         z * ((double)p.y - a.cy) / a.fy - a.tr[1], z - a.tr[2]};
                    X.x = a.Rr[0] * c[0] + a.Rr[3] * c[1] + a.Rr[6] * c[2];
                    X.y = a.Rr[1] * c[0] + a.Rr[4] * c[1] + a.Rr[7] * c[2];
                    X.z = a.Rr[2] * c[0] + a.Rr[5] * c[1] + a.Rr[8] * c[2];
                    X.w = 1.0;
                    used += 1.0;
                }
            }
        }
        a.X[i] = X;
    }
    block_partial(a, &used, 1, s_red, s_sum);
    grid.sync();
    if (lead) {
        grid_total(a, 0, 1, s_tot);
        if (threadIdx.x < 12) st[PS_POSE + threadIdx.x] = a.W0[threadIdx.x];
        if (threadIdx.x == 0) st[PS_NUSED] = s_tot[0];
    }
    grid.sync();
    const double n_used = __ldcg(st + PS_NUSED);
    // load a 12-entry pose from the state into shared memory
    auto load_pose = [&](int off) {
        if (threadIdx.x < 12) s_pose[threadIdx.x] = __ldcg(st + off + threadIdx.x);
        __syncthreads();
    };
    int it = 0;
    if (n_used >= 3.0) {
        for (; it < a.max_iters; ++it) {
            load_pose(PS_POSE);
            pnp_accumulate<true, false>(a, s_pose, s_pose + 9, acc);
            block_partial(a, acc, PNP_ACC, s_red, s_sum);
            grid.sync();
            if (lead) {
                grid_total(a, 0, PNP_ACC, s_tot);
                if (threadIdx.x == 0) {
                    double delta[6];
                    const bool ok = solve6(s_tot, s_tot + 21, delta);
                    for (int j = 0; j < 6; ++j) st[PS_DELTA + j] = delta[j];
                    st[PS_COST] = s_tot[27];
                    st[PS_STEP] = 1.0;
                    st[PS_FLAG] = ok ? 0.0 : 2.0;
                }
            }
            grid.sync();
            if (__ldcg(st + PS_FLAG) == 2.0) break;
            for (int bt = 0; bt <= 10; ++bt) {      // backtrack until the cost drops
                if (lead && threadIdx.x == 0) {
                    double W[12], d[6], Wt[12];
                    for (int j = 0; j < 12; ++j) W[j] = st[PS_POSE + j];
                    for (int j = 0; j < 6; ++j) d[j] = st[PS_DELTA + j];
                    apply_update(W, d, st[PS_STEP], Wt);
                    for (int j = 0; j < 12; ++j) st[PS_TRIAL + j] = Wt[j];
                }
                grid.sync();
                load_pose(PS_TRIAL);
                pnp_accumulate<false, false>(a, s_pose, s_pose + 9, acc);
                block_partial(a, acc + 27, 1, s_red, s_sum);
                grid.sync();
                if (lead) {
                    grid_total(a, 0, 1, s_tot);
                    if (threadIdx.x == 0) {
                        if (s_tot[0] < st[PS_COST]) {
                            for (int j = 0; j < 12; ++j) st[PS_POSE + j] = st[PS_TRIAL + j];
                            st[PS_FLAG] = 1.0;
                        } else {
                            st[PS_STEP] *= 0.5;
                        }
                    }
                }
                grid.sync();
                if (__ldcg(st + PS_FLAG) == 1.0) break;
            }
            if (__ldcg(st + PS_FLAG) != 1.0) break;  // no step lowers the cost: converged
            double dmax = 0.0;
            const double step = __ldcg(st + PS_STEP);
            for (int j = 0; j < 6; ++j) dmax = fmax(dmax, fabs(step * __ldcg(st + PS_DELTA + j)));
            if (dmax < a.tol) {
                ++it;
                break;
            }
        }
    }
    load_pose(PS_POSE);
    pnp_accumulate<false, true>(a, s_pose, s_pose + 9, acc);
    acc[2] = acc[27];
    block_partial(a, acc, 3, s_red, s_sum);
    grid.sync();
    if (lead) {
        grid_total(a, 0, 3, s_tot);
        if (threadIdx.x == 0) {
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c) a.out[4 * r + c] = s_pose[3 * r + c];
                a.out[4 * r + 3] = s_pose[9 + r];
            }
            a.out[12] = a.out[13] = a.out[14] = 0.0;
            a.out[15] = 1.0;
            a.out[16] = s_tot[1] > 0.0 ? sqrt(s_tot[0] / s_tot[1]) : 0.0;
            a.out[17] = s_tot[2];
            a.out[18] = n_used;
            a.out[19] = (double)it;
        }
    }
}

cudaError_t launch_refine_pnp(const double *pose_render, const double *pose_init, double fx, double fy, double cx,
                              double cy, int width, int height, const float *depth, const float *alpha,
                              const float *pairs, int n, int max_iters, double huber, double alpha_min, double tol,
                              double *X_scratch, double *out_dev, cudaStream_t st)
{
    PnpArgs a;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            a.Rr[3 * r + c] = pose_render[4 * r + c];
            a.W0[3 * r + c] = pose_init[4 * r + c];
        }
        a.tr[r] = pose_render[4 * r + 3];
        a.W0[9 + r] = pose_init[4 * r + 3];
    }
    a.fx = fx; a.fy = fy; a.cx = cx; a.cy = cy;
    a.width = width; a.height = height; a.n = n; a.max_iters = max_iters;
    a.huber = huber; a.alpha_min = alpha_min; a.tol = tol;
    a.depth = depth; a.alpha = alpha;
    a.pairs = reinterpret_cast<const float4 *>(pairs);
    a.X = reinterpret_cast<double4 *>(X_scratch);
    a.out = out_dev;
    // one block per SM at most (all resident: the launch is cooperative)
    int dev = 0, n_sm = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(n_sm, ceil_div(n, PNP_THREADS)));
    a.part = X_scratch + 4 * (int64_t)n;
    a.st = a.part + (int64_t)nb * PNP_ACC;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)k_refine_pnp, dim3(nb), dim3(PNP_THREADS), args, 0, st);
    return e;
}

}  // namespace reloc
