// project.cu -- K1 block-subset gather and K2 EWA projection + SH colour.
//
// K2 follows Sec. III-A of 3DGS-ReLoc: t = W mu (world-to-camera), pinhole
// projection m(mu) (Eq. proj), footprint covariance Sigma' = J W Sigma W^T J^T
// (Eq. foot_conv) with Sigma = R S S^T R^T, and the colour c_i (plain RGB, or
// real SH evaluated along the viewing ray).  One thread owns one Gaussian: it
// loads the attributes once (coalesced SoA loads) and projects them into every
// candidate view, so the map bytes are read once per call however many
// candidates there are.
#include "internal.cuh"

namespace reloc {

// ---------------------------------------------------------------- K1 ------

__global__ void k_gather_subset(const int64_t *__restrict__ run_begin, const int64_t *__restrict__ run_off,
                                int n_runs, int64_t S, uint32_t *__restrict__ gidx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    int lo = 0, hi = n_runs - 1;             // last run with run_off[r] <= i
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (run_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    gidx[i] = (uint32_t)(run_begin[lo] + (i - run_off[lo]));
}

cudaError_t launch_gather_subset(const int64_t *run_begin, const int64_t *run_off, int n_runs, int64_t total,
                                 uint32_t *gidx, cudaStream_t st)
{
    if (total <= 0 || n_runs <= 0) return cudaSuccess;
    k_gather_subset<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(run_begin, run_off, n_runs, total, gidx);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- K2 ------

template <typename T> __device__ __forceinline__ float ldattr(const T *p);
template <> __device__ __forceinline__ float ldattr<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldattr<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <> __device__ __forceinline__ float ldattr<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}

// Real orthonormal SH basis (Condon-Shortley phase) up to degree DEG for a
// unit direction, as explicit polynomials; normalisation constants are
// sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) (times sqrt 2 for m != 0) folded with the
// polynomial coefficients.
template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y)
{
    Y[0] = 0.28209479177387814f;
    if (DEG >= 1) {
        Y[1] = -0.48860251190291987f * y;
        Y[2] = 0.48860251190291987f * z;
        Y[3] = -0.48860251190291987f * x;
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = 1.0925484305920792f * x * y;
        Y[5] = -1.0925484305920792f * y * z;
        Y[6] = 0.31539156525252005f * (2.f * zz - xx - yy);
        Y[7] = -1.0925484305920792f * x * z;
        Y[8] = 0.5462742152960396f * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -0.5900435899266435f * y * (3.f * xx - yy);
            Y[10] = 2.890611442640554f * x * y * z;
            Y[11] = -0.4570457994644658f * y * (4.f * zz - xx - yy);
            Y[12] = 0.3731763325901154f * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -0.4570457994644658f * x * (4.f * zz - xx - yy);
            Y[14] = 1.445305721320277f * z * (xx - yy);
            Y[15] = -0.5900435899266435f * x * (xx - 3.f * yy);
        }
    }
}

constexpr int PROJ_VIEW_BATCH = 128;

// Principal-axis form of a footprint.  N = T M (2 x 3) holds the projected
// scaled axes of the Gaussian (T = J R_w, M = R S), so Sigma' = N N^T + eps I.
// With the eigenpairs (l1 >= l2, e1 orthogonal to e2) of Sigma',
//   -1/2 d^T Sigma'^-1 d = -1/2 (U^2 + V^2),  U = alpha . d,  V = beta . d,
//   alpha = e1 / sqrt(l1),  beta = e2 / sqrt(l2),
// which is what the record carries instead of the conic.  det(N N^T) is the
// squared norm of the cross product of N's rows (Lagrange's identity), a sum
// of squares: det(Sigma') = det(N N^T) + eps tr(N N^T) + eps^2 and
// l2 = det / l1 keep their relative precision for long thin footprints, where
// Sigma'_xx Sigma'_yy - Sigma'_xy^2 cancels.  The eigenvector is taken from
// the row of Sigma' - l1 I without cancellation (A - C and the root have the
// same sign).  Returns false unless Sigma' is positive definite; sxx, syy are
// the diagonal of Sigma' (the 3-sigma bounding box).  In FP32 the root that
// sets the eigenvector's direction is IEEE; the normalisation, l2 and the
// inverse square roots only scale the axes (by 1 + a few ulp, which moves the
// form by as little) and use the fast reciprocal (square root).
__device__ __forceinline__ float fp_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fp_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float fp_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fp_div(double a, double b) { return a / b; }
template <typename F>
__device__ __forceinline__ bool footprint_axes(const F (&n)[6], F eps, F &sxx, F &syy, F &det, F (&ab)[4])
{
    const F A0 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    const F C0 = n[3] * n[3] + n[4] * n[4] + n[5] * n[5];
    const F B0 = n[0] * n[3] + n[1] * n[4] + n[2] * n[5];
    const F x = n[1] * n[5] - n[2] * n[4];
    const F y = n[2] * n[3] - n[0] * n[5];
    const F z = n[0] * n[4] - n[1] * n[3];
    sxx = A0 + eps;
    syy = C0 + eps;
    det = (x * x + y * y + z * z) + eps * (A0 + C0 + eps);
    if (!(det > F(0))) return false;
    const F dd = A0 - C0;
    const F sq = sqrt(dd * dd + F(4) * B0 * B0);
    const F l1 = F(0.5) * (sxx + syy + sq);
    const F l2 = fp_div(det, l1);
    F ex, ey;
    if (dd >= F(0)) { ex = dd + sq; ey = F(2) * B0; }
    else { ex = F(2) * B0; ey = sq - dd; }
    const F en2 = ex * ex + ey * ey;
    if (en2 > F(0)) {
        const F ien = fp_rsqrt(en2);
        ex = ex * ien; ey = ey * ien;
    } else {
        ex = F(1); ey = F(0);
    }
    const F r1 = fp_rsqrt(l1), r2 = fp_rsqrt(l2);
    ab[0] = ex * r1; ab[1] = ey * r1;
    ab[2] = -ey * r2; ab[3] = ex * r2;
    return true;
}

template <typename T, int DEG>
__global__ void __launch_bounds__(PROJ_THREADS)
k_project(const float *__restrict__ mx, const float *__restrict__ my, const float *__restrict__ mz,
          const T *__restrict__ attr, int64_t n_map, const uint32_t *__restrict__ gidx, Layout L,
          const ViewParams *__restrict__ views, CamParams cam, float4 *__restrict__ rec,
          uint2 *__restrict__ rect, uint32_t *__restrict__ dkey)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    __shared__ ViewParams s_view[PROJ_VIEW_BATCH];

    // this block's query and Gaussians
    const int qi = find_segment(L.q_pblk, L.Q, (int)blockIdx.x);
    const int64_t S = L.q_gsub[qi + 1] - L.q_gsub[qi];
    const int64_t i = (int64_t)(blockIdx.x - L.q_pblk[qi]) * PROJ_THREADS + threadIdx.x;
    const bool active = i < S;
    const int v_begin = L.q_view[qi], V = L.q_view[qi + 1] - v_begin;

    // ---- per-Gaussian quantities, loaded and formed once ------------------
    float mu0 = 0, mu1 = 0, mu2 = 0, opac = 0;
    float m[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // M = R S, row-major
    float sh[3 * K];
    if (active) {
        const int64_t g = gidx[L.q_gsub[qi] + i];
        mu0 = __ldg(mx + g); mu1 = __ldg(my + g); mu2 = __ldg(mz + g);
        float s0 = ldattr(attr + (ATTR_SCALE + 0) * n_map + g);
        float s1 = ldattr(attr + (ATTR_SCALE + 1) * n_map + g);
        float s2 = ldattr(attr + (ATTR_SCALE + 2) * n_map + g);
        float qw = ldattr(attr + (ATTR_QUAT + 0) * n_map + g);
        float qx = ldattr(attr + (ATTR_QUAT + 1) * n_map + g);
        float qy = ldattr(attr + (ATTR_QUAT + 2) * n_map + g);
        float qz = ldattr(attr + (ATTR_QUAT + 3) * n_map + g);
        opac = ldattr(attr + ATTR_OPAC * n_map + g);
#pragma unroll
        for (int k = 0; k < 3 * K; ++k) sh[k] = ldattr(attr + (int64_t)(ATTR_SH + k) * n_map + g);
        // rotation from the normalised quaternion
        float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw /= qn; qx /= qn; qy /= qn; qz /= qn;
        float r00 = 1.f - 2.f * (qy * qy + qz * qz), r01 = 2.f * (qx * qy - qw * qz), r02 = 2.f * (qx * qz + qw * qy);
        float r10 = 2.f * (qx * qy + qw * qz), r11 = 1.f - 2.f * (qx * qx + qz * qz), r12 = 2.f * (qy * qz - qw * qx);
        float r20 = 2.f * (qx * qz - qw * qy), r21 = 2.f * (qy * qz + qw * qx), r22 = 1.f - 2.f * (qx * qx + qy * qy);
        // M = R S (Sigma = M M^T): column k is the k-th scaled axis
        m[0] = r00 * s0; m[1] = r01 * s1; m[2] = r02 * s2;
        m[3] = r10 * s0; m[4] = r11 * s1; m[5] = r12 * s2;
        m[6] = r20 * s0; m[7] = r21 * s1; m[8] = r22 * s2;
    }
    const float lopac = __log2f(opac);           // the record's log2 o, once per Gaussian
    const float cut2 = cam.cut;
    const float inv_tw = 1.0f / cam.tile_w, inv_th = 1.0f / cam.tile_h;

    for (int vb = 0; vb < V; vb += PROJ_VIEW_BATCH) {
        const int nb = min(PROJ_VIEW_BATCH, V - vb);
        __syncthreads();
        for (int k = threadIdx.x; k < nb * 16; k += PROJ_THREADS)
            reinterpret_cast<float *>(s_view)[k] = reinterpret_cast<const float *>(views + v_begin + vb)[k];
        __syncthreads();
        if (!active) continue;
        for (int vv = 0; vv < nb; ++vv) {
            const ViewParams &P = s_view[vv];
            const int v = v_begin + vb + vv;
            const int64_t o = L.vd_off[v] + i;
            // camera-space position t = R (mu - c)
            float d0 = (mu0 - P.c_hi[0]) - P.c_lo[0];
            float d1 = (mu1 - P.c_hi[1]) - P.c_lo[1];
            float d2 = (mu2 - P.c_hi[2]) - P.c_lo[2];
            float tx = P.R[0] * d0 + P.R[1] * d1 + P.R[2] * d2;
            float ty = P.R[3] * d0 + P.R[4] * d1 + P.R[5] * d2;
            float tz = P.R[6] * d0 + P.R[7] * d1 + P.R[8] * d2;
            uint32_t nt = 0;
            uint2 rc = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
            if (tz > cam.near_plane) {
                // Jacobian of the projection (FOV clamp in J only), from one
                // IEEE-rounded reciprocal of the depth (the pixel position
                // below keeps its IEEE divisions)
                const float iz = __frcp_rn(tz);
                float xz = fminf(fmaxf(tx * iz, -cam.limx), cam.limx);
                float yz = fminf(fmaxf(ty * iz, -cam.limy), cam.limy);
                float j00 = cam.fx * iz, j02 = -cam.fx * xz * iz;
                float j11 = cam.fy * iz, j12 = -cam.fy * yz * iz;
                // T = J R_w (2x3)
                float t00 = j00 * P.R[0] + j02 * P.R[6], t01 = j00 * P.R[1] + j02 * P.R[7], t02 = j00 * P.R[2] + j02 * P.R[8];
                float t10 = j11 * P.R[3] + j12 * P.R[6], t11 = j11 * P.R[4] + j12 * P.R[7], t12 = j11 * P.R[5] + j12 * P.R[8];
                // N = T M: the projected scaled axes (Sigma' = N N^T + eps I)
                float nn[6];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    nn[k] = t00 * m[k] + t01 * m[3 + k] + t02 * m[6 + k];
                    nn[3 + k] = t10 * m[k] + t11 * m[3 + k] + t12 * m[6 + k];
                }
                float ca, cc, det, ab[4];
                bool ok = footprint_axes(nn, cam.eps2d, ca, cc, det, ab);
                if (det < cam.det_fp64) {
                    // near-degenerate footprint: N, Sigma' and its axes in FP64
                    const double T0[3] = {(double)t00, (double)t01, (double)t02};
                    const double T1[3] = {(double)t10, (double)t11, (double)t12};
                    double nd[6];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        nd[k] = T0[0] * (double)m[k] + T0[1] * (double)m[3 + k] + T0[2] * (double)m[6 + k];
                        nd[3 + k] = T1[0] * (double)m[k] + T1[1] * (double)m[3 + k] + T1[2] * (double)m[6 + k];
                    }
                    double sxd, syd, dd, abd[4];
                    ok = footprint_axes(nd, (double)cam.eps2d, sxd, syd, dd, abd);
                    ca = (float)sxd; cc = (float)syd;
#pragma unroll
                    for (int k = 0; k < 4; ++k) ab[k] = (float)abd[k];
                    ok = ok && isfinite(ab[2]) && isfinite(ab[3]);
                }
                if (ok) {
                    float u = cam.fx * tx / tz + cam.cx;
                    float vpx = cam.fy * ty / tz + cam.cy;
                    float rx = cut2 * sqrtf(ca), ry = cut2 * sqrtf(cc);
                    float xlo = u - rx, xhi = u + rx, ylo = vpx - ry, yhi = vpx + ry;
                    if (!(xhi < 0.f || xlo >= (float)cam.width || yhi < 0.f || ylo >= (float)cam.height)) {
                        int x0 = max(0, (int)floorf(xlo * inv_tw));
                        int x1 = min(cam.ntx - 1, (int)floorf(xhi * inv_tw));
                        int y0 = max(0, (int)floorf(ylo * inv_th));
                        int y1 = min(cam.nty - 1, (int)floorf(yhi * inv_th));
                        nt = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
                        rc = make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16));
                        float cr, cg, cbl;
                        if (DEG == 0) {
                            cr = sh[0]; cg = sh[1]; cbl = sh[2];
                        } else {
                            float inv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
                            float Y[K];
                            sh_basis<DEG>(d0 * inv, d1 * inv, d2 * inv, Y);
                            cr = 0.5f; cg = 0.5f; cbl = 0.5f;
#pragma unroll
                            for (int k = 0; k < K; ++k) {
                                cr += sh[3 * k] * Y[k];
                                cg += sh[3 * k + 1] * Y[k];
                                cbl += sh[3 * k + 2] * Y[k];
                            }
                            cr = fmaxf(cr, 0.f); cg = fmaxf(cg, 0.f); cbl = fmaxf(cbl, 0.f);
                        }
                        // the blend's form: log2(o) and the axes scaled by
                        // sqrt(log2(e) / 2), so that the base-2 exponent is
                        // log2(o) - (alpha' . d)^2 - (beta' . d)^2
                        constexpr float KAPPA = 0.8493218002880191f;
                        float4 *rp = rec + 3 * o;
                        rp[0] = make_float4(u, vpx, tz, lopac);
                        rp[1] = make_float4(KAPPA * ab[0], KAPPA * ab[1], KAPPA * ab[2], KAPPA * ab[3]);
                        rp[2] = make_float4(cr, cg, cbl, 0.f);
                    }
                }
            }
            if (nt) rect[o] = rc;
            // the depth key doubles as the visibility flag (0xFFFFFFFF: culled, and
            // no rectangle written); visible depths are positive and finite
            dkey[o] = nt ? __float_as_uint(tz) : 0xFFFFFFFFu;
        }
    }
}

template <typename T>
static cudaError_t project_t(const float *mx, const float *my, const float *mz, const T *attr, int sh_degree,
                             int64_t n_map, const uint32_t *gidx, const Layout &L, int n_blocks,
                             const ViewParams *views, const CamParams &cam, float4 *rec, uint2 *rect,
                             uint32_t *dkey, cudaStream_t st)
{
    dim3 grid((unsigned)n_blocks);
    switch (sh_degree) {
    case 0: k_project<T, 0><<<grid, PROJ_THREADS, 0, st>>>(mx, my, mz, attr, n_map, gidx, L, views, cam, rec, rect, dkey); break;
    case 1: k_project<T, 1><<<grid, PROJ_THREADS, 0, st>>>(mx, my, mz, attr, n_map, gidx, L, views, cam, rec, rect, dkey); break;
    case 2: k_project<T, 2><<<grid, PROJ_THREADS, 0, st>>>(mx, my, mz, attr, n_map, gidx, L, views, cam, rec, rect, dkey); break;
    case 3: k_project<T, 3><<<grid, PROJ_THREADS, 0, st>>>(mx, my, mz, attr, n_map, gidx, L, views, cam, rec, rect, dkey); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_project(const float *mx, const float *my, const float *mz, const void *attr, int precision,
                           int sh_degree, int64_t n_map, const uint32_t *gidx, const Layout &L, int n_blocks,
                           const ViewParams *views, const CamParams &cam, float4 *rec, uint2 *rect,
                           uint32_t *dkey, cudaStream_t st)
{
    if (n_blocks <= 0) return cudaSuccess;
    switch (precision) {
    case 0: return project_t(mx, my, mz, (const float *)attr, sh_degree, n_map, gidx, L, n_blocks, views, cam, rec, rect, dkey, st);
    case 1: return project_t(mx, my, mz, (const __half *)attr, sh_degree, n_map, gidx, L, n_blocks, views, cam, rec, rect, dkey, st);
    case 2: return project_t(mx, my, mz, (const __nv_bfloat16 *)attr, sh_degree, n_map, gidx, L, n_blocks, views, cam, rec, rect, dkey, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------ pose chain --
// Per (view, Gaussian) of one query: the gradients of the view's NCC with
// respect to the Gaussian's projected mean and conic (gin: u, v, a, b, c)
// carried back through the conic inverse A = Sigma'^-1 (dL/dSigma' =
// -A G_A A), Sigma' = T Sigma T^T + eps I (dL/dT = 2 dL/dSigma' T Sigma),
// T = J R and the projection u = fx tx/tz + cx, v = fy ty/tz + cy, J(t) (a
// clamped ratio in J is a constant) to the camera point t and the rotation R,
// then to the left pose update: d/d rho = dL/dt, d/d phi = t x dL/dt +
// (N12 - N21, N20 - N02, N01 - N10) with N = R (dL/dR)^T.  FP32 per pair;
// each block sums its Gaussians per view into part[block][view][6] (FP64).
template <typename T>
__global__ void __launch_bounds__(PROJ_THREADS)
k_pose_chain(const float *__restrict__ mx, const float *__restrict__ my, const float *__restrict__ mz,
             const T *__restrict__ attr, int64_t n_map, const uint32_t *__restrict__ gidx, Layout L,
             const ViewParams *__restrict__ views, CamParams cam, const float *__restrict__ gin,
             double *__restrict__ part)
{
    __shared__ float s_red[PROJ_THREADS / 32][6];
    const int qi = find_segment(L.q_pblk, L.Q, (int)blockIdx.x);
    const int64_t S = L.q_gsub[qi + 1] - L.q_gsub[qi];
    const int64_t i = (int64_t)(blockIdx.x - L.q_pblk[qi]) * PROJ_THREADS + threadIdx.x;
    const bool active = i < S;
    const int v_begin = L.q_view[qi], V = L.q_view[qi + 1] - v_begin;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float mu0 = 0, mu1 = 0, mu2 = 0;
    float Sg[6] = {0, 0, 0, 0, 0, 0};          // Sigma: 00 01 02 11 12 22
    if (active) {
        const int64_t g = gidx[L.q_gsub[qi] + i];
        mu0 = __ldg(mx + g); mu1 = __ldg(my + g); mu2 = __ldg(mz + g);
        const float s0 = ldattr(attr + (ATTR_SCALE + 0) * n_map + g);
        const float s1 = ldattr(attr + (ATTR_SCALE + 1) * n_map + g);
        const float s2 = ldattr(attr + (ATTR_SCALE + 2) * n_map + g);
        float qw = ldattr(attr + (ATTR_QUAT + 0) * n_map + g);
        float qx = ldattr(attr + (ATTR_QUAT + 1) * n_map + g);
        float qy = ldattr(attr + (ATTR_QUAT + 2) * n_map + g);
        float qz = ldattr(attr + (ATTR_QUAT + 3) * n_map + g);
        const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw /= qn; qx /= qn; qy /= qn; qz /= qn;
        const float r[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                            2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                            2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
        const float sc[3] = {s0, s1, s2};
        float m[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) m[3 * a + b] = r[3 * a + b] * sc[b];
        int k = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b) Sg[k++] = m[3 * a] * m[3 * b] + m[3 * a + 1] * m[3 * b + 1] + m[3 * a + 2] * m[3 * b + 2];
    }
    const float Sm[9] = {Sg[0], Sg[1], Sg[2], Sg[1], Sg[3], Sg[4], Sg[2], Sg[4], Sg[5]};
    for (int vv = 0; vv < V; ++vv) {
        const int v = v_begin + vv;
        float acc[6] = {0, 0, 0, 0, 0, 0};
        const float *g5 = active ? gin + 5 * (L.vd_off[v] + i) : nullptr;
        const float gu = active ? g5[0] : 0.f, gv = active ? g5[1] : 0.f, ga = active ? g5[2] : 0.f;
        const float gb = active ? g5[3] : 0.f, gc = active ? g5[4] : 0.f;
        if (gu != 0.f || gv != 0.f || ga != 0.f || gb != 0.f || gc != 0.f) {
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
            float Tm[6];                                          // T = J R (2 x 3)
            for (int b = 0; b < 3; ++b) {
                Tm[b] = J00 * P.R[b] + J02 * P.R[6 + b];
                Tm[3 + b] = J11 * P.R[3 + b] + J12 * P.R[6 + b];
            }
            float TS[6];                                          // T Sigma (2 x 3)
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 3; ++b)
                    TS[3 * a + b] = Tm[3 * a] * Sm[b] + Tm[3 * a + 1] * Sm[3 + b] + Tm[3 * a + 2] * Sm[6 + b];
            const float sa = TS[0] * Tm[0] + TS[1] * Tm[1] + TS[2] * Tm[2] + cam.eps2d;
            const float sb = TS[0] * Tm[3] + TS[1] * Tm[4] + TS[2] * Tm[5];
            const float scc = TS[3] * Tm[3] + TS[4] * Tm[4] + TS[5] * Tm[5] + cam.eps2d;
            const float idet = 1.f / (sa * scc - sb * sb);
            const float A00 = scc * idet, A01 = -sb * idet, A11 = sa * idet;
            // dL/dSigma' = -A G_A A, G_A = [[ga, gb/2], [gb/2, gc]]
            const float h = 0.5f * gb;
            const float M00 = A00 * ga + A01 * h, M01 = A00 * h + A01 * gc;
            const float M10 = A01 * ga + A11 * h, M11 = A01 * h + A11 * gc;
            const float GS00 = -(M00 * A00 + M01 * A01), GS01 = -(M00 * A01 + M01 * A11);
            const float GS11 = -(M10 * A01 + M11 * A11);
            // dL/dT = 2 GS T Sigma
            float dT[6];
            for (int b = 0; b < 3; ++b) {
                dT[b] = 2.f * (GS00 * TS[b] + GS01 * TS[3 + b]);
                dT[3 + b] = 2.f * (GS01 * TS[b] + GS11 * TS[3 + b]);
            }
            // dL/dR = J^T dT, dL/dJ = dT R^T (the four non-zero entries of J)
            float dR[9];
            for (int b = 0; b < 3; ++b) {
                dR[b] = J00 * dT[b];
                dR[3 + b] = J11 * dT[3 + b];
                dR[6 + b] = J02 * dT[b] + J12 * dT[3 + b];
            }
            const float dJ00 = dT[0] * P.R[0] + dT[1] * P.R[1] + dT[2] * P.R[2];
            const float dJ02 = dT[0] * P.R[6] + dT[1] * P.R[7] + dT[2] * P.R[8];
            const float dJ11 = dT[3] * P.R[3] + dT[4] * P.R[4] + dT[5] * P.R[5];
            const float dJ12 = dT[3] * P.R[6] + dT[4] * P.R[7] + dT[5] * P.R[8];
            // dL/dt from u, v and J
            float gt0 = gu * cam.fx * iz, gt1 = gv * cam.fy * iz;
            float gt2 = -(gu * cam.fx * t[0] + gv * cam.fy * t[1]) * iz * iz;
            gt2 += -(dJ00 * cam.fx + dJ11 * cam.fy) * iz * iz;
            // J02 = -fx xz / tz, xz = tx / tz unless clamped
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
            // N = R dR^T
            float N[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    N[3 * a + b] = P.R[3 * a] * dR[3 * b] + P.R[3 * a + 1] * dR[3 * b + 1] + P.R[3 * a + 2] * dR[3 * b + 2];
            acc[0] = gt0; acc[1] = gt1; acc[2] = gt2;
            acc[3] = t[1] * gt2 - t[2] * gt1 + (N[5] - N[7]);
            acc[4] = t[2] * gt0 - t[0] * gt2 + (N[6] - N[2]);
            acc[5] = t[0] * gt1 - t[1] * gt0 + (N[1] - N[3]);
        }
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            float x = acc[m];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) s_red[warp][m] = x;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            double x = 0.0;
            for (int w = 0; w < PROJ_THREADS / 32; ++w) x += (double)s_red[w][threadIdx.x];
            part[((int64_t)(blockIdx.x - L.q_pblk[qi]) * V + vv) * 6 + threadIdx.x] = x;
        }
        __syncthreads();
    }
}

// out[v][6] = sum over the n_blk blocks of part[block][v][6], in block order.
__global__ void k_pose_reduce(const double *__restrict__ part, int n_blk, int V, double *__restrict__ out)
{
    __shared__ double s[6][8];
    const int v = blockIdx.x;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < n_blk; b += blockDim.x)
        for (int m = 0; m < 6; ++m) acc[m] += part[((int64_t)b * V + v) * 6 + m];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int m = 0; m < 6; ++m) {
        double x = acc[m];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s[m][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += s[threadIdx.x][w];
        out[6 * (int64_t)v + threadIdx.x] = x;
    }
}

template <typename T>
static cudaError_t pose_chain_t(const float *mx, const float *my, const float *mz, const T *attr, int64_t n_map,
                                const uint32_t *gidx, const Layout &L, int n_blocks, const ViewParams *views,
                                const CamParams &cam, const float *gin, double *part, double *out, cudaStream_t st)
{
    k_pose_chain<T><<<n_blocks, PROJ_THREADS, 0, st>>>(mx, my, mz, attr, n_map, gidx, L, views, cam, gin, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pose_reduce<<<L.V, 256, 0, st>>>(part, n_blocks, L.V, out);
    return cudaGetLastError();
}

cudaError_t launch_pose_chain(const float *mx, const float *my, const float *mz, const void *attr, int precision,
                              int64_t n_map, const uint32_t *gidx, const Layout &L, int n_blocks,
                              const ViewParams *views, const CamParams &cam, const float *gin, double *part,
                              double *out, cudaStream_t st)
{
    if (n_blocks <= 0 || L.V <= 0) return cudaSuccess;
    switch (precision) {
    case 0: return pose_chain_t(mx, my, mz, (const float *)attr, n_map, gidx, L, n_blocks, views, cam, gin, part, out, st);
    case 1: return pose_chain_t(mx, my, mz, (const __half *)attr, n_map, gidx, L, n_blocks, views, cam, gin, part, out, st);
    case 2: return pose_chain_t(mx, my, mz, (const __nv_bfloat16 *)attr, n_map, gidx, L, n_blocks, views, cam, gin, part, out, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace reloc
