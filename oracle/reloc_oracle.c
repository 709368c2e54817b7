/*
 * reloc_oracle.c -- FP64 CPU oracle of the 3DGS-ReLoc relocalization hot path
 * (Jiang, Pandey, Saripalli, "3DGS-ReLoc", arXiv 2403.11367).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   - Gaussian parameterisation g = [mu, S, R, c, o] with Sigma = R S S^T R^T
 *     and R = q2R(q)                                             (Sec. III-A)
 *   - world-to-camera transform and pinhole projection m(mu)     (Eq. proj)
 *   - EWA footprint covariance Sigma^c = J W Sigma W^T J^T, 2x2  (Eq. foot_conv)
 *   - footprint q_i = o_i G(x - mu_hat)                          (Eq. footprint)
 *   - front-to-back colour compositing, Max's model              (Sec. III-A, Eq. 1)
 *   - depth compositing with z_i = camera-space depth            (Sec. III-A, depth eq.)
 *   - normalised cross-correlation                               (Sec. III-C.1, Eq. ncc)
 *   - block (2D voxel) selection around a coarse pose            (Sec. III-B.2, III-C.1)
 *   - argmax over the candidate grid                             (Sec. III-C.1)
 *   - map-training loss L_rgb = (1 - lambda) L1 + lambda D-SSIM  (Sec. III-B.3, Eq. 3)
 *     in L = w_photo L_photo + w_reproj L_reproj                  (Eqs. 4-6)
 *     with SSIM of Wang, Bovik, Sheikh and Simoncelli (2004), and its
 *     derivatives along parameter directions (forward mode)
 * plus an integer replay of the tile|depth key build and stable sort so the
 * GPU's keys and tile lists can be compared bit for bit.
 *
 * Readings taken where the paper is silent or garbled (each one is a
 * parameter or a documented rule below):
 *   - the 1/(|J^-1||W^-1|) factor of Eq. footprint is dropped (W is rigid;
 *     the unnormalised kernel keeps alpha <= o <= 1);
 *   - mu_hat is the projected mean (first two components of m(mu));
 *   - inclusion: pixel centre x is inside iff d^T Sigma'^-1 d <= cut^2 (cut = 3);
 *   - alpha = min(alpha_max, o exp(power)); skipped if alpha < alpha_min;
 *   - transmittance stop: if T (1 - alpha) < t_min the Gaussian is not added
 *     and the pixel is finished;
 *   - Sigma' gets eps (px^2) added to its diagonal; J uses tx/tz, ty/tz
 *     clamped to +-fov_clamp * tan(half FOV);
 *   - cull if tz <= near, det(Sigma') <= 0 or the 3-sigma box misses the image;
 *   - SH degree 0 is plain RGB; degree >= 1 is max(0, sum c_lm Y_lm(dir) + 0.5)
 *     with real orthonormal SH (Condon-Shortley phase), dir = mu - camera centre;
 *   - depth order: ascending camera depth, ties by Gaussian index;
 *   - NCC over all 3*H*W samples as one vector with one mean each (or, with
 *     the P_NCC_GRAY parameter, over the H*W gray values (R + G + B) / 3).
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC (no fast-math: IEEE FP64 throughout).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- parameter vector (double[16]) --------------------------------------- */
enum {
    P_NEAR = 0, P_FOV_CLAMP, P_EPS2D, P_ALPHA_MIN, P_ALPHA_MAX, P_T_MIN, P_CUT,
    P_TILE_W, P_TILE_H,
    P_FLAG_POWER, P_FLAG_ALPHA, P_FLAG_T, P_FLAG_DEPTH, P_FLAG_SIG, P_FLAG_POS,
    P_NCC_GRAY,           /* != 0: NCC over the gray values (R + G + B) / 3 */
    P_COUNT = 16
};

/* ---- camera vector (double[6]): width, height, fx, fy, cx, cy ------------- */
enum { C_W = 0, C_H, C_FX, C_FY, C_CX, C_CY };

/* ---- projected record (double[OR_REC]) ------------------------------------ */
enum {
    R_VISIBLE = 0, R_U, R_V, R_DEPTH,
    R_COV_A, R_COV_B, R_COV_C,           /* Sigma' (dilated): [[a, b], [b, c]] */
    R_CON_A, R_CON_B, R_CON_C,           /* inverse of Sigma'                  */
    R_RX, R_RY,                          /* cut * sqrt(Sigma'_xx), ... (px)    */
    R_RED, R_GREEN, R_BLUE, R_OPACITY,
    R_TX0, R_TY0, R_TX1, R_TY1,          /* inclusive tile rectangle           */
    R_DET_UNDIL, R_DET, R_TCX, R_TCY,    /* undilated det, det, camera x, y    */
    OR_REC
};

int or_rec_stride(void) { return OR_REC; }
int or_param_count(void) { return P_COUNT; }
int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ========================================================================= */
/* Rotation from a quaternion (w, x, y, z), normalised first.  Sec. III-A.   */
/* ========================================================================= */
void or_quat_to_rot(const double qin[4], double R[9])
{
    double n = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
    double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* ========================================================================= */
/* Real orthonormal spherical harmonics, any degree, from their definition:   */
/*   Y_l0  = K_l0 P_l^0(z)                                                   */
/*   Y_lm  = sqrt2 K_lm cos(m phi) P_l^m(z)     (m > 0)                      */
/*   Y_l-m = sqrt2 K_lm sin(m phi) P_l^m(z)     (m > 0)                      */
/*   K_lm  = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)                               */
/* with P_l^m the associated Legendre functions including (-1)^m.  For a unit */
/* direction, cos(m phi) sin^m(theta) = Re((x+iy)^m) and likewise Im for sin, */
/* so P_l^m / sin^m(theta) is a polynomial in z obtained by the usual         */
/* three-term recurrence.  Output index: l*l + l + m.                         */
/* ========================================================================= */
static double factorial(int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; }

void or_sh_basis(int deg, const double d[3], double *Y)
{
    double re[8], im[8];          /* (x + i y)^m */
    re[0] = 1; im[0] = 0;
    for (int m = 1; m <= deg; ++m) {
        re[m] = re[m - 1] * d[0] - im[m - 1] * d[1];
        im[m] = re[m - 1] * d[1] + im[m - 1] * d[0];
    }
    double z = d[2];
    for (int m = 0; m <= deg; ++m) {
        /* Ptilde_m^m = (-1)^m (2m-1)!! */
        double pmm = 1;
        for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1);
        double p_prev2 = 0, p_prev = 0;
        for (int l = m; l <= deg; ++l) {
            double p;
            if (l == m) p = pmm;
            else if (l == m + 1) p = z * (2 * m + 1) * pmm;
            else p = ((2 * l - 1) * z * p_prev - (l + m - 1) * p_prev2) / (l - m);
            p_prev2 = p_prev; p_prev = p;
            double K = sqrt((2 * l + 1) / (4 * M_PI) * factorial(l - m) / factorial(l + m));
            if (m == 0) {
                Y[l * l + l] = K * p;
            } else {
                Y[l * l + l + m] = sqrt(2.0) * K * re[m] * p;
                Y[l * l + l - m] = sqrt(2.0) * K * im[m] * p;
            }
        }
    }
}

/* ========================================================================= */
/* Projection of one Gaussian for one camera (Eqs. proj, foot_conv).          */
/* ========================================================================= */
static void project_one(const float *mean, const float *scale, const float *quat, float opac,
                        const float *sh, int sh_deg, const double *Wm, const double *cam,
                        const double *p, double *rec)
{
    memset(rec, 0, sizeof(double) * OR_REC);
    const double Rw[9] = {Wm[0], Wm[1], Wm[2], Wm[4], Wm[5], Wm[6], Wm[8], Wm[9], Wm[10]};
    const double tw[3] = {Wm[3], Wm[7], Wm[11]};
    const double mu[3] = {mean[0], mean[1], mean[2]};
    double t[3];
    for (int i = 0; i < 3; ++i) t[i] = Rw[3 * i] * mu[0] + Rw[3 * i + 1] * mu[1] + Rw[3 * i + 2] * mu[2] + tw[i];
    rec[R_DEPTH] = t[2];
    rec[R_TCX] = t[0];
    rec[R_TCY] = t[1];
    if (!(t[2] > p[P_NEAR])) return;

    /* 3D covariance Sigma = (R S)(R S)^T */
    double q[4] = {quat[0], quat[1], quat[2], quat[3]}, R[9], M[9], S3[9];
    or_quat_to_rot(q, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * (double)scale[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S3[3 * i + j] = M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2];

    /* Jacobian of the pinhole projection at t (FOV clamp applied in J only) */
    const double fx = cam[C_FX], fy = cam[C_FY];
    double limx = p[P_FOV_CLAMP] * (0.5 * cam[C_W]) / fx;
    double limy = p[P_FOV_CLAMP] * (0.5 * cam[C_H]) / fy;
    double xz = t[0] / t[2], yz = t[1] / t[2];
    if (xz < -limx) xz = -limx; if (xz > limx) xz = limx;
    if (yz < -limy) yz = -limy; if (yz > limy) yz = limy;
    double J[6] = {fx / t[2], 0, -fx * xz / t[2],
                   0, fy / t[2], -fy * yz / t[2]};
    /* T = J W_R  (2x3);  Sigma' = T Sigma T^T */
    double T[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = J[3 * i] * Rw[j] + J[3 * i + 1] * Rw[3 + j] + J[3 * i + 2] * Rw[6 + j];
    double TS[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            TS[3 * i + j] = T[3 * i] * S3[j] + T[3 * i + 1] * S3[3 + j] + T[3 * i + 2] * S3[6 + j];
    double c00 = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2];
    double c01 = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    double c11 = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5];
    rec[R_DET_UNDIL] = c00 * c11 - c01 * c01;
    double a = c00 + p[P_EPS2D], b = c01, c = c11 + p[P_EPS2D];
    double det = a * c - b * b;
    rec[R_COV_A] = a; rec[R_COV_B] = b; rec[R_COV_C] = c; rec[R_DET] = det;
    if (!(det > 0)) return;
    rec[R_CON_A] = c / det; rec[R_CON_B] = -b / det; rec[R_CON_C] = a / det;

    /* projected mean m(mu) */
    double u = fx * t[0] / t[2] + cam[C_CX];
    double v = fy * t[1] / t[2] + cam[C_CY];
    double rx = p[P_CUT] * sqrt(a), ry = p[P_CUT] * sqrt(c);
    rec[R_U] = u; rec[R_V] = v; rec[R_RX] = rx; rec[R_RY] = ry;

    /* conservative tile rectangle of the cut-sigma box */
    const int width = (int)cam[C_W], height = (int)cam[C_H];
    const int tw_ = (int)p[P_TILE_W], th_ = (int)p[P_TILE_H];
    const int ntx = (width + tw_ - 1) / tw_, nty = (height + th_ - 1) / th_;
    double xlo = u - rx, xhi = u + rx, ylo = v - ry, yhi = v + ry;
    if (xhi < 0 || xlo >= width || yhi < 0 || ylo >= height) return;
    int tx0 = (int)floor(xlo / tw_), tx1 = (int)floor(xhi / tw_);
    int ty0 = (int)floor(ylo / th_), ty1 = (int)floor(yhi / th_);
    if (tx0 < 0) tx0 = 0; if (ty0 < 0) ty0 = 0;
    if (tx1 > ntx - 1) tx1 = ntx - 1; if (ty1 > nty - 1) ty1 = nty - 1;
    rec[R_TX0] = tx0; rec[R_TY0] = ty0; rec[R_TX1] = tx1; rec[R_TY1] = ty1;

    /* colour */
    if (sh_deg == 0) {
        rec[R_RED] = sh[0]; rec[R_GREEN] = sh[1]; rec[R_BLUE] = sh[2];
    } else {
        /* camera centre C = -R_w^T t_w;  dir = normalise(mu - C) */
        double C[3];
        for (int i = 0; i < 3; ++i) C[i] = -(Rw[i] * tw[0] + Rw[3 + i] * tw[1] + Rw[6 + i] * tw[2]);
        double d[3] = {mu[0] - C[0], mu[1] - C[1], mu[2] - C[2]};
        double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        d[0] /= nd; d[1] /= nd; d[2] /= nd;
        double Y[64];
        or_sh_basis(sh_deg, d, Y);
        int K = (sh_deg + 1) * (sh_deg + 1);
        for (int ch = 0; ch < 3; ++ch) {
            double s = 0;
            for (int k = 0; k < K; ++k) s += (double)sh[3 * k + ch] * Y[k];
            s += 0.5;
            rec[R_RED + ch] = s > 0 ? s : 0;
        }
    }
    rec[R_OPACITY] = opac;
    rec[R_VISIBLE] = 1;
}

/* Project n Gaussians for one camera pose W (row-major 4x4, world-to-camera). */
void or_project(const float *means, const float *scales, const float *quats, const float *opac,
                const float *sh, int sh_deg, int64_t n, const double *W, const double *cam,
                const double *params, double *recs)
{
    const int K = (sh_deg + 1) * (sh_deg + 1);
    for (int64_t i = 0; i < n; ++i)
        project_one(means + 3 * i, scales + 3 * i, quats + 4 * i, opac[i], sh + (int64_t)3 * K * i,
                    sh_deg, W, cam, params, recs + (int64_t)OR_REC * i);
}

/* ========================================================================= */
/* Stable merge sorts.                                                        */
/* ========================================================================= */
static void msort_by_double(int64_t *idx, int64_t *tmp, int64_t n, const double *key)
{
    if (n < 2) return;
    int64_t h = n / 2;
    msort_by_double(idx, tmp, h, key);
    msort_by_double(idx + h, tmp, n - h, key);
    int64_t i = 0, j = h, k = 0;
    while (i < h && j < n) {
        if (key[idx[j]] < key[idx[i]]) tmp[k++] = idx[j++];   /* equal: left first */
        else tmp[k++] = idx[i++];
    }
    while (i < h) tmp[k++] = idx[i++];
    while (j < n) tmp[k++] = idx[j++];
    memcpy(idx, tmp, sizeof(int64_t) * n);
}

static void msort_u64(uint64_t *k, uint32_t *v, uint64_t *tk, uint32_t *tv, int64_t n)
{
    if (n < 2) return;
    int64_t h = n / 2;
    msort_u64(k, v, tk, tv, h);
    msort_u64(k + h, v + h, tk, tv, n - h);
    int64_t i = 0, j = h, o = 0;
    while (i < h && j < n) {
        if (k[j] < k[i]) { tk[o] = k[j]; tv[o++] = v[j++]; }
        else { tk[o] = k[i]; tv[o++] = v[i++]; }
    }
    while (i < h) { tk[o] = k[i]; tv[o++] = v[i++]; }
    while (j < n) { tk[o] = k[j]; tv[o++] = v[j++]; }
    memcpy(k, tk, sizeof(uint64_t) * n);
    memcpy(v, tv, sizeof(uint32_t) * n);
}

void or_stable_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n)
{
    if (n < 2) return;
    uint64_t *tk = (uint64_t *)malloc(sizeof(uint64_t) * n);
    uint32_t *tv = (uint32_t *)malloc(sizeof(uint32_t) * n);
    msort_u64(keys, vals, tk, tv, n);
    free(tk); free(tv);
}

/* O(n^2) insertion sort: the plain definition of a stable sort (pins the above). */
void or_insertion_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n)
{
    for (int64_t i = 1; i < n; ++i) {
        uint64_t k = keys[i]; uint32_t v = vals[i];
        int64_t j = i - 1;
        while (j >= 0 && keys[j] > k) { keys[j + 1] = keys[j]; vals[j + 1] = vals[j]; --j; }
        keys[j + 1] = k; vals[j + 1] = v;
    }
}

/* ========================================================================= */
/* Front-to-back compositing of RGB and depth (Sec. III-A).                   */
/* recs: projected records of n Gaussians (index order = tie order).          */
/* brute != 0: every pixel tests every visible Gaussian (pins the splat form). */
/*                                                                            */
/* Flags mark pixels where an FP32 evaluation may take a different branch     */
/* than this FP64 one AND the branch matters.  A decision taken the other way */
/* at a footprint or alpha-skip edge moves the pixel by at most ~2 alpha T;   */
/* swapping two consecutive contributors of near-equal depth moves colour by  */
/* T_prev alpha_prev alpha |c - c_prev| (depth and alpha are unchanged); so a */
/* band hit is flagged only when that effect reaches P_FLAG_SIG.  The band   */
/* of the footprint test is P_FLAG_POWER |lim| plus the change of the power   */
/* under a shift of P_FLAG_POS pixels of the projected mean (its gradient).   */
/*   bit 1: footprint boundary, 2: alpha-skip boundary, 4: stop boundary,     */
/*   8: depth near-tie between consecutive contributors (or the stopper).     */
/* ========================================================================= */
typedef struct {
    double T, r, g, b, d;
    double last_z, last_T, last_a, last_c[3];
    int done, any;
} pix_state;

static inline void composite(pix_state *s, const double *rc, double px, double py,
                             const double *p, uint8_t *flag, double *bnd, int64_t *n_eval)
{
    if (s->done) return;
    double dx = px - rc[R_U], dy = py - rc[R_V];
    double power = -0.5 * (rc[R_CON_A] * dx * dx + rc[R_CON_C] * dy * dy) - rc[R_CON_B] * dx * dy;
    double lim = -0.5 * p[P_CUT] * p[P_CUT];
    const double sig = p[P_FLAG_SIG];
    const double gx = rc[R_CON_A] * dx + rc[R_CON_B] * dy, gy = rc[R_CON_B] * dx + rc[R_CON_C] * dy;
    const double band = p[P_FLAG_POWER] * fabs(lim) + p[P_FLAG_POS] * (fabs(gx) + fabs(gy));
    if (fabs(power - lim) <= band) {
        /* including or dropping this Gaussian moves the pixel by <= 2 alpha T */
        double e = 2 * s->T * fmin(p[P_ALPHA_MAX], rc[R_OPACITY] * exp(power));
        if (e >= sig) { *flag |= 1; *bnd += e; }
    }
    if (power < lim) return;
    (*n_eval)++;
    double raw = rc[R_OPACITY] * exp(power);
    double alpha = raw < p[P_ALPHA_MAX] ? raw : p[P_ALPHA_MAX];
    if (fabs(raw - p[P_ALPHA_MIN]) <= (p[P_FLAG_ALPHA] + band) * p[P_ALPHA_MIN]) {
        double e = 2 * s->T * raw;
        if (e >= sig) { *flag |= 2; *bnd += e; }
    }
    if (alpha < p[P_ALPHA_MIN]) return;
    double tn = s->T * (1 - alpha);
    /* stopping one Gaussian earlier or later moves the pixel by <= T */
    if (fabs(tn - p[P_T_MIN]) <= p[P_FLAG_T] * p[P_T_MIN]) { *flag |= 4; *bnd += s->T; }
    double z = rc[R_DEPTH];
    const double col[3] = {rc[R_RED], rc[R_GREEN], rc[R_BLUE]};
    int tie = s->any && fabs(z - s->last_z) <= p[P_FLAG_DEPTH] * fabs(z);
    if (tn < p[P_T_MIN]) {
        if (tie) {
            double e = 2 * s->last_T * fmax(s->last_a, alpha);
            if (e >= sig) { *flag |= 8; *bnd += e; }
        }
        s->done = 1;
        return;
    }
    if (tie) {
        /* swapping two consecutive contributors changes colour by exactly
           T_prev alpha_prev alpha (c - c_prev); T afterwards is unchanged */
        double dc = 0;
        for (int k = 0; k < 3; ++k) dc = fmax(dc, fabs(col[k] - s->last_c[k]));
        double e = s->last_T * s->last_a * alpha * dc;
        if (e >= sig) { *flag |= 8; *bnd += e; }
    }
    double w = alpha * s->T;
    s->r += col[0] * w; s->g += col[1] * w; s->b += col[2] * w;
    s->d += z * w;
    s->last_T = s->T; s->last_a = alpha;
    s->last_c[0] = col[0]; s->last_c[1] = col[1]; s->last_c[2] = col[2];
    s->T = tn; s->last_z = z; s->any = 1;
}

int64_t or_render(const double *recs, int64_t n, const double *cam, const double *p,
                  double *rgb, double *depth, double *alpha, uint8_t *flags, double *bound, int brute)
{
    const int W = (int)cam[C_W], H = (int)cam[C_H];
    const int64_t npx = (int64_t)W * H;
    int64_t nvis = 0;
    for (int64_t i = 0; i < n; ++i) nvis += recs[OR_REC * i + R_VISIBLE] != 0;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (nvis + 1));
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (nvis + 1));
    double *zkey = (double *)malloc(sizeof(double) * (n + 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        zkey[i] = recs[OR_REC * i + R_DEPTH];
        if (recs[OR_REC * i + R_VISIBLE] != 0) order[k++] = i;
    }
    msort_by_double(order, tmp, nvis, zkey);   /* depth ascending, ties by index */

    pix_state *st = (pix_state *)calloc(npx, sizeof(pix_state));
    uint8_t *fl = (uint8_t *)calloc(npx, 1);
    double *bd = (double *)calloc(npx, sizeof(double));
    for (int64_t q = 0; q < npx; ++q) st[q].T = 1;
    int64_t n_eval = 0;
    if (brute) {
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int64_t j = 0; j < nvis; ++j)
                    composite(&st[(int64_t)y * W + x], recs + OR_REC * order[j], x + 0.5, y + 0.5, p,
                              &fl[(int64_t)y * W + x], &bd[(int64_t)y * W + x], &n_eval);
    } else {
        for (int64_t j = 0; j < nvis; ++j) {
            const double *rc = recs + OR_REC * order[j];
            /* every pixel whose centre can lie inside the cut-sigma ellipse */
            int x0 = (int)floor(rc[R_U] - rc[R_RX] - 1), x1 = (int)ceil(rc[R_U] + rc[R_RX]);
            int y0 = (int)floor(rc[R_V] - rc[R_RY] - 1), y1 = (int)ceil(rc[R_V] + rc[R_RY]);
            if (x0 < 0) x0 = 0; if (y0 < 0) y0 = 0;
            if (x1 > W - 1) x1 = W - 1; if (y1 > H - 1) y1 = H - 1;
            for (int y = y0; y <= y1; ++y)
                for (int x = x0; x <= x1; ++x)
                    composite(&st[(int64_t)y * W + x], rc, x + 0.5, y + 0.5, p,
                              &fl[(int64_t)y * W + x], &bd[(int64_t)y * W + x], &n_eval);
        }
    }
    for (int64_t q = 0; q < npx; ++q) {
        if (rgb) { rgb[q] = st[q].r; rgb[npx + q] = st[q].g; rgb[2 * npx + q] = st[q].b; }
        if (depth) depth[q] = st[q].d;
        if (alpha) alpha[q] = 1 - st[q].T;
        if (flags) flags[q] = fl[q];
        if (bound) bound[q] = bd[q];
    }
    free(st); free(fl); free(bd); free(order); free(tmp); free(zkey);
    return n_eval;
}

/* ========================================================================= */
/* NCC (Eq. ncc), two-pass: means first, then centred sums.                   */
/* Returns 0 and sets *degenerate when either centred sum of squares is       */
/* <= 1e-12 * n (zero-variance image: NCC undefined).                         */
/* ========================================================================= */
double or_ncc(const double *a, const double *b, int64_t n, int *degenerate)
{
    double ma = 0, mb = 0;
    for (int64_t i = 0; i < n; ++i) { ma += a[i]; mb += b[i]; }
    ma /= n; mb /= n;
    double sab = 0, saa = 0, sbb = 0;
    for (int64_t i = 0; i < n; ++i) {
        double da = a[i] - ma, db = b[i] - mb;
        sab += da * db; saa += da * da; sbb += db * db;
    }
    if (degenerate) *degenerate = 0;
    if (saa <= 1e-12 * n || sbb <= 1e-12 * n) { if (degenerate) *degenerate = 1; return 0; }
    return sab / (sqrt(saa) * sqrt(sbb));
}

/* Argmax with the lowest index on ties. */
int or_argmax(const double *s, int n)
{
    int best = 0;
    for (int i = 1; i < n; ++i) if (s[i] > s[best]) best = i;
    return best;
}

/* ========================================================================= */
/* Candidate grid around a coarse pose (Sec. III-C.1; Sec. IV-A grid).        */
/* Offsets (dx, dy) in the world ground plane and a yaw about world z through */
/* the camera centre; height, pitch and roll are the seed's.                  */
/* Candidate index = ix + nx * (iy + ny * iyaw); offsets centred on zero.     */
/* ========================================================================= */
void or_grid_poses(const double *seed, int nx, int ny, int nyaw, double step_xy,
                   double step_yaw_deg, double *out)
{
    const double R[9] = {seed[0], seed[1], seed[2], seed[4], seed[5], seed[6], seed[8], seed[9], seed[10]};
    const double t[3] = {seed[3], seed[7], seed[11]};
    double C[3];
    for (int i = 0; i < 3; ++i) C[i] = -(R[i] * t[0] + R[3 + i] * t[1] + R[6 + i] * t[2]);
    for (int iyaw = 0; iyaw < nyaw; ++iyaw)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int k = ix + nx * (iy + ny * iyaw);
                double dx = (ix - 0.5 * (nx - 1)) * step_xy;
                double dy = (iy - 0.5 * (ny - 1)) * step_xy;
                double psi = (iyaw - 0.5 * (nyaw - 1)) * step_yaw_deg * M_PI / 180.0;
                /* camera-to-world rotation Rcw' = Rz(psi) R^T, so R' = R Rz(psi)^T */
                double Rz[9] = {cos(psi), -sin(psi), 0, sin(psi), cos(psi), 0, 0, 0, 1};
                double Rn[9];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        Rn[3 * i + j] = R[3 * i] * Rz[3 * j] + R[3 * i + 1] * Rz[3 * j + 1] + R[3 * i + 2] * Rz[3 * j + 2];
                double Cn[3] = {C[0] + dx, C[1] + dy, C[2]};
                double *o = out + 16 * k;
                for (int i = 0; i < 3; ++i) {
                    o[4 * i] = Rn[3 * i]; o[4 * i + 1] = Rn[3 * i + 1]; o[4 * i + 2] = Rn[3 * i + 2];
                    o[4 * i + 3] = -(Rn[3 * i] * Cn[0] + Rn[3 * i + 1] * Cn[1] + Rn[3 * i + 2] * Cn[2]);
                }
                o[12] = 0; o[13] = 0; o[14] = 0; o[15] = 1;
            }
}

/* ========================================================================= */
/* Random search of Sec. IV-A: the order in which grid cells are visited.     */
/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the state advances by     */
/* the odd constant 0x9E3779B97F4A7C15 and each output is the new state mixed */
/* by xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31.  The      */
/* cells 0..n-1 are shuffled by Fisher-Yates: for i = n-1 down to 1, draw the */
/* next output x and swap cells i and x mod (i + 1).                          */
/* ========================================================================= */
static uint64_t or_sm64_next(uint64_t *state)
{
    uint64_t x = *state + 0x9E3779B97F4A7C15ULL;
    *state = x;
    x ^= x >> 30; x *= 0xBF58476D1CE4E5B9ULL;
    x ^= x >> 27; x *= 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

void or_splitmix64(uint64_t seed, int64_t count, uint64_t *out)
{
    uint64_t st = seed;
    for (int64_t k = 0; k < count; ++k) out[k] = or_sm64_next(&st);
}

void or_search_order(uint64_t seed, int64_t n, int32_t *cells)
{
    uint64_t st = seed;
    for (int64_t i = 0; i < n; ++i) cells[i] = (int32_t)i;
    for (int64_t i = n - 1; i >= 1; --i) {
        const int64_t j = (int64_t)(or_sm64_next(&st) % (uint64_t)(i + 1));
        const int32_t t = cells[i]; cells[i] = cells[j]; cells[j] = t;
    }
}

/* ========================================================================= */
/* 2D voxel blocks (Sec. III-B.2): block (floor(x/B), floor(y/B)); the map is */
/* ordered by block key (bx, by) ascending, Gaussians of a block in index     */
/* order.  Selection (Sec. III-C.1): every block whose centre lies within     */
/* radius of (cx, cy), by a plain distance scan.  Writes the selected          */
/* Gaussians' original indices in that order; returns their count.            */
/* ========================================================================= */
typedef struct { int64_t bx, by, idx; } blk_item;
static int cmp_blk(const void *a, const void *b)
{
    const blk_item *x = (const blk_item *)a, *y = (const blk_item *)b;
    if (x->bx != y->bx) return x->bx < y->bx ? -1 : 1;
    if (x->by != y->by) return x->by < y->by ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);   /* index order inside a block */
}

int64_t or_block_select(const float *means, int64_t n, double B, double cx, double cy, double radius,
                        int64_t *out_idx, int64_t *out_nblocks)
{
    blk_item *it = (blk_item *)malloc(sizeof(blk_item) * (n + 1));
    for (int64_t i = 0; i < n; ++i) {
        it[i].bx = (int64_t)floor(means[3 * i] / B);
        it[i].by = (int64_t)floor(means[3 * i + 1] / B);
        it[i].idx = i;
    }
    qsort(it, n, sizeof(blk_item), cmp_blk);
    int64_t cnt = 0, nb = 0;
    for (int64_t i = 0; i < n;) {
        int64_t j = i;
        while (j < n && it[j].bx == it[i].bx && it[j].by == it[i].by) ++j;
        double ccx = (it[i].bx + 0.5) * B, ccy = (it[i].by + 0.5) * B;
        double dd = sqrt((ccx - cx) * (ccx - cx) + (ccy - cy) * (ccy - cy));
        if (dd <= radius) {
            ++nb;
            for (int64_t k = i; k < j; ++k) { if (out_idx) out_idx[cnt] = it[k].idx; ++cnt; }
        }
        i = j;
    }
    if (out_nblocks) *out_nblocks = nb;
    free(it);
    return cnt;
}

/* ========================================================================= */
/* Tile|depth key replay (integer logic only).  Inputs per (view, Gaussian):  */
/* visibility, float32 depth bit pattern and inclusive tile rectangle, as the */
/* GPU recorded them.  Emits one (key, value) per covered tile in view-major, */
/* Gaussian-index order:                                                      */
/*   key = view << (32 + tile_bits) | tile << 32 | depth_bits, value = index  */
/* tile = ty * ntx + tx; tile_bits = bits needed for ntx*nty - 1.             */
/* keys == NULL: count only.                                                  */
/* ========================================================================= */
int or_tile_bits(int n_tiles)
{
    int b = 0;
    while ((1LL << b) < n_tiles) ++b;
    return b;
}

int64_t or_tile_keys(int n_views, int64_t n, const uint8_t *vis, const uint32_t *dbits,
                     const int32_t *rect, int ntx, int nty, uint64_t *keys, uint32_t *vals)
{
    int tb = or_tile_bits(ntx * nty);
    int64_t o = 0;
    for (int v = 0; v < n_views; ++v)
        for (int64_t i = 0; i < n; ++i) {
            int64_t q = (int64_t)v * n + i;
            if (!vis[q]) continue;
            const int32_t *r = rect + 4 * q;
            for (int ty = r[1]; ty <= r[3]; ++ty)
                for (int tx = r[0]; tx <= r[2]; ++tx) {
                    if (keys) {
                        uint64_t tile = (uint64_t)(ty * ntx + tx);
                        keys[o] = ((uint64_t)v << (32 + tb)) | (tile << 32) | (uint64_t)dbits[q];
                        vals[o] = (uint32_t)i;
                    }
                    ++o;
                }
        }
    return o;
}

/* [begin, end) of every (view, tile) in a sorted key list; empty = [0, 0). */
void or_tile_ranges(const uint64_t *keys, int64_t n, int n_views, int n_tiles, int64_t *ranges)
{
    int tb = or_tile_bits(n_tiles);
    memset(ranges, 0, sizeof(int64_t) * 2 * (int64_t)n_views * n_tiles);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t vt = keys[i] >> 32;
        int64_t v = (int64_t)(vt >> tb), t = (int64_t)(vt & ((1ULL << tb) - 1));
        int64_t slot = v * n_tiles + t;
        if (i == 0 || (keys[i - 1] >> 32) != vt) ranges[2 * slot] = i;
        if (i == n - 1 || (keys[i + 1] >> 32) != vt) ranges[2 * slot + 1] = i + 1;
    }
}

/* ========================================================================= */
/* Whole views: project + composite + NCC for V poses, in parallel over views. */
/* query: 3*H*W doubles or NULL (then scores are not computed).               */
/* Optional outputs (NULL = skip): images per view, flags, and counts per     */
/* view {n_visible, n_instances (tile rectangle sizes), n_eval}.             */
/* ========================================================================= */
void or_render_views(const float *means, const float *scales, const float *quats, const float *opac,
                     const float *sh, int sh_deg, int64_t n, const double *poses, int n_views,
                     const double *cam, const double *p, const double *query,
                     double *scores, int *degenerate, double *rgb, double *depth, double *alpha,
                     uint8_t *flags, double *bound, int64_t *counts)
{
    const int W = (int)cam[C_W], H = (int)cam[C_H];
    const int64_t npx = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < n_views; ++v) {
        double *recs = (double *)malloc(sizeof(double) * OR_REC * (n + 1));
        or_project(means, scales, quats, opac, sh, sh_deg, n, poses + 16 * v, cam, p, recs);
        double *img = rgb ? rgb + 3 * npx * v : (double *)malloc(sizeof(double) * 3 * npx);
        int64_t ne = or_render(recs, n, cam, p, img, depth ? depth + npx * v : NULL,
                               alpha ? alpha + npx * v : NULL, flags ? flags + npx * v : NULL,
                               bound ? bound + npx * v : NULL, 0);
        if (counts) {
            int64_t nv = 0, ni = 0;
            for (int64_t i = 0; i < n; ++i) {
                const double *r = recs + OR_REC * i;
                if (r[R_VISIBLE] == 0) continue;
                ++nv;
                ni += (int64_t)(r[R_TX1] - r[R_TX0] + 1) * (int64_t)(r[R_TY1] - r[R_TY0] + 1);
            }
            counts[3 * v] = nv; counts[3 * v + 1] = ni; counts[3 * v + 2] = ne;
        }
        if (query && scores) {
            int dg = 0;
            if (p[P_NCC_GRAY] != 0) {
                double *gi = (double *)malloc(sizeof(double) * (npx + 1)), *gq = (double *)malloc(sizeof(double) * (npx + 1));
                for (int64_t k = 0; k < npx; ++k) {
                    gi[k] = (img[k] + img[npx + k] + img[2 * npx + k]) / 3.0;
                    gq[k] = (query[k] + query[npx + k] + query[2 * npx + k]) / 3.0;
                }
                scores[v] = or_ncc(gi, gq, npx, &dg);
                free(gi); free(gq);
            } else {
                scores[v] = or_ncc(img, query, 3 * npx, &dg);
            }
            if (degenerate) degenerate[v] = dg;
        }
        if (!rgb) free(img);
        free(recs);
    }
}

/* ========================================================================= */
/* Pose refinement of Sec. III-C.2 (the PnP step; the matcher is an input):   */
/* back-project render pixels with the view's depth D / A (bilinear at        */
/* (u - 0.5, v - 0.5)), then minimise sum_i huber(|pi(W X_i) - q_i|) over the */
/* world-to-camera pose W by reweighted Gauss-Newton: the update (rho, phi)   */
/* acts on the left, P' = Exp(phi) P + rho for camera points P = R X + t.    */
/* ========================================================================= */
static double or_bilinear(const float *img, int W, double sx, double sy)
{
    const int x0 = (int)floor(sx), y0 = (int)floor(sy);
    const double ax = sx - x0, ay = sy - y0;
    const double a = img[(int64_t)y0 * W + x0], b = img[(int64_t)y0 * W + x0 + 1];
    const double c = img[(int64_t)(y0 + 1) * W + x0], d = img[(int64_t)(y0 + 1) * W + x0 + 1];
    return (1.0 - ay) * ((1.0 - ax) * a + ax * b) + ay * ((1.0 - ax) * c + ax * d);
}

/* Rodrigues: Exp(phi) = I + sin(th)/th K + (1 - cos(th))/th^2 K^2. */
static void or_so3_exp(const double phi[3], double E[9])
{
    const double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    const double K[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            K2[3 * i + j] = 0;
            for (int m = 0; m < 3; ++m) K2[3 * i + j] += K[3 * i + m] * K[3 * m + j];
        }
    double s1, s2;
    if (th < 1e-8) { s1 = 1.0 - th * th / 6.0; s2 = 0.5 - th * th / 24.0; }
    else { s1 = sin(th) / th; s2 = (1.0 - cos(th)) / (th * th); }
    for (int i = 0; i < 9; ++i) E[i] = (i % 4 == 0 ? 1.0 : 0.0) + s1 * K[i] + s2 * K2[i];
}

/* pose (4x4 row-major) updated by s * delta on the left. */
void or_pnp_apply(const double *pose, const double *delta, double s, double *out)
{
    const double phi[3] = {s * delta[3], s * delta[4], s * delta[5]};
    double E[9];
    or_so3_exp(phi, E);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 4; ++j) {
            double v = 0;
            for (int m = 0; m < 3; ++m) v += E[3 * i + m] * pose[4 * m + j];
            out[4 * i + j] = v;
        }
        out[4 * i + 3] += s * delta[i];
    }
    out[12] = out[13] = out[14] = 0; out[15] = 1;
}

/* residual (2) and its Jacobian (2 x 6, row-major) w.r.t. (rho, phi) at 0. */
int or_pnp_residual(const double *pose, const double *X, const double *cam, const double *q, double *r, double *J)
{
    double P[3];
    for (int i = 0; i < 3; ++i) P[i] = pose[4 * i] * X[0] + pose[4 * i + 1] * X[1] + pose[4 * i + 2] * X[2] + pose[4 * i + 3];
    if (P[2] <= 1e-6) return 0;
    const double fx = cam[C_FX], fy = cam[C_FY];
    r[0] = fx * P[0] / P[2] + cam[C_CX] - q[0];
    r[1] = fy * P[1] / P[2] + cam[C_CY] - q[1];
    if (J) {
        /* d pixel / d P */
        const double Jp[6] = {fx / P[2], 0, -fx * P[0] / (P[2] * P[2]), 0, fy / P[2], -fy * P[1] / (P[2] * P[2])};
        /* d P / d (rho, phi) = [I | -[P]x] */
        const double M[18] = {1, 0, 0, 0, P[2], -P[1],
                              0, 1, 0, -P[2], 0, P[0],
                              0, 0, 1, P[1], -P[0], 0};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 6; ++b) {
                J[6 * a + b] = 0;
                for (int m = 0; m < 3; ++m) J[6 * a + b] += Jp[3 * a + m] * M[6 * m + b];
            }
    }
    return 1;
}

static double or_huber(double e, double k) { return e <= k ? 0.5 * e * e : k * (e - 0.5 * k); }

static double or_pnp_cost(const double *pose, const double *X, const uint8_t *use, const double *q, int64_t n,
                          const double *cam, double k, double *sq, int64_t *cnt)
{
    double c = 0, s2 = 0; int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!use[i]) continue;
        double r[2];
        if (!or_pnp_residual(pose, X + 3 * i, cam, q + 2 * i, r, NULL)) continue;
        const double e = sqrt(r[0] * r[0] + r[1] * r[1]);
        c += or_huber(e, k); s2 += e * e; ++m;
    }
    if (sq) *sq = s2;
    if (cnt) *cnt = m;
    return c;
}

/* Solve A x = b for a symmetric positive definite 6 x 6 A (Gaussian
 * elimination with partial pivoting; returns 0 if singular). */
static int or_solve6(double A[36], double b[6], double x[6])
{
    for (int c = 0; c < 6; ++c) {
        int p = c;
        for (int r = c + 1; r < 6; ++r) if (fabs(A[6 * r + c]) > fabs(A[6 * p + c])) p = r;
        if (fabs(A[6 * p + c]) < 1e-300) return 0;
        if (p != c) {
            for (int j = 0; j < 6; ++j) { double t = A[6 * c + j]; A[6 * c + j] = A[6 * p + j]; A[6 * p + j] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < 6; ++r) {
            const double f = A[6 * r + c] / A[6 * c + c];
            for (int j = c; j < 6; ++j) A[6 * r + j] -= f * A[6 * c + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = 5; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < 6; ++j) s -= A[6 * r + j] * x[j];
        x[r] = s / A[6 * r + r];
    }
    return 1;
}

/* World point of render pixel (u, v): use[i] = 0 when its 2 x 2 neighbourhood
 * leaves the image or the alpha there is below alpha_min.  Returns the count used. */
int64_t or_pnp_backproject(const double *pose_render, const double *cam, const float *depth, const float *alpha,
                           const double *uv, int64_t n, double alpha_min, double *X, uint8_t *use)
{
    const int W = (int)cam[C_W], H = (int)cam[C_H];
    int64_t n_used = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double u = uv[2 * i], v = uv[2 * i + 1];
        const double sx = u - 0.5, sy = v - 0.5;
        use[i] = 0;
        X[3 * i] = X[3 * i + 1] = X[3 * i + 2] = 0;
        if (!isfinite(sx) || !isfinite(sy)) continue;
        if (floor(sx) < 0 || floor(sy) < 0 || floor(sx) + 1 >= W || floor(sy) + 1 >= H) continue;
        const double A = or_bilinear(alpha, W, sx, sy);
        if (A < alpha_min) continue;
        const double z = or_bilinear(depth, W, sx, sy) / A;
        const double Pc[3] = {z * (u - cam[C_CX]) / cam[C_FX], z * (v - cam[C_CY]) / cam[C_FY], z};
        /* X = R^T (P - t) */
        for (int k = 0; k < 3; ++k) {
            double s = 0;
            for (int m = 0; m < 3; ++m) s += pose_render[4 * m + k] * (Pc[m] - pose_render[4 * m + 3]);
            X[3 * i + k] = s;
        }
        use[i] = 1; ++n_used;
    }
    return n_used;
}

/* out[20]: pose[16], rms, cost, n_used, iterations. */
void or_refine_pnp(const double *pose_render, const double *pose_init, const double *cam, const float *depth,
                   const float *alpha, const float *pairs, int64_t n, int max_iters, double huber,
                   double alpha_min, double tol, double *out)
{
    double *X = (double *)calloc((size_t)(3 * n + 1), sizeof(double));
    double *q = (double *)calloc((size_t)(2 * n + 1), sizeof(double));
    double *uv = (double *)calloc((size_t)(2 * n + 1), sizeof(double));
    uint8_t *use = (uint8_t *)calloc((size_t)(n + 1), 1);
    for (int64_t i = 0; i < n; ++i) {
        uv[2 * i] = pairs[4 * i]; uv[2 * i + 1] = pairs[4 * i + 1];
        q[2 * i] = pairs[4 * i + 2]; q[2 * i + 1] = pairs[4 * i + 3];
    }
    int64_t n_used = or_pnp_backproject(pose_render, cam, depth, alpha, uv, n, alpha_min, X, use);
    for (int64_t i = 0; i < n; ++i)
        if (use[i] && !(isfinite(q[2 * i]) && isfinite(q[2 * i + 1]))) { use[i] = 0; --n_used; }
    double pose[16], trial[16];
    memcpy(pose, pose_init, sizeof pose);
    int it = 0;
    if (n_used >= 3) {
        for (; it < max_iters; ++it) {
            double Hm[36] = {0}, g[6] = {0};
            const double c0 = or_pnp_cost(pose, X, use, q, n, cam, huber, NULL, NULL);
            for (int64_t i = 0; i < n; ++i) {
                if (!use[i]) continue;
                double r[2], J[12];
                if (!or_pnp_residual(pose, X + 3 * i, cam, q + 2 * i, r, J)) continue;
                const double e = sqrt(r[0] * r[0] + r[1] * r[1]);
                const double w = e <= huber ? 1.0 : huber / e;
                for (int a = 0; a < 6; ++a) {
                    g[a] += w * (J[a] * r[0] + J[6 + a] * r[1]);
                    for (int b = 0; b < 6; ++b) Hm[6 * a + b] += w * (J[a] * J[b] + J[6 + a] * J[6 + b]);
                }
            }
            const double tr = Hm[0] + Hm[7] + Hm[14] + Hm[21] + Hm[28] + Hm[35];
            for (int a = 0; a < 6; ++a) { Hm[7 * a] += 1e-9 * tr / 6.0; g[a] = -g[a]; }
            double delta[6];
            if (!or_solve6(Hm, g, delta)) break;
            double s = 1.0;
            int ok = 0;
            for (int bt = 0; bt <= 10; ++bt) {
                or_pnp_apply(pose, delta, s, trial);
                if (or_pnp_cost(trial, X, use, q, n, cam, huber, NULL, NULL) < c0) { ok = 1; break; }
                s *= 0.5;
            }
            if (!ok) break;
            memcpy(pose, trial, sizeof pose);
            double dmax = 0;
            for (int a = 0; a < 6; ++a) dmax = fmax(dmax, fabs(s * delta[a]));
            if (dmax < tol) { ++it; break; }
        }
    }
    double sq = 0; int64_t cnt = 0;
    const double cost = or_pnp_cost(pose, X, use, q, n, cam, huber, &sq, &cnt);
    memcpy(out, pose, sizeof pose);
    out[16] = cnt ? sqrt(sq / (double)cnt) : 0.0;
    out[17] = cost;
    out[18] = (double)n_used;
    out[19] = (double)it;
    free(X); free(q); free(uv); free(use);
}

/* ========================================================================= */
/* NCC pose gradient (the paper's future direction: direct pose descent on   */
/* NCC), by forward-mode differentiation: every quantity of the projection,   */
/* compositing and NCC above is carried as a value plus its six derivatives  */
/* with respect to the pose update delta = (rho, phi), W(delta) =             */
/* [Exp(phi) R | Exp(phi) t + rho], at delta = 0.  Inclusion, alpha-skip,     */
/* clamp and stop decisions are taken on the values (the derivative of the    */
/* function with those decisions fixed).  Colour must be view-independent     */
/* (SH degree 0).                                                             */
/* ========================================================================= */
typedef struct { double v, d[6]; } dual;

static dual dk(double v) { dual r; r.v = v; for (int k = 0; k < 6; ++k) r.d[k] = 0; return r; }
static dual dadd(dual a, dual b) { for (int k = 0; k < 6; ++k) a.d[k] += b.d[k]; a.v += b.v; return a; }
static dual dsub(dual a, dual b) { for (int k = 0; k < 6; ++k) a.d[k] -= b.d[k]; a.v -= b.v; return a; }
static dual dmul(dual a, dual b)
{
    dual r; r.v = a.v * b.v;
    for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
static dual ddiv(dual a, dual b)
{
    dual r; r.v = a.v / b.v;
    for (int k = 0; k < 6; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
    return r;
}
static dual dscale(dual a, double s) { a.v *= s; for (int k = 0; k < 6; ++k) a.d[k] *= s; return a; }
static dual dexp(dual a) { dual r; r.v = exp(a.v); for (int k = 0; k < 6; ++k) r.d[k] = r.v * a.d[k]; return r; }
static dual dsqrt(dual a) { dual r; r.v = sqrt(a.v); for (int k = 0; k < 6; ++k) r.d[k] = a.d[k] / (2 * r.v); return r; }

typedef struct { dual u, v, A, B, C; double z, o, col[3], rx, ry; int vis; } drec;

/* Project one Gaussian (SH degree 0) as in project_one, in duals. */
static void dproject(const float *mu, const float *scale, const float *quat, float opac, const float *rgb,
                     const double *W, const double *cam, const double *p, drec *out)
{
    out->vis = 0;
    double Rw[9] = {W[0], W[1], W[2], W[4], W[5], W[6], W[8], W[9], W[10]};
    double tv[3];
    for (int i = 0; i < 3; ++i) tv[i] = Rw[3 * i] * mu[0] + Rw[3 * i + 1] * mu[1] + Rw[3 * i + 2] * mu[2] + W[4 * i + 3];
    if (!(tv[2] > p[P_NEAR])) return;
    /* t(delta) = Exp(phi) t + rho: d t / d rho_k = e_k, d t / d phi_k = e_k x t */
    dual t[3];
    for (int i = 0; i < 3; ++i) t[i] = dk(tv[i]);
    for (int k = 0; k < 3; ++k) t[k].d[k] = 1.0;
    t[1].d[3] = -tv[2]; t[2].d[3] = tv[1];        /* e_0 x t = (0, -t2, t1) */
    t[0].d[4] = tv[2];  t[2].d[4] = -tv[0];       /* e_1 x t = (t2, 0, -t0) */
    t[0].d[5] = -tv[1]; t[1].d[5] = tv[0];        /* e_2 x t = (-t1, t0, 0) */
    /* R(delta) = Exp(phi) R: d R / d phi_k = [e_k]x R */
    dual R[9];
    for (int i = 0; i < 9; ++i) R[i] = dk(Rw[i]);
    for (int k = 0; k < 3; ++k) {
        double E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};       /* [e_k]x */
        if (k == 0) { E[5] = -1; E[7] = 1; }
        if (k == 1) { E[2] = 1; E[6] = -1; }
        if (k == 2) { E[1] = -1; E[3] = 1; }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                R[3 * i + j].d[3 + k] = E[3 * i] * Rw[j] + E[3 * i + 1] * Rw[3 + j] + E[3 * i + 2] * Rw[6 + j];
    }
    double q[4] = {quat[0], quat[1], quat[2], quat[3]}, Rq[9], M[9], S3[9];
    or_quat_to_rot(q, Rq);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = Rq[3 * i + j] * (double)scale[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S3[3 * i + j] = M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2];
    const double fx = cam[C_FX], fy = cam[C_FY];
    const double limx = p[P_FOV_CLAMP] * (0.5 * cam[C_W]) / fx, limy = p[P_FOV_CLAMP] * (0.5 * cam[C_H]) / fy;
    dual xz = ddiv(t[0], t[2]), yz = ddiv(t[1], t[2]);
    if (xz.v < -limx) xz = dk(-limx); if (xz.v > limx) xz = dk(limx);
    if (yz.v < -limy) yz = dk(-limy); if (yz.v > limy) yz = dk(limy);
    dual J[6] = {ddiv(dk(fx), t[2]), dk(0), dscale(ddiv(xz, t[2]), -fx),
                 dk(0), ddiv(dk(fy), t[2]), dscale(ddiv(yz, t[2]), -fy)};
    dual T[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = dadd(dadd(dmul(J[3 * i], R[j]), dmul(J[3 * i + 1], R[3 + j])), dmul(J[3 * i + 2], R[6 + j]));
    dual TS[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            TS[3 * i + j] = dadd(dadd(dscale(T[3 * i], S3[j]), dscale(T[3 * i + 1], S3[3 + j])),
                                 dscale(T[3 * i + 2], S3[6 + j]));
    dual c00 = dadd(dadd(dmul(TS[0], T[0]), dmul(TS[1], T[1])), dmul(TS[2], T[2]));
    dual c01 = dadd(dadd(dmul(TS[0], T[3]), dmul(TS[1], T[4])), dmul(TS[2], T[5]));
    dual c11 = dadd(dadd(dmul(TS[3], T[3]), dmul(TS[4], T[4])), dmul(TS[5], T[5]));
    dual a = dadd(c00, dk(p[P_EPS2D])), b = c01, c = dadd(c11, dk(p[P_EPS2D]));
    dual det = dsub(dmul(a, c), dmul(b, b));
    if (!(det.v > 0)) return;
    out->A = ddiv(c, det); out->B = dscale(ddiv(b, det), -1.0); out->C = ddiv(a, det);
    out->u = dadd(dscale(ddiv(t[0], t[2]), fx), dk(cam[C_CX]));
    out->v = dadd(dscale(ddiv(t[1], t[2]), fy), dk(cam[C_CY]));
    out->rx = p[P_CUT] * sqrt(a.v); out->ry = p[P_CUT] * sqrt(c.v);
    const double W_ = cam[C_W], H_ = cam[C_H];
    if (out->u.v + out->rx < 0 || out->u.v - out->rx >= W_ || out->v.v + out->ry < 0 || out->v.v - out->ry >= H_) return;
    out->z = tv[2]; out->o = opac;
    out->col[0] = rgb[0]; out->col[1] = rgb[1]; out->col[2] = rgb[2];
    out->vis = 1;
}

typedef struct { dual T, c[3]; int done; } dpix;

/* out[7]: NCC and its six derivatives (rho_x, rho_y, rho_z, phi_x, phi_y, phi_z). */
void or_ncc_pose_grad(const float *means, const float *scales, const float *quats, const float *opac,
                      const float *rgb, int64_t n, const double *W, const double *cam, const double *p,
                      const double *query, double *out)
{
    const int Wd = (int)cam[C_W], Hd = (int)cam[C_H];
    const int64_t npx = (int64_t)Wd * Hd;
    drec *r = (drec *)malloc(sizeof(drec) * (n + 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    double *zkey = (double *)malloc(sizeof(double) * (n + 1));
    int64_t nv = 0;
    for (int64_t i = 0; i < n; ++i) {
        dproject(means + 3 * i, scales + 3 * i, quats + 4 * i, opac[i], rgb + 3 * i, W, cam, p, &r[i]);
        zkey[i] = r[i].vis ? r[i].z : 0;
        if (r[i].vis) order[nv++] = i;
    }
    msort_by_double(order, tmp, nv, zkey);
    dpix *px = (dpix *)malloc(sizeof(dpix) * npx);
    for (int64_t k = 0; k < npx; ++k) { px[k].T = dk(1.0); px[k].c[0] = px[k].c[1] = px[k].c[2] = dk(0); px[k].done = 0; }
    const double lim = -0.5 * p[P_CUT] * p[P_CUT];
    for (int64_t j = 0; j < nv; ++j) {
        const drec *g = &r[order[j]];
        int x0 = (int)floor(g->u.v - g->rx - 1), x1 = (int)ceil(g->u.v + g->rx);
        int y0 = (int)floor(g->v.v - g->ry - 1), y1 = (int)ceil(g->v.v + g->ry);
        if (x0 < 0) x0 = 0; if (y0 < 0) y0 = 0;
        if (x1 > Wd - 1) x1 = Wd - 1; if (y1 > Hd - 1) y1 = Hd - 1;
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                dpix *s = &px[(int64_t)y * Wd + x];
                if (s->done) continue;
                dual dx = dsub(dk(x + 0.5), g->u), dy = dsub(dk(y + 0.5), g->v);
                dual pw = dsub(dscale(dadd(dmul(g->A, dmul(dx, dx)), dmul(g->C, dmul(dy, dy))), -0.5),
                               dmul(g->B, dmul(dx, dy)));
                if (pw.v < lim) continue;
                dual raw = dscale(dexp(pw), g->o);
                dual al = raw.v < p[P_ALPHA_MAX] ? raw : dk(p[P_ALPHA_MAX]);
                if (al.v < p[P_ALPHA_MIN]) continue;
                dual tn = dmul(s->T, dsub(dk(1.0), al));
                if (tn.v < p[P_T_MIN]) { s->done = 1; continue; }
                dual w = dmul(al, s->T);
                for (int ch = 0; ch < 3; ++ch) s->c[ch] = dadd(s->c[ch], dscale(w, g->col[ch]));
                s->T = tn;
            }
    }
    /* NCC over all 3 H W samples (or the H W gray values), two-pass, in duals
     * (query constant) */
    const int gray = p[P_NCC_GRAY] != 0;
    const int nch = gray ? 1 : 3;
    const int64_t ns = nch * npx;
    dual *rs = (dual *)malloc(sizeof(dual) * (ns + 1));
    double *qs = (double *)malloc(sizeof(double) * (ns + 1));
    for (int ch = 0; ch < nch; ++ch)
        for (int64_t k = 0; k < npx; ++k) {
            if (gray) {
                rs[k] = dscale(dadd(dadd(px[k].c[0], px[k].c[1]), px[k].c[2]), 1.0 / 3.0);
                qs[k] = (query[k] + query[npx + k] + query[2 * npx + k]) / 3.0;
            } else {
                rs[ch * npx + k] = px[k].c[ch];
                qs[ch * npx + k] = query[ch * npx + k];
            }
        }
    dual mr = dk(0); double mq = 0;
    for (int64_t k = 0; k < ns; ++k) { mr = dadd(mr, rs[k]); mq += qs[k]; }
    mr = dscale(mr, 1.0 / ns); mq /= ns;
    dual sab = dk(0), saa = dk(0); double sbb = 0;
    for (int64_t k = 0; k < ns; ++k) {
        dual da = dsub(rs[k], mr);
        const double db = qs[k] - mq;
        sab = dadd(sab, dscale(da, db));
        saa = dadd(saa, dmul(da, da));
        sbb += db * db;
    }
    free(rs); free(qs);
    out[0] = 0;
    for (int k = 0; k < 6; ++k) out[1 + k] = 0;
    if (saa.v > 1e-12 * ns && sbb > 1e-12 * ns) {
        dual ncc = ddiv(sab, dscale(dsqrt(saa), sqrt(sbb)));
        out[0] = ncc.v;
        for (int k = 0; k < 6; ++k) out[1 + k] = ncc.d[k];
    }
    free(r); free(order); free(tmp); free(zkey); free(px);
}

/* ========================================================================= */
/* Map training loss (Sec. III-B.3): L = w_photo L_photo + w_reproj L_reproj */
/* with L_rgb(I1, I2) = (1 - lambda) L1(I1, I2) + lambda L_D-SSIM(I1, I2),    */
/* L1 the mean absolute difference over all 3 H W samples of a view (the     */
/* SSIM and re-projection parts follow below).                               */
/* Directional derivatives of the loss along six directions in               */
/* the space of all Gaussian parameters -- mean (3), scale (3), quaternion    */
/* (4), opacity (1), RGB (3): 14 per Gaussian, SH degree 0 -- by forward-mode */
/* duals through the same projection and compositing as above.               */
/* dirs: [n][14][6] tangents.  out: [7] = loss and its six derivatives.       */
/* ========================================================================= */
enum { NPAR = 14 };
typedef struct { dual u, v, A, B, C, o, col[3], zd; double z, rx, ry; int vis; } dprec;

static void dproject_params(const float *mu, const float *scale, const float *quat, float opac, const float *rgb,
                            const double *dir, const double *W, const double *cam, const double *p, dprec *out)
{
    out->vis = 0;
    dual m[3], sc[3], q[4];
    for (int i = 0; i < 3; ++i) { m[i] = dk(mu[i]); sc[i] = dk(scale[i]); }
    for (int i = 0; i < 4; ++i) q[i] = dk(quat[i]);
    dual o = dk(opac), col[3];
    for (int i = 0; i < 3; ++i) col[i] = dk(rgb[i]);
    for (int k = 0; k < 6; ++k) {
        for (int i = 0; i < 3; ++i) { m[i].d[k] = dir[6 * i + k]; sc[i].d[k] = dir[6 * (3 + i) + k]; }
        for (int i = 0; i < 4; ++i) q[i].d[k] = dir[6 * (6 + i) + k];
        o.d[k] = dir[6 * 10 + k];
        for (int i = 0; i < 3; ++i) col[i].d[k] = dir[6 * (11 + i) + k];
    }
    dual t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = dadd(dadd(dadd(dscale(m[0], W[4 * i]), dscale(m[1], W[4 * i + 1])), dscale(m[2], W[4 * i + 2])),
                    dk(W[4 * i + 3]));
    if (!(t[2].v > p[P_NEAR])) return;
    /* rotation of the normalised quaternion, Sigma = (R S)(R S)^T */
    dual nq = dsqrt(dadd(dadd(dmul(q[0], q[0]), dmul(q[1], q[1])), dadd(dmul(q[2], q[2]), dmul(q[3], q[3]))));
    dual w = ddiv(q[0], nq), x = ddiv(q[1], nq), y = ddiv(q[2], nq), z = ddiv(q[3], nq);
    dual one = dk(1.0);
    dual R[9] = {dsub(one, dscale(dadd(dmul(y, y), dmul(z, z)), 2)), dscale(dsub(dmul(x, y), dmul(w, z)), 2),
                 dscale(dadd(dmul(x, z), dmul(w, y)), 2),
                 dscale(dadd(dmul(x, y), dmul(w, z)), 2), dsub(one, dscale(dadd(dmul(x, x), dmul(z, z)), 2)),
                 dscale(dsub(dmul(y, z), dmul(w, x)), 2),
                 dscale(dsub(dmul(x, z), dmul(w, y)), 2), dscale(dadd(dmul(y, z), dmul(w, x)), 2),
                 dsub(one, dscale(dadd(dmul(x, x), dmul(y, y)), 2))};
    dual M[9], S3[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = dmul(R[3 * i + j], sc[j]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S3[3 * i + j] = dadd(dadd(dmul(M[3 * i], M[3 * j]), dmul(M[3 * i + 1], M[3 * j + 1])),
                                 dmul(M[3 * i + 2], M[3 * j + 2]));
    const double fx = cam[C_FX], fy = cam[C_FY];
    const double limx = p[P_FOV_CLAMP] * (0.5 * cam[C_W]) / fx, limy = p[P_FOV_CLAMP] * (0.5 * cam[C_H]) / fy;
    dual xz = ddiv(t[0], t[2]), yz = ddiv(t[1], t[2]);
    if (xz.v < -limx) xz = dk(-limx); if (xz.v > limx) xz = dk(limx);
    if (yz.v < -limy) yz = dk(-limy); if (yz.v > limy) yz = dk(limy);
    dual J[6] = {ddiv(dk(fx), t[2]), dk(0), dscale(ddiv(xz, t[2]), -fx),
                 dk(0), ddiv(dk(fy), t[2]), dscale(ddiv(yz, t[2]), -fy)};
    const double Rw[9] = {W[0], W[1], W[2], W[4], W[5], W[6], W[8], W[9], W[10]};
    dual T[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = dadd(dadd(dscale(J[3 * i], Rw[j]), dscale(J[3 * i + 1], Rw[3 + j])),
                                dscale(J[3 * i + 2], Rw[6 + j]));
    dual TS[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            TS[3 * i + j] = dadd(dadd(dmul(T[3 * i], S3[j]), dmul(T[3 * i + 1], S3[3 + j])),
                                 dmul(T[3 * i + 2], S3[6 + j]));
    dual c00 = dadd(dadd(dmul(TS[0], T[0]), dmul(TS[1], T[1])), dmul(TS[2], T[2]));
    dual c01 = dadd(dadd(dmul(TS[0], T[3]), dmul(TS[1], T[4])), dmul(TS[2], T[5]));
    dual c11 = dadd(dadd(dmul(TS[3], T[3]), dmul(TS[4], T[4])), dmul(TS[5], T[5]));
    dual a = dadd(c00, dk(p[P_EPS2D])), b = c01, c = dadd(c11, dk(p[P_EPS2D]));
    dual det = dsub(dmul(a, c), dmul(b, b));
    if (!(det.v > 0)) return;
    out->A = ddiv(c, det); out->B = dscale(ddiv(b, det), -1.0); out->C = ddiv(a, det);
    out->u = dadd(dscale(ddiv(t[0], t[2]), fx), dk(cam[C_CX]));
    out->v = dadd(dscale(ddiv(t[1], t[2]), fy), dk(cam[C_CY]));
    out->rx = p[P_CUT] * sqrt(a.v); out->ry = p[P_CUT] * sqrt(c.v);
    if (out->u.v + out->rx < 0 || out->u.v - out->rx >= cam[C_W] || out->v.v + out->ry < 0 || out->v.v - out->ry >= cam[C_H])
        return;
    out->z = t[2].v; out->zd = t[2]; out->o = o;
    for (int i = 0; i < 3; ++i) out->col[i] = col[i];
    out->vis = 1;
}

/* Composite one view in duals: img[3][H][W] duals (caller-allocated); dep and
 * alp [H][W] (may be NULL): depth D = sum w z and alpha A = sum w. */
static void dcomposite_view(const dprec *r, int64_t n, const double *cam, const double *p, dual *img, dual *dep,
                            dual *alp)
{
    const int Wd = (int)cam[C_W], Hd = (int)cam[C_H];
    const int64_t npx = (int64_t)Wd * Hd;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    double *zkey = (double *)malloc(sizeof(double) * (n + 1));
    int64_t nv = 0;
    for (int64_t i = 0; i < n; ++i) {
        zkey[i] = r[i].vis ? r[i].z : 0;
        if (r[i].vis) order[nv++] = i;
    }
    msort_by_double(order, tmp, nv, zkey);
    dual *T = (dual *)malloc(sizeof(dual) * npx);
    uint8_t *done = (uint8_t *)calloc(npx, 1);
    for (int64_t k = 0; k < npx; ++k) {
        T[k] = dk(1.0);
        img[k] = img[npx + k] = img[2 * npx + k] = dk(0);
        if (dep) dep[k] = dk(0);
        if (alp) alp[k] = dk(0);
    }
    const double lim = -0.5 * p[P_CUT] * p[P_CUT];
    for (int64_t j = 0; j < nv; ++j) {
        const dprec *g = &r[order[j]];
        int x0 = (int)floor(g->u.v - g->rx - 1), x1 = (int)ceil(g->u.v + g->rx);
        int y0 = (int)floor(g->v.v - g->ry - 1), y1 = (int)ceil(g->v.v + g->ry);
        if (x0 < 0) x0 = 0; if (y0 < 0) y0 = 0;
        if (x1 > Wd - 1) x1 = Wd - 1; if (y1 > Hd - 1) y1 = Hd - 1;
        for (int y = y0; y <= y1; ++y)
            for (int xx = x0; xx <= x1; ++xx) {
                const int64_t k = (int64_t)y * Wd + xx;
                if (done[k]) continue;
                dual dx = dsub(dk(xx + 0.5), g->u), dy = dsub(dk(y + 0.5), g->v);
                dual pw = dsub(dscale(dadd(dmul(g->A, dmul(dx, dx)), dmul(g->C, dmul(dy, dy))), -0.5),
                               dmul(g->B, dmul(dx, dy)));
                if (pw.v < lim) continue;
                dual raw = dmul(dexp(pw), g->o);
                dual al = raw.v < p[P_ALPHA_MAX] ? raw : dk(p[P_ALPHA_MAX]);
                if (al.v < p[P_ALPHA_MIN]) continue;
                dual tn = dmul(T[k], dsub(dk(1.0), al));
                if (tn.v < p[P_T_MIN]) { done[k] = 1; continue; }
                dual wgt = dmul(al, T[k]);
                for (int ch = 0; ch < 3; ++ch) img[ch * npx + k] = dadd(img[ch * npx + k], dmul(wgt, g->col[ch]));
                if (dep) dep[k] = dadd(dep[k], dmul(wgt, g->zd));
                if (alp) alp[k] = dadd(alp[k], wgt);
                T[k] = tn;
            }
    }
    free(order); free(tmp); free(zkey); free(T); free(done);
}

/* ---- SSIM (the D-SSIM term of Eq. 3) --------------------------------------
 * SSIM of Wang, Bovik, Sheikh and Simoncelli (2004) as 3D Gaussian Splatting
 * uses it: at every pixel the local means, variances and covariance under an
 * 11 x 11 Gaussian window (standard deviation 1.5 px, weights summing to 1),
 * samples outside the image counting as 0, and
 *   SSIM = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
 * sx^2 = E[x^2] - mx^2, sxy = E[xy] - mx my, C1 = 0.01^2, C2 = 0.03^2 (unit
 * dynamic range).  D-SSIM = 1 - the mean of SSIM over pixels and channels. */
enum { SSIM_R = 5, SSIM_N = 2 * SSIM_R + 1 };
static const double SSIM_C1 = 0.01 * 0.01, SSIM_C2 = 0.03 * 0.03;

static void ssim_window(double w[SSIM_N][SSIM_N])
{
    double s = 0.0;
    for (int i = 0; i < SSIM_N; ++i)
        for (int j = 0; j < SSIM_N; ++j) {
            const double di = i - SSIM_R, dj = j - SSIM_R;
            w[i][j] = exp(-(di * di + dj * dj) / (2.0 * 1.5 * 1.5));
            s += w[i][j];
        }
    for (int i = 0; i < SSIM_N; ++i)
        for (int j = 0; j < SSIM_N; ++j) w[i][j] /= s;
}

/* SSIM map of one channel: x, y, out [H][W]. */
void or_ssim_map(const double *x, const double *y, int H, int W, double *out)
{
    double w[SSIM_N][SSIM_N];
    ssim_window(w);
#pragma omp parallel for schedule(static)
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            double mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
            for (int i = 0; i < SSIM_N; ++i) {
                const int yy = py + i - SSIM_R;
                if (yy < 0 || yy >= H) continue;
                for (int j = 0; j < SSIM_N; ++j) {
                    const int xx = px + j - SSIM_R;
                    if (xx < 0 || xx >= W) continue;
                    const double a = x[(int64_t)yy * W + xx], b = y[(int64_t)yy * W + xx], c = w[i][j];
                    mx += c * a; my += c * b; exx += c * a * a; eyy += c * b * b; exy += c * a * b;
                }
            }
            const double sx = exx - mx * mx, sy = eyy - my * my, sxy = exy - mx * my;
            out[(int64_t)py * W + px] = ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) /
                                        ((mx * mx + my * my + SSIM_C1) * (sx + sy + SSIM_C2));
        }
}

/* Sum over the pixels of one channel of SSIM(x, y), x in duals, y fixed. */
static dual dssim_sum(const dual *x, const double *y, int H, int W)
{
    double w[SSIM_N][SSIM_N];
    ssim_window(w);
    const int64_t npx = (int64_t)H * W;
    dual *xx = (dual *)malloc(sizeof(dual) * (npx + 1));
    dual *rows = (dual *)malloc(sizeof(dual) * (H + 1));
    for (int64_t k = 0; k < npx; ++k) xx[k] = dmul(x[k], x[k]);
#pragma omp parallel for schedule(static)
    for (int py = 0; py < H; ++py) {
        dual acc = dk(0);
        for (int px = 0; px < W; ++px) {
            dual mx = dk(0), exx = dk(0), exy = dk(0);
            double my = 0, eyy = 0;
            for (int i = 0; i < SSIM_N; ++i) {
                const int yy = py + i - SSIM_R;
                if (yy < 0 || yy >= H) continue;
                for (int j = 0; j < SSIM_N; ++j) {
                    const int xc = px + j - SSIM_R;
                    if (xc < 0 || xc >= W) continue;
                    const int64_t k = (int64_t)yy * W + xc;
                    const double c = w[i][j], b = y[k];
                    mx = dadd(mx, dscale(x[k], c));
                    exx = dadd(exx, dscale(xx[k], c));
                    exy = dadd(exy, dscale(x[k], c * b));
                    my += c * b;
                    eyy += c * b * b;
                }
            }
            const dual sx = dsub(exx, dmul(mx, mx));
            const double sy = eyy - my * my;
            const dual sxy = dsub(exy, dscale(mx, my));
            const dual num = dmul(dadd(dscale(mx, 2 * my), dk(SSIM_C1)), dadd(dscale(sxy, 2), dk(SSIM_C2)));
            const dual den = dmul(dadd(dmul(mx, mx), dk(my * my + SSIM_C1)), dadd(sx, dk(sy + SSIM_C2)));
            acc = dadd(acc, ddiv(num, den));
        }
        rows[py] = acc;
    }
    dual s = dk(0);
    for (int py = 0; py < H; ++py) s = dadd(s, rows[py]);
    free(xx); free(rows);
    return s;
}

/* L_rgb (Eq. 3) of one view's image x (duals, [3][H][W]) against y:
 * (1 - lambda) mean |x - y| + lambda (1 - mean SSIM(x, y)). */
static dual drgb_loss(const dual *x, const double *y, int H, int W, double lambda)
{
    const int64_t npx = (int64_t)H * W;
    const double inv = 1.0 / (3.0 * (double)npx);
    dual l1 = dk(0);
    for (int64_t k = 0; k < 3 * npx; ++k) {
        dual d = dsub(x[k], dk(y[k]));
        l1 = dadd(l1, dscale(d, d.v >= 0 ? 1.0 : -1.0));
    }
    dual l = dscale(l1, (1.0 - lambda) * inv);
    if (lambda != 0.0) {
        dual ss = dk(0);
        for (int ch = 0; ch < 3; ++ch) ss = dadd(ss, dssim_sum(x + ch * npx, y + ch * npx, H, W));
        l = dadd(l, dscale(dsub(dk(1.0), dscale(ss, inv)), lambda));
    }
    return l;
}

/* ---- re-projection (the P of Eq. 5) ---------------------------------------
 * Reading: the pairs are consecutive training views (t, t+1).  A pixel p of
 * view t whose rendered alpha A = sum w (1 - T) reaches alpha_min takes the
 * depth d = D / A of its rendered depth D (the depth equation of Sec. III-A),
 * is lifted to the camera point d ((p_x + 0.5 - cx) / fx, (p_y + 0.5 - cy) /
 * fy, 1), carried through the world into view t+1 (poses W_t, W_{t+1}) and
 * projected to q; when q lies in front of the near plane and its four
 * bilinear neighbours (pixel centres at +0.5) lie in the image, the
 * re-projected image at p is I_{t+1} sampled bilinearly at q, otherwise it
 * keeps I_t(p) (no residual).  out [3][H][W] duals. */
static void dwarp_view(const dual *dep, const dual *alp, const double *Wt, const double *Wn, const double *cam,
                       const double *p, double alpha_min, const double *It, const double *In, dual *out)
{
    const int Wd = (int)cam[C_W], Hd = (int)cam[C_H];
    const int64_t npx = (int64_t)Wd * Hd;
    for (int py = 0; py < Hd; ++py)
        for (int px = 0; px < Wd; ++px) {
            const int64_t k = (int64_t)py * Wd + px;
            for (int ch = 0; ch < 3; ++ch) out[ch * npx + k] = dk(It[ch * npx + k]);
            if (!(alp[k].v >= alpha_min)) continue;
            const dual d = ddiv(dep[k], alp[k]);
            const double ray[3] = {(px + 0.5 - cam[C_CX]) / cam[C_FX], (py + 0.5 - cam[C_CY]) / cam[C_FY], 1.0};
            dual Pc[3], X[3], Pn[3];
            for (int i = 0; i < 3; ++i) Pc[i] = dsub(dscale(d, ray[i]), dk(Wt[4 * i + 3]));
            for (int i = 0; i < 3; ++i)   /* X = R_t^T (P_c - t_t) */
                X[i] = dadd(dadd(dscale(Pc[0], Wt[i]), dscale(Pc[1], Wt[4 + i])), dscale(Pc[2], Wt[8 + i]));
            for (int i = 0; i < 3; ++i)
                Pn[i] = dadd(dadd(dadd(dscale(X[0], Wn[4 * i]), dscale(X[1], Wn[4 * i + 1])), dscale(X[2], Wn[4 * i + 2])),
                             dk(Wn[4 * i + 3]));
            if (!(Pn[2].v > p[P_NEAR])) continue;
            const dual sx = dadd(dscale(ddiv(Pn[0], Pn[2]), cam[C_FX]), dk(cam[C_CX] - 0.5));
            const dual sy = dadd(dscale(ddiv(Pn[1], Pn[2]), cam[C_FY]), dk(cam[C_CY] - 0.5));
            const double x0 = floor(sx.v), y0 = floor(sy.v);
            if (!(x0 >= 0 && x0 <= Wd - 2 && y0 >= 0 && y0 <= Hd - 2)) continue;
            const dual fx = dsub(sx, dk(x0)), fy = dsub(sy, dk(y0));
            const dual gx = dsub(dk(1.0), fx), gy = dsub(dk(1.0), fy);
            const int64_t k00 = (int64_t)y0 * Wd + (int64_t)x0;
            for (int ch = 0; ch < 3; ++ch) {
                const double *I = In + ch * npx;
                out[ch * npx + k] = dadd(dadd(dscale(dmul(gx, gy), I[k00]), dscale(dmul(fx, gy), I[k00 + 1])),
                                         dadd(dscale(dmul(gx, fy), I[k00 + Wd]), dscale(dmul(fx, fy), I[k00 + Wd + 1])));
            }
        }
}

/* The map-training loss of Eq. 6, L = w_photo L_photo + w_reproj L_reproj:
 * L_photo = (1/V) sum_t L_rgb(R(G, W_t), I_t) (Eq. 4), L_reproj = (1/(V-1))
 * sum over consecutive pairs of L_rgb(P(D(G_t), ...), I_t) (Eq. 5, the
 * re-projection read as above), and its derivatives along six parameter
 * directions.  out[7] = (L, dL[6]). */
void or_train_loss_jvp(const float *means, const float *scales, const float *quats, const float *opac,
                       const float *rgb, int64_t n, const double *dirs, const double *poses, int n_views,
                       const double *cam, const double *p, const double *gt, double lambda, double w_photo,
                       double w_reproj, double alpha_min, double *out)
{
    const int Wd = (int)cam[C_W], Hd = (int)cam[C_H];
    const int64_t npx = (int64_t)Wd * Hd;
    const int reproj = w_reproj != 0.0 && n_views > 1;
    dprec *r = (dprec *)malloc(sizeof(dprec) * (n + 1));
    dual *img = (dual *)malloc(sizeof(dual) * 3 * npx);
    dual *dep = reproj ? (dual *)malloc(sizeof(dual) * npx) : NULL;
    dual *alp = reproj ? (dual *)malloc(sizeof(dual) * npx) : NULL;
    dual *wimg = reproj ? (dual *)malloc(sizeof(dual) * 3 * npx) : NULL;
    dual loss = dk(0);
    for (int v = 0; v < n_views; ++v) {
        for (int64_t i = 0; i < n; ++i)
            dproject_params(means + 3 * i, scales + 3 * i, quats + 4 * i, opac[i], rgb + 3 * i,
                            dirs + (int64_t)NPAR * 6 * i, poses + 16 * v, cam, p, &r[i]);
        const int pair = reproj && v + 1 < n_views;
        dcomposite_view(r, n, cam, p, img, pair ? dep : NULL, pair ? alp : NULL);
        const double *I = gt + (int64_t)v * 3 * npx;
        if (w_photo != 0.0) loss = dadd(loss, dscale(drgb_loss(img, I, Hd, Wd, lambda), w_photo / n_views));
        if (pair) {
            dwarp_view(dep, alp, poses + 16 * v, poses + 16 * (v + 1), cam, p, alpha_min, I, I + 3 * npx, wimg);
            loss = dadd(loss, dscale(drgb_loss(wimg, I, Hd, Wd, lambda), w_reproj / (n_views - 1)));
        }
    }
    out[0] = loss.v;
    for (int k = 0; k < 6; ++k) out[1 + k] = loss.d[k];
    free(r); free(img); free(dep); free(alp); free(wimg);
}
