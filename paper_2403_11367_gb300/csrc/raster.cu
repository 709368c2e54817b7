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

// Compensated FP32 sums by error-free extraction (Rump, Ogita and Oishi,
// "Accurate floating-point summation part I: faithful rounding", 2008): with
// SIGMA = 1.5 * 2^10, h = fl(x + SIGMA) - SIGMA is x rounded to a multiple of
// 2^-13 (exactly, for |x| < 2^9) and x - h is exact.  A sum is carried as
// hi + lo: the extracted parts h are added into hi, where every partial sum
// is a multiple of 2^-13 below 2^11 -- at most 2^24 grid steps, so each
// addition is exact (a warp block sums 192 samples of magnitude up to 4: the
// colours, their squares and their products with the query, with room to
// spare) -- and the remainders x - h (at most 2^-14 each) into lo, whose
// rounding errors are 2^-37 of the samples' size.  A product a b adds its
// exact rounding error fma(a, b, -ab) to lo as well.  Both parts cross the
// warp butterfly as plain sums (hi exactly), and hi + lo is combined in
// FP64.  The _rn intrinsics keep the compiler from fusing or reordering
// these steps.
constexpr float CS_SIGMA = 1536.f;
struct CSum {
    float hi, lo;
};
__device__ __forceinline__ void cs_add(CSum &c, float x)
{
    const float h = __fsub_rn(__fadd_rn(x, CS_SIGMA), CS_SIGMA);
    c.hi = __fadd_rn(c.hi, h);
    c.lo = __fadd_rn(c.lo, __fsub_rn(x, h));
}
__device__ __forceinline__ void cs_add_prod(CSum &c, float a, float b)
{
    const float p = __fmul_rn(a, b);
    cs_add(c, p);
    c.lo = __fadd_rn(c.lo, __fmaf_rn(a, b, -p));      // a b - p, exactly
}
// butterfly over the warp: every lane ends with the warp's total
__device__ __forceinline__ double cs_warp_total(CSum c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c.hi = __fadd_rn(c.hi, __shfl_xor_sync(0xffffffffu, c.hi, o));
        c.lo = __fadd_rn(c.lo, __shfl_xor_sync(0xffffffffu, c.lo, o));
    }
    return (double)c.hi + (double)c.lo;
}

// Warp reduce-scatter of NP values per lane (NP a power of two, 2 .. 16):
// recursive halving, each step exchanging half of the remaining values with
// the partner lane (offsets 16, 8, ...), then a plain sum over the last
// 32 / NP lanes.  Returns the warp's total of value (lane / (32 / NP)) on
// every lane: (NP - 1) + log2(32 / NP) shuffles instead of 5 NP for NP
// separate sums.
template <int NP>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NP], int lane)
{
#pragma unroll
    for (int n = NP, o = 16; n > 1; n >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            const float send = up ? v[i] : v[n / 2 + i];
            const float keep = up ? v[n / 2 + i] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    float x = v[0];
#pragma unroll
    for (int o = 16 / NP; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Fixed grid and fixed reduction order: the sums are deterministic.
// grid (QS_BLOCKS, Q): block (b, q) sums its share of query q.
__global__ void __launch_bounds__(QS_THREADS) k_query_stats(Layout L, int64_t HW, int gray, double *part)
{
    __shared__ double s[2][QS_THREADS / 32];
    const float *q = L.q_img[blockIdx.y];
    const int64_t n = gray ? HW : 3 * HW;
    double a = 0, b = 0;
    for (int64_t j = (int64_t)blockIdx.x * QS_THREADS + threadIdx.x; j < n; j += (int64_t)QS_BLOCKS * QS_THREADS) {
        const double x = gray ? ((double)q[j] + (double)q[HW + j] + (double)q[2 * HW + j]) / 3.0 : (double)q[j];
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
        double *o = part + 2 * ((int64_t)blockIdx.y * QS_BLOCKS + blockIdx.x);
        o[0] = A;
        o[1] = B;
    }
}

// A block per query: its QS_BLOCKS partials summed by a fixed tree (one per
// thread, then a warp and a block reduction), so the sums are deterministic.
constexpr int QSF_THREADS = 160;                 // >= QS_BLOCKS, whole warps
static_assert(QSF_THREADS >= QS_BLOCKS && QSF_THREADS % 32 == 0, "one partial per thread");
__global__ void __launch_bounds__(QSF_THREADS) k_query_stats_final(const double *part, double *qstats)
{
    __shared__ double s[2][QSF_THREADS / 32];
    const int q = blockIdx.x, k = threadIdx.x;
    double A = 0, B = 0;
    if (k < QS_BLOCKS) {
        A = part[2 * ((int64_t)q * QS_BLOCKS + k)];
        B = part[2 * ((int64_t)q * QS_BLOCKS + k) + 1];
    }
    A = warp_sum_d(A);
    B = warp_sum_d(B);
    if ((k & 31) == 0) { s[0][k >> 5] = A; s[1][k >> 5] = B; }
    __syncthreads();
    if (k == 0) {
        A = 0;
        B = 0;
        for (int w = 0; w < QSF_THREADS / 32; ++w) { A += s[0][w]; B += s[1][w]; }
        qstats[2 * q] = A;
        qstats[2 * q + 1] = B;
    }
}

cudaError_t launch_query_stats(const Layout &L, int64_t HW, bool gray, double *block_scratch, double *qstats,
                               cudaStream_t st)
{
    if (L.Q <= 0) return cudaSuccess;
    k_query_stats<<<dim3(QS_BLOCKS, L.Q), QS_THREADS, 0, st>>>(L, HW, gray ? 1 : 0, block_scratch);
    k_query_stats_final<<<L.Q, QSF_THREADS, 0, st>>>(block_scratch, qstats);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ K6 -----
// One CTA per (view, tile).  Each thread owns two vertically adjacent pixels,
// so a warp covers a TW x (64/TW) pixel block, and the warps of a tile run
// independently (no barrier until the NCC epilogue).  A warp walks the tile's
// sorted list RPL*32 records at a time: each lane loads its records (the
// tile's warps read the same records, so after the first they hit L1),
// derives the power threshold below which a record cannot contribute --
// max(-cut^2/2, ln(alpha_min / o) - 1e-3), the margin covering the float
// logarithm and exponential -- and keeps the record if the ellipse
// {power >= threshold}, widened by 1%, meets the warp's pixel block (exact
// ellipse-rectangle test: the least value of the quadratic form over the
// block).  A ballot compacts the kept records, in list order,
// into the warp's shared-memory slots, and the warp blends only those; a
// pixel below a record's threshold also skips the exponential.  Both tests
// only drop pairs the exact per-pixel tests would drop, so the result is that
// of testing every pixel of the tile against every record of its list.  A
// warp stops once all its pixels' transmittance has run out.

// Packed FP32 pairs (two pixels per thread): one 64-bit register holds
// (low = pixel row y, high = pixel row y + 1); fma/mul/add.rn.f32x2 operate on
// both halves with IEEE round-to-nearest, like two scalar instructions.
typedef unsigned long long f32x2;
__device__ __forceinline__ unsigned lanemask_lt_u()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ f32x2 pk(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f32x2 v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Records carry (u, v, depth, log2 o | a1, a2, b1, b2 | r, g, b, -): the
// footprint in principal-axis form, scaled for base 2: with d the offset of a
// pixel centre from the projected mean, U = a1 dx + a2 dy and V = b1 dx + b2 dy,
// the exponent is p' = log2(o) + power log2(e) = log2(o) - (U^2 + V^2), so
// alpha = min(alpha_max, 2^p') = min(alpha_max, o exp(power)).
// q(d) = U^2 + V^2 = qa dx^2 + 2 qb dx dy + qc dy^2 is the scaled conic.
struct Conic {
    float a, b, c;
};
__device__ __forceinline__ Conic conic_of(float4 ab)
{
    return {fmaf(ab.x, ab.x, ab.z * ab.z), fmaf(ab.x, ab.y, ab.z * ab.w), fmaf(ab.y, ab.y, ab.w * ab.w)};
}

// Minimum over the rectangle [x0,x1] x [y0,y1] (offsets from the ellipse
// centre) of q.  q is strictly convex with its minimum 0 at the centre, so
// unless the centre is inside, the rectangle's minimum lies on a side facing
// the centre (from any other point q falls along the segment towards the
// centre without leaving the rectangle).  Those sides are x = X and y = Y with
// X, Y the coordinates of the rectangle nearest 0; where 0 lies between x0 and
// x1 the segment x = 0 crosses the rectangle and only bounds the minimum from
// above.  So the minimum is the lesser of the two 1D minima along x = X and
// y = Y (each a clamped quadratic), and 0 when the centre is inside
// (X = Y = 0).  The minimisers -qb X / qc and -qb Y / qa use the fast
// reciprocal: any point of a side gives q at or above that side's minimum, and
// one off by a few ulp raises it by qc (delta)^2, orders below the callers'
// widening of the bound, so the cull stays conservative.  q is evaluated at
// those points as U^2 + V^2, which does not cancel along long thin
// footprints (the conic form does, by orders of magnitude).
__device__ __forceinline__ float quad_min_rect(float4 ab, Conic q, float x0, float x1, float y0, float y1)
{
    const float X = fminf(fmaxf(0.f, x0), x1), Y = fminf(fmaxf(0.f, y0), y1);
    const float dy = fminf(fmaxf(__fdividef(-q.b, q.c) * X, y0), y1);   // along x = X
    const float dx = fminf(fmaxf(__fdividef(-q.b, q.a) * Y, x0), x1);   // along y = Y
    const float u1 = fmaf(ab.x, X, ab.y * dy), v1 = fmaf(ab.z, X, ab.w * dy);
    const float u2 = fmaf(ab.x, dx, ab.y * Y), v2 = fmaf(ab.z, dx, ab.w * Y);
    return fminf(fmaf(u1, u1, v1 * v1), fmaf(u2, u2, v2 * v2));
}

// Block-centred staging of a kept record for one warp block whose pixel
// centres lie around (ocx, ocy).  With the block centre's offset from the mean
// d_b and a pixel's fixed offset delta from the block centre,
//   p'(delta) = P0 + Gx dx + Gy dy - (qa dx^2 + 2 qb dx dy + qc dy^2),
// P0 = log2(o) - Ub^2 - Vb^2 the exponent at the block centre and
// G = -2 (Ub (a1, a2) + Vb (b1, b2)) its gradient there, Ub and Vb the axis
// coordinates of d_b.  P0 and G come from the axes (no cancellation however
// far the centre lies along a long footprint), and the quadratic term only
// sees offsets within the block (|delta| <= 8 px), so the conic form's
// cancellation stays at that scale.  Per pixel pair this costs three scalar
// and two packed FMAs.
//   s0 = (-qa, Gx, -2 qb, Gy), s1 = (-qc, -qc, P0, thr)
__device__ __forceinline__ void block_stage(float4 pa, float4 ab, Conic q, float thr, float ocx, float ocy,
                                            float4 &s0, float4 &s1)
{
    const float dbx = ocx - pa.x, dby = ocy - pa.y;
    const float Ub = fmaf(ab.x, dbx, ab.y * dby), Vb = fmaf(ab.z, dbx, ab.w * dby);
    const float P0 = fmaf(-Vb, Vb, fmaf(-Ub, Ub, pa.w));
    const float Gx = -2.f * fmaf(Ub, ab.x, Vb * ab.z), Gy = -2.f * fmaf(Ub, ab.y, Vb * ab.w);
    s0 = make_float4(-q.a, Gx, -2.f * q.b, Gy);
    s1 = make_float4(-q.c, -q.c, P0, thr);
}

// Warp blocks: 64 pixels, BW x BH with BW = min(TW, 16), each lane owning two
// vertically adjacent pixels; a TW x TH tile holds (TW / BW) x (TH / BH) of them.
template <int TW, int TH>
struct BlockGeom {
    static constexpr int BW = TW < 16 ? TW : 16;
    static constexpr int BH = 64 / BW;
    static constexpr int NBX = TW / BW;
    static constexpr int WPT = TW * TH / 64;
    static_assert(WPT >= 1 && TW % BW == 0 && TH % BH == 0, "tile shape");
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Pixel arithmetic in base 2 (block_stage): p' = power log2(e) + log2(o),
// alpha = min(alpha_max, 2^p') = min(alpha_max, o exp(power)).  The 3-sigma
// rule (power >= -cut^2/2) and alpha >= alpha_min become one threshold on p':
// p' >= thr = max(-cut^2/2 log2(e) + log2(o), log2(alpha_min)), i.e.
// q <= min(cut^2/2 log2(e), log2(o) - log2(alpha_min)).  The transmittance
// is carried as T' = prod (1 - alpha) past the stop: T' only decreases, so a
// pixel's stop (T (1 - alpha) < t_min, the stopping Gaussian not added) is the
// first record where T' falls below t_min, and a weight is kept while T' after
// it is >= t_min -- no flag, and one fused T + T (-alpha) per record on the
// dependency chain (rounded once).  The kernel carries -alpha and minus the
// weights, so that update is a single FMA, and negates the sums at the end;
// the alpha output is the sum of the kept weights, which telescopes to
// 1 - T before the stop.  Both tests are 0/1 factors from one float compare
// each (set.ge), which runs on the ALU pipe beside the FMA-bound arithmetic.
// The column terms P0 + Gx dx - qa dx^2 and Gy - 2 qb dx are shared by the
// pixel pair and computed once (scalar); the row terms run packed.  DA:
// accumulate depth and alpha too (image export); the scoring launches need
// colour only.
// 1.0f if a >= b (a < b) else 0.0f: one float compare, on the ALU pipe
__device__ __forceinline__ float step_ge(float a, float b)
{
    float d;
    asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float step_lt(float a, float b)
{
    float d;
    asm("set.lt.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
// One 64-pixel warp block (unit `unit` of view v, its list range r): the
// blend and the epilogue (image export to slot out_v, NCC partials).
template <int TW, int TH, int RPL, bool DA>
__device__ __forceinline__ void blend_unit(const float4 *__restrict__ rec, const Layout &L,
                                           const uint32_t *__restrict__ inst_gauss, const CamParams &cam,
                                           double *__restrict__ partials, float *__restrict__ rgb,
                                           float *__restrict__ depth, float *__restrict__ alpha, int v, int out_v,
                                           int unit, int2 r, float4 (*s_rec)[32 * RPL])
{
    using GM = BlockGeom<TW, TH>;
    constexpr int BW = GM::BW, BH = GM::BH, WPT = GM::WPT;
    constexpr int CH = 32 * RPL;             // records per warp step
    // kept records compacted in s_rec: (-qa, Gx, -2 qb, Gy) (-qc, -qc, P0, thr)
    // (r, r, g, g) (b, b, z, z)
    const int tile = unit / WPT, warp = unit - tile * WPT;
    const int tx = tile % cam.ntx, ty = tile / cam.ntx;
    const int lane = threadIdx.x;
    const int bx0p = tx * TW + (warp % GM::NBX) * BW, by0p = ty * TH + (warp / GM::NBX) * BH;
    const int px = bx0p + lane % BW;
    const int py0 = by0p + 2 * (lane / BW);
    const int py1 = py0 + 1;
    const bool in0 = px < cam.width && py0 < cam.height;
    const bool in1 = px < cam.width && py1 < cam.height;
    // centre of the block's pixel centres and this lane's offsets from it (exact)
    const float ocx = (float)bx0p + 0.5f * BW, ocy = (float)by0p + 0.5f * BH;
    const float DX = (float)(lane % BW) + 0.5f - 0.5f * BW;
    const float dy0 = (float)(2 * (lane / BW)) + 0.5f - 0.5f * BH;
    const f32x2 DY2 = pk(dy0, dy0 + 1.f);
    const uint32_t *list = inst_gauss + L.io_off[v];
    const float4 *vrec = rec + L.vd_off[v] * 3;
    constexpr float L2E = 1.4426950408889634f;
    const float limL = -0.5f * cam.cut * cam.cut * L2E;
    const float l2amin = log2f(cam.alpha_min);
    float4(*const sw)[CH] = s_rec;
    const unsigned lt = lanemask_lt_u();

    // pixel pair state (low = row y, high = row y + 1): transmittance, colour,
    // depth and weight sums
    f32x2 T2 = pk(in0 ? 1.f : 0.f, in1 ? 1.f : 0.f);
    f32x2 R2 = 0ull, G2 = 0ull, B2 = 0ull, Z2 = 0ull, S2 = 0ull;
    const f32x2 NEG1 = pk(-1.f, -1.f);

    // software pipeline: list indices two steps ahead, records one step ahead
    uint32_t gnext[RPL];
    float4 qa[RPL], qb[RPL], qc[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
        const int j0 = r.x + q * 32 + lane, j1 = j0 + CH;
        if (j0 < r.y) {
            const float4 *p = vrec + 3 * (int64_t)__ldg(list + j0);
            qa[q] = __ldg(p); qb[q] = __ldg(p + 1); qc[q] = __ldg(p + 2);
        }
        gnext[q] = j1 < r.y ? __ldg(list + j1) : 0u;
    }
    for (int b = r.x; b < r.y; b += CH) {
        // pixel-centre box of the pixels still compositing (a pixel has stopped
        // once T < t_min and takes nothing more, so records that miss this box
        // would add nothing)
        float bx0, bx1, by0, by1;
        {
            float t0, t1;
            upk(T2, t0, t1);
            const bool a0 = t0 >= cam.t_min && in0, a1 = t1 >= cam.t_min && in1;
            if (__all_sync(0xffffffffu, !a0 && !a1)) break;
            const unsigned rlo = __reduce_min_sync(0xffffffffu, a0 ? (unsigned)py0 : (a1 ? (unsigned)py1 : 0xffffu));
            const unsigned rhi = __reduce_max_sync(0xffffffffu, a1 ? (unsigned)py1 : (a0 ? (unsigned)py0 : 0u));
            const unsigned clo = __reduce_min_sync(0xffffffffu, (a0 || a1) ? (unsigned)px : 0xffffu);
            const unsigned chi = __reduce_max_sync(0xffffffffu, (a0 || a1) ? (unsigned)px : 0u);
            bx0 = (float)clo + 0.5f; bx1 = (float)chi + 0.5f;
            by0 = (float)rlo + 0.5f; by1 = (float)rhi + 0.5f;
        }
        int nk = 0;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
            const int j = b + q * 32 + lane;
            bool hit = false;
            const float4 pa = qa[q], pb = qb[q], pc = qc[q];
            // issue the next step's loads before working on this one
            const int jn = j + CH, jnn = j + 2 * CH;
            if (jn < r.y) {
                const float4 *p = vrec + 3 * (int64_t)gnext[q];
                qa[q] = __ldg(p); qb[q] = __ldg(p + 1); qc[q] = __ldg(p + 2);
            }
            gnext[q] = jnn < r.y ? __ldg(list + jnn) : 0u;
            // pa: u v z log2(o) | pb: scaled axes | pc: rgb.  A pixel counts iff
            // q <= min(-limL, log2 o - log2 alpha_min); keep the record iff the
            // ellipse at that bound (plus a margin for the float arithmetic,
            // widened 1%) meets the box
            const Conic cq = conic_of(pb);
            const float qbound = fminf(-limL, pa.w - l2amin + 1.5e-3f);
            if (j < r.y && qbound > 0.f) {
                const float qmin = quad_min_rect(pb, cq, bx0 - pa.x, bx1 - pa.x, by0 - pa.y, by1 - pa.y);
                hit = qmin <= qbound * 1.01f + 1e-3f;
            }
            const unsigned keep = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int k = nk + __popc(keep & lt);
                float4 t0, t1;
                block_stage(pa, pb, cq, fmaxf(limL + pa.w, l2amin), ocx, ocy, t0, t1);
                sw[0][k] = t0;
                sw[1][k] = t1;
                sw[2][k] = make_float4(pc.x, pc.x, pc.y, pc.y);
                sw[3][k] = DA ? make_float4(pc.z, pc.z, pa.z, pa.z) : make_float4(pc.z, pc.z, 0.f, 0.f);
            }
            nk += __popc(keep);
        }
        __syncwarp();
#pragma unroll 4
        for (int k = 0; k < nk; ++k) {
            const float4 s0 = sw[0][k], s1 = sw[1][k];
            const float k1 = fmaf(s0.z, DX, s0.w), k0 = fmaf(fmaf(s0.x, DX, s0.y), DX, s1.z);
            const f32x2 P2 = fma2(DY2, fma2(pk(s1.x, s1.y), DY2, pk(k1, k1)), pk(k0, k0));
            float p0, p1;
            upk(P2, p0, p1);
            // p' >= threshold
            const f32x2 IN2 = pk(step_ge(p0, s1.w), step_ge(p1, s1.w));
            // -alpha = max(-alpha_max, -2^p') (exact negation of the clamp)
            const float na0 = fmaxf(-cam.alpha_max, -ex2_approx(p0));
            const float na1 = fmaxf(-cam.alpha_max, -ex2_approx(p1));
            // T' = T (1 - alpha), formed as one fused T + T (-alpha), carries on
            // past the stop: it only decreases, so T' >= t_min holds up to the
            // stop and never after; the weight is kept while it holds (one
            // instruction on the dependency chain)
            const f32x2 NAIN = mul2(pk(na0, na1), IN2);
            const f32x2 TN2 = fma2(T2, NAIN, T2);
            float n0, n1;
            upk(TN2, n0, n1);
            // T (1 - alpha) >= t_min
            const f32x2 GO2 = pk(step_ge(n0, cam.t_min), step_ge(n1, cam.t_min));
            // minus the weight: the sums below accumulate negated
            const f32x2 NWF = mul2(mul2(T2, NAIN), GO2);
            T2 = TN2;
            const float4 c0 = sw[2][k], c1 = sw[3][k];
            R2 = fma2(pk(c0.x, c0.y), NWF, R2);
            G2 = fma2(pk(c0.z, c0.w), NWF, G2);
            B2 = fma2(pk(c1.x, c1.y), NWF, B2);
            if (DA) {
                Z2 = fma2(pk(c1.z, c1.w), NWF, Z2);
                S2 = add2(S2, NWF);
            }
        }
        __syncwarp();
    }

    float R0, R1, G0, G1, B0, B1, D0, D1, A0, A1;
    upk(mul2(R2, NEG1), R0, R1);
    upk(mul2(G2, NEG1), G0, G1);
    upk(mul2(B2, NEG1), B0, B1);
    upk(mul2(Z2, NEG1), D0, D1);
    upk(mul2(S2, NEG1), A0, A1);
    const int64_t HW = (int64_t)cam.width * cam.height;
    const int64_t pix0 = (int64_t)py0 * cam.width + px, pix1 = pix0 + cam.width;
    if (rgb) {
        float *o = rgb + (int64_t)out_v * 3 * HW;
        if (in0) { o[pix0] = R0; o[HW + pix0] = G0; o[2 * HW + pix0] = B0; }
        if (in1) { o[pix1] = R1; o[HW + pix1] = G1; o[2 * HW + pix1] = B1; }
    }
    if (depth) {
        if (in0) depth[(int64_t)out_v * HW + pix0] = D0;
        if (in1) depth[(int64_t)out_v * HW + pix1] = D1;
    }
    if (alpha) {
        if (in0) alpha[(int64_t)out_v * HW + pix0] = A0;
        if (in1) alpha[(int64_t)out_v * HW + pix1] = A1;
    }
    if (partials) {
        const float *query = L.q_img[L.view_q[v]];
        // pixels outside the image have zero colour and contribute nothing;
        // the block's S_r, S_rr and S_rq are compensated FP32 sums
        CSum sr = {0.f, 0.f}, srr = {0.f, 0.f}, srq = {0.f, 0.f};
        if (cam.ncc_gray) {
            // gray values (R + G + B) / 3 of render and query
            const float third = 1.f / 3.f;
            const float r0 = (R0 + G0 + B0) * third, r1 = (R1 + G1 + B1) * third;
            cs_add(sr, r0);
            cs_add(sr, r1);
            cs_add_prod(srr, r0, r0);
            cs_add_prod(srr, r1, r1);
            if (in0) cs_add_prod(srq, r0, (__ldg(query + pix0) + __ldg(query + HW + pix0) + __ldg(query + 2 * HW + pix0)) * third);
            if (in1) cs_add_prod(srq, r1, (__ldg(query + pix1) + __ldg(query + HW + pix1) + __ldg(query + 2 * HW + pix1)) * third);
        } else {
            const float c[6] = {R0, G0, B0, R1, G1, B1};
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                cs_add(sr, c[k]);
                cs_add_prod(srr, c[k], c[k]);
            }
            if (in0) {
                cs_add_prod(srq, R0, __ldg(query + pix0));
                cs_add_prod(srq, G0, __ldg(query + HW + pix0));
                cs_add_prod(srq, B0, __ldg(query + 2 * HW + pix0));
            }
            if (in1) {
                cs_add_prod(srq, R1, __ldg(query + pix1));
                cs_add_prod(srq, G1, __ldg(query + HW + pix1));
                cs_add_prod(srq, B1, __ldg(query + 2 * HW + pix1));
            }
        }
        const double tr = cs_warp_total(sr), trr = cs_warp_total(srr), trq = cs_warp_total(srq);
        if (lane == 0) {
            double *o = partials + ((int64_t)out_v * cam.n_tiles * WPT + unit) * 3;
            o[0] = tr;
            o[1] = trr;
            o[2] = trq;
        }
    }
}

// Persistent K6: a grid of resident one-warp blocks (as many as fit on the
// SMs) takes the launch's units -- (view, tile, 64-pixel block) of every view
// of every query in the call -- from one queue (an atomic ticket per unit).
// The units of heavy tiles (lists of at least BLEND_HEAVY records, listed by
// k_blend_heavy: the horizon's tiles, whose units run up to twenty times the
// mean) are handed out first, the rest in view-major order (the heavy ones
// skipped there), so that no long unit starts near the end of the launch.
// A warp holds its next ticket, the next unit's view and list range while it
// blends the current one, so the dependent loads that start a unit are off
// the critical path, and no block launch separates units (a per-unit grid
// spent about a quarter of its warp slots idle).  Each unit is processed
// whole by one warp and writes only its own outputs, so the result does not
// depend on which warp takes which unit, nor on the order of the heavy list.
// Register budget: 64 per thread (32 one-warp blocks per SM) for the scoring
// launches; the export launches (DA) carry depth and alpha sums too and get
// 72 (28 blocks per SM) rather than spill (same-box A/B: winner export
// 0.233 -> 0.208 ms).
constexpr int BLEND_HEAVY = 1024;
constexpr int BQ_LIST = 4;                       // queue[0] ticket, [1] heavy count, list from [4]

// queue[BQ_LIST + k] = vi * n_tiles + tile for each (view slot, tile) whose
// list holds at least BLEND_HEAVY records; queue[1] counts them (zeroed on
// the stream before the launch).  Nothing is listed after an overflow.
__global__ void k_blend_heavy(const int2 *__restrict__ ranges, const int *__restrict__ view_sel, int n_views,
                              int n_tiles, const int *__restrict__ overflow, int *__restrict__ queue)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_views * n_tiles || *overflow != 0) return;
    const int vi = (int)(i / n_tiles), t = (int)(i - (int64_t)vi * n_tiles);
    const int v = view_sel ? view_sel[vi] : vi;
    if (v < 0) return;
    const int2 r = ranges[(int64_t)v * n_tiles + t];
    if (r.y - r.x >= BLEND_HEAVY) queue[BQ_LIST + atomicAdd(queue + 1, 1)] = (int)i;
}

template <int TW, int TH, int RPL, bool DA>
__global__ void __launch_bounds__(32, RPL == 1 ? (DA ? 28 : 32) : 24)
k_blend(const float4 *__restrict__ rec, Layout L, const uint32_t *__restrict__ inst_gauss,
        const int2 *__restrict__ ranges, CamParams cam, double *__restrict__ partials, float *__restrict__ rgb,
        float *__restrict__ depth, float *__restrict__ alpha, const int *__restrict__ view_sel, int n_views,
        const int *__restrict__ overflow, int *__restrict__ queue)
{
    __shared__ float4 s_rec[4][32 * RPL];
    constexpr int WPT = BlockGeom<TW, TH>::WPT;
    const int upv = cam.n_tiles * WPT;                          // units per view
    const int64_t total = (int64_t)upv * n_views;
    const bool ovf = *overflow != 0;
    // heavy units, handed out first (and skipped in order) when the launch
    // listed them
    const bool listed = blend_launches(n_views) > 1;
    const int64_t hh = listed ? (int64_t)queue[1] * WPT : 0;
    const int lane = threadIdx.x;
    // view and list range of unit u (empty past the end or after an overflow)
    auto locate = [&](int64_t u, int &v, int2 &r) {
        v = -1;
        r = make_int2(0, 0);
        if (u < total) {
            const int vi = (int)(u / upv), loc = (int)(u - (int64_t)vi * upv);
            v = view_sel ? view_sel[vi] : vi;
            if (!ovf && v >= 0) r = ranges[(int64_t)v * cam.n_tiles + loc / WPT];
        }
    };
    // the next unit of the queue: the heavy list's, then the rest in order
    auto next = [&](int64_t &u, int &v, int2 &r) {
        while (true) {
            int64_t t = 0;
            if (lane == 0) t = atomicAdd(queue, 1);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t < hh) {
                const int h = queue[BQ_LIST + (int)(t / WPT)];
                u = (int64_t)(h / cam.n_tiles) * upv + (int64_t)(h % cam.n_tiles) * WPT + (int)(t % WPT);
                locate(u, v, r);
                return;
            }
            u = t - hh;
            locate(u, v, r);
            if (u >= total || !listed || r.y - r.x < BLEND_HEAVY) return;
        }
    };
    int64_t u;
    int v;
    int2 r;
    next(u, v, r);
    while (u < total) {
        // the next unit: ticket, view and range in flight during this one
        int64_t un;
        int vn;
        int2 rn;
        next(un, vn, rn);
        const int vi = (int)(u / upv);
        blend_unit<TW, TH, RPL, DA>(rec, L, inst_gauss, cam, partials, rgb, depth, alpha, v < 0 ? 0 : v, vi,
                                    (int)(u - (int64_t)vi * upv), v < 0 ? make_int2(0, 0) : r, s_rec);
        __syncwarp();
        u = un;
        v = vn;
        r = rn;
    }
}

// resident one-warp blocks per SM of a blend kernel on the current device
template <typename K>
static int resident_blocks(K kernel)
{
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32, 0) != cudaSuccess)
            return 0;
        cached[dev] = sms * (per_sm > 0 ? per_sm : 1);
    }
    return cached[dev];
}

template <int TW, int TH, int RPL>
static cudaError_t blend_t(const float4 *rec, const Layout &L, const uint32_t *inst_gauss, const int2 *ranges,
                           const CamParams &cam, double *partials, float *rgb, float *depth, float *alpha,
                           const int *view_sel, int n_sel, const int *overflow, int *queue, cudaStream_t st)
{
    const int nv = view_sel ? n_sel : L.V;
    const int64_t units = (int64_t)cam.n_tiles * (TW * TH / 64) * nv;
    cudaError_t e = cudaMemsetAsync(queue, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (blend_launches(nv) > 1) {
        const int64_t nt = (int64_t)nv * cam.n_tiles;
        k_blend_heavy<<<(unsigned)ceil_div(nt, 256), 256, 0, st>>>(ranges, view_sel, nv, cam.n_tiles, overflow,
                                                                   queue);
    }
    if (depth || alpha) {
        const int g = resident_blocks(k_blend<TW, TH, RPL, true>);
        if (g <= 0) return cudaErrorInvalidValue;
        k_blend<TW, TH, RPL, true><<<(unsigned)min64(units, g), 32, 0, st>>>(rec, L, inst_gauss, ranges, cam, partials,
                                                                             rgb, depth, alpha, view_sel, nv, overflow,
                                                                             queue);
    } else {
        const int g = resident_blocks(k_blend<TW, TH, RPL, false>);
        if (g <= 0) return cudaErrorInvalidValue;
        k_blend<TW, TH, RPL, false><<<(unsigned)min64(units, g), 32, 0, st>>>(rec, L, inst_gauss, ranges, cam,
                                                                              partials, rgb, depth, alpha, view_sel, nv,
                                                                              overflow, queue);
    }
    return cudaGetLastError();
}

cudaError_t launch_blend(const float4 *rec, const Layout &L, const uint32_t *inst_gauss, const int2 *ranges,
                         const CamParams &cam, double *partials, float *rgb, float *depth, float *alpha,
                         const int *view_sel, int n_sel, const int *overflow, int *queue, cudaStream_t st)
{
    if ((view_sel ? n_sel : L.V) <= 0) return cudaSuccess;
#define RELOC_BLEND_CASE(W_, H_, R_)                                                                             \
    if (cam.tile_w == W_ && cam.tile_h == H_ && cam.blend_rpl == R_)                                            \
        return blend_t<W_, H_, R_>(rec, L, inst_gauss, ranges, cam, partials, rgb, depth, alpha, view_sel, n_sel, \
                                   overflow, queue, st);
    RELOC_BLEND_CASE(16, 16, 1)
    RELOC_BLEND_CASE(16, 16, 2)
    RELOC_BLEND_CASE(8, 8, 1)
    RELOC_BLEND_CASE(8, 8, 2)
    RELOC_BLEND_CASE(32, 8, 1)
    RELOC_BLEND_CASE(32, 8, 2)
    RELOC_BLEND_CASE(16, 8, 1)
    RELOC_BLEND_CASE(16, 8, 2)
    RELOC_BLEND_CASE(8, 16, 1)
    RELOC_BLEND_CASE(8, 16, 2)
    RELOC_BLEND_CASE(32, 16, 1)
    RELOC_BLEND_CASE(32, 16, 2)
#undef RELOC_BLEND_CASE
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ K7 -----
// NCC = (S_rq - S_r S_q / n) / sqrt((S_rr - S_r^2 / n)(S_qq - S_q^2 / n)),
// the one-pass form of Eq. ncc, summed in FP64 in a fixed order.

constexpr int NCC_THREADS = 256;

__global__ void __launch_bounds__(NCC_THREADS)
k_ncc_finalize(const double *__restrict__ partials, const double *__restrict__ qstats, Layout L, int n_units,
               int64_t n, double *__restrict__ scores, int *__restrict__ degenerate, double *__restrict__ coef)
{
    __shared__ double s[3][NCC_THREADS / 32];
    const int v = blockIdx.x;
    const double *p = partials + (int64_t)v * n_units * 3;
    double a = 0, b = 0, c = 0;
    for (int t = threadIdx.x; t < n_units; t += NCC_THREADS) {
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
        const int q = L.view_q[v];
        const double Sq = qstats[2 * q], Sqq = qstats[2 * q + 1];
        const double cov = Srq - Sr * Sq / nn;
        const double vr = Srr - Sr * Sr / nn;
        const double vq = Sqq - Sq * Sq / nn;
        const bool dg = !(vr > 1e-12 * nn) || !(vq > 1e-12 * nn);
        scores[v] = dg ? 0.0 : cov / (sqrt(vr) * sqrt(vq));
        if (degenerate) degenerate[v] = dg ? 1 : 0;
        if (coef) {
            // d NCC / d r_i = (q_i - mean q) / sqrt(vr vq) - NCC (r_i - mean r) / vr
            double *o = coef + 4 * (int64_t)v;
            o[0] = dg ? 0.0 : 1.0 / (sqrt(vr) * sqrt(vq));
            o[1] = dg ? 0.0 : scores[v] / vr;
            o[2] = Sr / nn;
            o[3] = Sq / nn;
        }
    }
}

cudaError_t launch_ncc_finalize(const double *partials, const double *qstats, const Layout &L, int n_units,
                                int64_t n_samples, double *scores, int *degenerate, double *coef, cudaStream_t st)
{
    if (L.V <= 0) return cudaSuccess;
    k_ncc_finalize<<<L.V, NCC_THREADS, 0, st>>>(partials, qstats, L, n_units, n_samples, scores, degenerate, coef);
    return cudaGetLastError();
}

// ------------------------------------------------------- K6 backward ------
// Gradients of a view's loss with respect to its Gaussians' projected means
// (u, v) and conics (a, b, c), for the view's fixed set of included
// (pixel, Gaussian) pairs.  A warp per 64-pixel block walks the tile's list
// with the forward's cull and the forward's arithmetic (base-2 exponent, the
// inclusion, clamp and stop tests as exact 0/1 compares, the fused
// transmittance update, the pixel pair packed in f32x2), so its decisions are
// the forward's bit for bit:
// first, unless the forward's render is given, compositing the pair to its
// final colour C, then again front to back, where for contributor j with
// weight w_j = alpha_j T_j,
//   dL/d alpha_j = T_j S_j - K_j / (1 - alpha_j),
// S_j = G . c_j (+ G_D z_j + G_A in image mode: depth and alpha as two more
// channels with values z_j and 1) and K_j = the sum of w S over the
// contributors after j (K starts at G . C (+ G_D D + G_A A) and loses w_j S_j
// at j); alpha = o exp(power) unclamped gives dL/d power = alpha dL/d alpha,
// and power = -(a dx^2 + 2 b dx dy + c dy^2)/2 with dx = x - u, so
// d power/du = a dx + b dy and d power/dv = b dx + c dy, taken as the
// gradient at the block centre (-G / 2, from the axes, no cancellation) plus
// the conic times the pixel's offset within the block, in the scaled units of
// the staging (divided by log2(e) / 2); d power/da = -dx^2/2, d/db = -dx dy,
// d/dc = -dy^2/2.  The warp
// sums each record's gradients over its 64 pixels (a reduce-scatter: lane
// 32/NP * m holds total m) and adds them to the (view, Gaussian) entry of
// gout.
// IMG = false: L is the view's NCC (G from coef), five outputs (u, v, a, b, c).
// IMG = true: G is given per pixel (gimg [V][3][H][W], an image loss's
// gradient), and optionally G_D, G_A (gda [V][2][H][W]); ten outputs: also
// dL/d colour = sum w G, dL/d opacity = dL/d power / o and dL/dz = sum w G_D.
// cimg (image mode, may be null): the forward's render of the views
// ([V][3][H][W], with cdep, calp [V][H][W] when gda is given) replaces the
// first walk.
template <int TW, int TH, bool IMG>
__global__ void __launch_bounds__(32, IMG ? 24 : 32)
k_blend_grad(const float4 *__restrict__ rec, Layout L, const uint32_t *__restrict__ inst_gauss,
             const int2 *__restrict__ ranges, CamParams cam, const double *__restrict__ coef,
             const float *__restrict__ gimg, const float *__restrict__ gda, const float *__restrict__ cimg,
             const float *__restrict__ cdep, const float *__restrict__ calp, float *__restrict__ gout,
             const int *__restrict__ overflow)
{
    constexpr int NOUT = IMG ? 10 : 5;
    constexpr int NP = IMG ? 16 : 8;           // NOUT padded to a power of two
    constexpr int GRP = 32 / NP;                // lanes holding each total
    using GM = BlockGeom<TW, TH>;
    constexpr int BW = GM::BW, BH = GM::BH, WPT = GM::WPT;
    constexpr float L2E = 1.4426950408889634f;
    // kept records: the forward's (-qa, Gx, -2 qb, Gy) (-qc, -qc, P0, thr)
    // (r, r, g, g) (b, b, z, z), then the block centre's offset from the mean
    // and 1/o: (dbx, 1/o, dby, dby), and the scaled conic (qa, qb, qc, -)
    __shared__ float4 s_rec[6][32];
    __shared__ uint32_t s_g[32];
    const int unit = blockIdx.x;
    const int tile = unit / WPT, warp = unit - tile * WPT;
    const int v = blockIdx.y;
    const int tx = tile % cam.ntx, ty = tile / cam.ntx;
    const int lane = threadIdx.x;
    const int bx0p = tx * TW + (warp % GM::NBX) * BW, by0p = ty * TH + (warp / GM::NBX) * BH;
    const int px = bx0p + lane % BW;
    const int py0 = by0p + 2 * (lane / BW);
    const bool in[2] = {px < cam.width && py0 < cam.height, px < cam.width && py0 + 1 < cam.height};
    const float ocx = (float)bx0p + 0.5f * BW, ocy = (float)by0p + 0.5f * BH;
    const float DX = (float)(lane % BW) + 0.5f - 0.5f * BW;
    const float dy0 = (float)(2 * (lane / BW)) + 0.5f - 0.5f * BH;
    const f32x2 DY2 = pk(dy0, dy0 + 1.f);
    if (*overflow) return;
    const int2 r = ranges[(int64_t)v * cam.n_tiles + tile];
    const uint32_t *list = inst_gauss + L.io_off[v];
    const float4 *vrec = rec + L.vd_off[v] * 3;
    const float limL = -0.5f * cam.cut * cam.cut * L2E;
    const float l2amin = log2f(cam.alpha_min);
    const float amax = cam.alpha_max;
    const unsigned lt = lanemask_lt_u();
    const f32x2 NEG1 = pk(-1.f, -1.f);
    // the natural conic is the scaled one over log2(e) / 2
    constexpr float IK2 = 2.f / L2E;

    // the forward's cull and compaction, one step of 32 records, against the
    // box of the pixels still compositing (T > 0)
    auto stage = [&](int b, f32x2 T2) -> int {
        float t0, t1;
        upk(T2, t0, t1);
        const bool a0 = t0 >= cam.t_min && in[0], a1 = t1 >= cam.t_min && in[1];
        const unsigned rlo = __reduce_min_sync(0xffffffffu, a0 ? (unsigned)py0 : (a1 ? (unsigned)py0 + 1u : 0xffffu));
        const unsigned rhi = __reduce_max_sync(0xffffffffu, a1 ? (unsigned)py0 + 1u : (a0 ? (unsigned)py0 : 0u));
        const unsigned clo = __reduce_min_sync(0xffffffffu, (a0 || a1) ? (unsigned)px : 0xffffu);
        const unsigned chi = __reduce_max_sync(0xffffffffu, (a0 || a1) ? (unsigned)px : 0u);
        const float bx0 = (float)clo + 0.5f, bx1 = (float)chi + 0.5f;
        const float by0 = (float)rlo + 0.5f, by1 = (float)rhi + 0.5f;
        const int j = b + lane;
        bool hit = false;
        float4 pa = make_float4(0, 0, 0, 0), pb = pa, pc = pa;
        Conic cq = {0.f, 0.f, 0.f};
        uint32_t gi = 0;
        if (j < r.y) {
            gi = __ldg(list + j);
            const float4 *p = vrec + 3 * (int64_t)gi;
            pa = __ldg(p); pb = __ldg(p + 1); pc = __ldg(p + 2);
            cq = conic_of(pb);
            const float qbound = fminf(-limL, pa.w - l2amin + 1.5e-3f);
            if (qbound > 0.f) {
                const float qmin = quad_min_rect(pb, cq, bx0 - pa.x, bx1 - pa.x, by0 - pa.y, by1 - pa.y);
                hit = qmin <= qbound * 1.01f + 1e-3f;
            }
        }
        const unsigned keep = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int k = __popc(keep & lt);
            float4 t0, t1;
            block_stage(pa, pb, cq, fmaxf(limL + pa.w, l2amin), ocx, ocy, t0, t1);
            s_rec[0][k] = t0;
            s_rec[1][k] = t1;
            s_rec[2][k] = make_float4(pc.x, pc.x, pc.y, pc.y);
            s_rec[3][k] = make_float4(pc.z, pc.z, pa.z, pa.z);
            s_rec[4][k] = make_float4(ocx - pa.x, ex2_approx(-pa.w), ocy - pa.y, ocy - pa.y);
            s_rec[5][k] = make_float4(cq.a, cq.b, cq.c, 0.f);
            s_g[k] = gi;
        }
        __syncwarp();
        return __popc(keep);
    };

    const int64_t HW = (int64_t)cam.width * cam.height;
    // pass 1: final colour (depth, alpha) of the pixel pair, as the forward
    f32x2 T2 = pk(in[0] ? 1.f : 0.f, in[1] ? 1.f : 0.f);
    f32x2 CR2 = 0ull, CG2 = 0ull, CB2 = 0ull, CZ2 = 0ull, CS2 = 0ull;
    if (IMG && cimg) {
        float c[5][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
#pragma unroll
        for (int p = 0; p < 2; ++p)
            if (in[p]) {
                const int64_t pix = (int64_t)(py0 + p) * cam.width + px;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) c[ch][p] = __ldg(cimg + ((int64_t)v * 3 + ch) * HW + pix);
                if (gda) {
                    c[3][p] = __ldg(cdep + (int64_t)v * HW + pix);
                    c[4][p] = __ldg(calp + (int64_t)v * HW + pix);
                }
            }
        CR2 = pk(c[0][0], c[0][1]); CG2 = pk(c[1][0], c[1][1]); CB2 = pk(c[2][0], c[2][1]);
        CZ2 = pk(c[3][0], c[3][1]); CS2 = pk(c[4][0], c[4][1]);
    } else {
        for (int b = r.x; b < r.y; b += 32) {
            {
                float t0, t1;
                upk(T2, t0, t1);
                if (__all_sync(0xffffffffu, !(t0 >= cam.t_min && in[0]) && !(t1 >= cam.t_min && in[1]))) break;
            }
            const int nk = stage(b, T2);
            for (int k = 0; k < nk; ++k) {
                const float4 s0 = s_rec[0][k], s1 = s_rec[1][k];
                const float k1 = fmaf(s0.z, DX, s0.w), k0 = fmaf(fmaf(s0.x, DX, s0.y), DX, s1.z);
                const f32x2 P2 = fma2(DY2, fma2(pk(s1.x, s1.y), DY2, pk(k1, k1)), pk(k0, k0));
                float p0, p1;
                upk(P2, p0, p1);
                const f32x2 IN2 = pk(step_ge(p0, s1.w), step_ge(p1, s1.w));
                const float na0 = fmaxf(-amax, -ex2_approx(p0)), na1 = fmaxf(-amax, -ex2_approx(p1));
                const f32x2 NAIN = mul2(pk(na0, na1), IN2);
                const f32x2 TN2 = fma2(T2, NAIN, T2);
                float n0, n1;
                upk(TN2, n0, n1);
                const f32x2 GO2 = pk(step_ge(n0, cam.t_min), step_ge(n1, cam.t_min));
                const f32x2 NWF = mul2(mul2(T2, NAIN), GO2);
                T2 = TN2;
                const float4 c0 = s_rec[2][k], c1 = s_rec[3][k];
                CR2 = fma2(pk(c0.x, c0.y), NWF, CR2);
                CG2 = fma2(pk(c0.z, c0.w), NWF, CG2);
                CB2 = fma2(pk(c1.x, c1.y), NWF, CB2);
                if (IMG) {
                    CZ2 = fma2(pk(c1.z, c1.w), NWF, CZ2);
                    CS2 = add2(CS2, NWF);
                }
            }
            __syncwarp();
        }
        // the sums ran over minus the weights
        CR2 = mul2(CR2, NEG1); CG2 = mul2(CG2, NEG1); CB2 = mul2(CB2, NEG1);
        CZ2 = mul2(CZ2, NEG1); CS2 = mul2(CS2, NEG1);
    }
    float C[2][3], DA[2][2];
    upk(CR2, C[0][0], C[1][0]);
    upk(CG2, C[0][1], C[1][1]);
    upk(CB2, C[0][2], C[1][2]);
    upk(CZ2, DA[0][0], DA[1][0]);
    upk(CS2, DA[0][1], DA[1][1]);

    // dL/dC per pixel
    float G[2][3] = {{0, 0, 0}, {0, 0, 0}};
    float GDA[2][2] = {{0, 0}, {0, 0}};
    if (IMG) {
        const float *gi = gimg + (int64_t)v * 3 * HW;
#pragma unroll
        for (int p = 0; p < 2; ++p)
            if (in[p]) {
                const int64_t pix = (int64_t)(py0 + p) * cam.width + px;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) G[p][ch] = __ldg(gi + ch * HW + pix);
                if (gda) {
                    GDA[p][0] = __ldg(gda + (int64_t)v * 2 * HW + pix);
                    GDA[p][1] = __ldg(gda + (int64_t)v * 2 * HW + HW + pix);
                }
            }
    } else {
        // NCC: dNCC/dC = (q - mean q) / sqrt(var_r var_q) - NCC (C - mean r) / var_r
        const double *cf = coef + 4 * (int64_t)v;
        const float k_q = (float)cf[0], k_r = (float)cf[1], mr = (float)cf[2], mq = (float)cf[3];
        const float *query = L.q_img[L.view_q[v]];
#pragma unroll
        for (int p = 0; p < 2; ++p)
            if (in[p]) {
                const int64_t pix = (int64_t)(py0 + p) * cam.width + px;
                if (cam.ncc_gray) {
                    // gray NCC: dNCC/dC_ch = dNCC/d gray / 3
                    const float qg = (__ldg(query + pix) + __ldg(query + HW + pix) + __ldg(query + 2 * HW + pix)) / 3.f;
                    const float rg = (C[p][0] + C[p][1] + C[p][2]) / 3.f;
                    const float gg = (k_q * (qg - mq) - k_r * (rg - mr)) / 3.f;
                    G[p][0] = G[p][1] = G[p][2] = gg;
                } else {
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch)
                        G[p][ch] = k_q * (__ldg(query + ch * HW + pix) - mq) - k_r * (C[p][ch] - mr);
                }
            }
    }
    const f32x2 G0 = pk(G[0][0], G[1][0]), G1 = pk(G[0][1], G[1][1]), G2 = pk(G[0][2], G[1][2]);
    const f32x2 GD = pk(GDA[0][0], GDA[1][0]), GA = pk(GDA[0][1], GDA[1][1]);
    f32x2 K2 = pk(G[0][0] * C[0][0] + G[0][1] * C[0][1] + G[0][2] * C[0][2] + GDA[0][0] * DA[0][0] + GDA[0][1] * DA[0][1],
                  G[1][0] * C[1][0] + G[1][1] * C[1][1] + G[1][2] * C[1][2] + GDA[1][0] * DA[1][0] + GDA[1][1] * DA[1][1]);

    // pass 2: front to back again, gradients per record
    T2 = pk(in[0] ? 1.f : 0.f, in[1] ? 1.f : 0.f);
    for (int b = r.x; b < r.y; b += 32) {
        {
            float t0, t1;
            upk(T2, t0, t1);
            if (__all_sync(0xffffffffu, !(t0 >= cam.t_min && in[0]) && !(t1 >= cam.t_min && in[1]))) break;
        }
        const int nk = stage(b, T2);
        for (int k = 0; k < nk; ++k) {
            const float4 s0 = s_rec[0][k], s1 = s_rec[1][k];
            const float k1 = fmaf(s0.z, DX, s0.w), k0 = fmaf(fmaf(s0.x, DX, s0.y), DX, s1.z);
            const f32x2 P2 = fma2(DY2, fma2(pk(s1.x, s1.y), DY2, pk(k1, k1)), pk(k0, k0));
            float p0, p1;
            upk(P2, p0, p1);
            const float i0 = step_ge(p0, s1.w), i1 = step_ge(p1, s1.w);
            const float r0 = ex2_approx(p0), r1 = ex2_approx(p1);
            // the forward's arithmetic: -alpha, T' = T + T (-alpha) fused, minus the weight
            const float na0 = fmaxf(-amax, -r0), na1 = fmaxf(-amax, -r1);
            const float a0 = -na0, a1 = -na1;
            const f32x2 NAIN = mul2(pk(na0, na1), pk(i0, i1));
            const f32x2 TN2 = fma2(T2, NAIN, T2);
            float n0, n1;
            upk(TN2, n0, n1);
            const float o0 = step_ge(n0, cam.t_min), o1 = step_ge(n1, cam.t_min);
            const f32x2 GO2 = pk(o0, o1);
            const f32x2 NWF = mul2(mul2(T2, NAIN), GO2);
            float w0, w1;
            upk(NWF, w0, w1);
            if (!__any_sync(0xffffffffu, w0 < 0.f || w1 < 0.f)) {
                T2 = TN2;
                continue;
            }
            const float4 c0 = s_rec[2][k], c1 = s_rec[3][k], db = s_rec[4][k], cn = s_rec[5][k];
            // S = G . c (+ G_D z + G_A); K loses w S
            f32x2 S2 = fma2(G0, pk(c0.x, c0.y), fma2(G1, pk(c0.z, c0.w), mul2(G2, pk(c1.x, c1.y))));
            if (IMG) S2 = fma2(GD, pk(c1.z, c1.w), add2(S2, GA));
            K2 = fma2(NWF, S2, K2);
            // dL/d alpha = T S - K / (1 - alpha), masked to the included, unstopped pairs;
            // 1 / (1 - alpha): alpha <= alpha_max < 1, fast reciprocal (2 ulp)
            const f32x2 NR2 = pk(__fdividef(-1.f, 1.f - a0), __fdividef(-1.f, 1.f - a1));
            const f32x2 GAL = mul2(fma2(K2, NR2, mul2(T2, S2)), mul2(pk(i0, i1), GO2));
            // dL/d power = alpha dL/d alpha (0 where the clamp holds)
            const f32x2 GP = mul2(GAL, pk(a0 * step_lt(r0, amax), a1 * step_lt(r1, amax)));
            // offsets of the pixels from the mean: dx = dbx + DX, dy = dby + dy_lane
            const float dx = db.x + DX;
            const f32x2 DYM = add2(pk(db.z, db.w), DY2);
            const f32x2 GX = mul2(GP, pk(dx, dx)), GY = mul2(GP, DYM), GK = mul2(GP, pk(IK2, IK2));
            // d power/du, d power/dv in scaled units: -G/2 + (qa dx + qb dy, qb dx + qc dy) over the block offsets
            const float cu = fmaf(cn.x, DX, -0.5f * s0.y), cv = fmaf(cn.y, DX, -0.5f * s0.w);
            float g[NP];
#pragma unroll
            for (int m = NOUT; m < NP; ++m) g[m] = 0.f;
            float lo, hi;
            upk(mul2(GK, fma2(pk(cn.y, cn.y), DY2, pk(cu, cu))), lo, hi);        // d/du: a dx + b dy
            g[0] = lo + hi;
            upk(mul2(GK, fma2(pk(cn.z, cn.z), DY2, pk(cv, cv))), lo, hi);        // d/dv: b dx + c dy
            g[1] = lo + hi;
            upk(mul2(GX, pk(-0.5f * dx, -0.5f * dx)), lo, hi);                     // d/da: -dx^2 / 2
            g[2] = lo + hi;
            upk(mul2(GX, mul2(DYM, NEG1)), lo, hi);                                // d/db: -dx dy
            g[3] = lo + hi;
            upk(mul2(GY, mul2(DYM, pk(-0.5f, -0.5f))), lo, hi);                     // d/dc: -dy^2 / 2
            g[4] = lo + hi;
            if (IMG) {
                // colour and depth: w G, from minus the weight
                upk(mul2(NWF, G0), lo, hi);
                g[5] = -lo - hi;
                upk(mul2(NWF, G1), lo, hi);
                g[6] = -lo - hi;
                upk(mul2(NWF, G2), lo, hi);
                g[7] = -lo - hi;
                upk(mul2(GP, pk(db.y, db.y)), lo, hi);                             // d/do = dL/d power / o
                g[8] = lo + hi;
                upk(mul2(NWF, GD), lo, hi);
                g[9] = -lo - hi;
            }
            T2 = TN2;
            const float tot = warp_reduce_scatter<NP>(g, lane);
            const int m = lane / GRP;
            if (lane % GRP == 0 && m < NOUT && tot != 0.f)
                atomicAdd(gout + NOUT * (L.vd_off[v] + (int64_t)s_g[k]) + m, tot);
        }
        __syncwarp();
    }
}

template <int TW, int TH>
static cudaError_t blend_grad_t(const float4 *rec, const Layout &L, const uint32_t *inst_gauss, const int2 *ranges,
                                const CamParams &cam, const double *coef, const float *gimg, const float *gda,
                                const float *cimg, const float *cdep, const float *calp, float *gout,
                                const int *overflow, cudaStream_t st)
{
    dim3 grid(cam.n_tiles * (TW * TH / 64), L.V);
    if (gimg)
        k_blend_grad<TW, TH, true><<<grid, 32, 0, st>>>(rec, L, inst_gauss, ranges, cam, coef, gimg, gda, cimg, cdep,
                                                        calp, gout, overflow);
    else
        k_blend_grad<TW, TH, false><<<grid, 32, 0, st>>>(rec, L, inst_gauss, ranges, cam, coef, gimg, gda, nullptr,
                                                         nullptr, nullptr, gout, overflow);
    return cudaGetLastError();
}

cudaError_t launch_blend_grad(const float4 *rec, const Layout &L, const uint32_t *inst_gauss, const int2 *ranges,
                              const CamParams &cam, const double *coef, const float *gimg, const float *gda,
                              const float *cimg, const float *cdep, const float *calp, float *gout,
                              const int *overflow, cudaStream_t st)
{
    if (L.V <= 0) return cudaSuccess;
#define RELOC_GRAD_CASE(W_, H_) \
    if (cam.tile_w == W_ && cam.tile_h == H_) \
        return blend_grad_t<W_, H_>(rec, L, inst_gauss, ranges, cam, coef, gimg, gda, cimg, cdep, calp, gout, \
                                    overflow, st);
    RELOC_GRAD_CASE(16, 16)
    RELOC_GRAD_CASE(8, 8)
    RELOC_GRAD_CASE(32, 8)
    RELOC_GRAD_CASE(16, 8)
    RELOC_GRAD_CASE(8, 16)
    RELOC_GRAD_CASE(32, 16)
#undef RELOC_GRAD_CASE
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ K8 -----

__device__ __forceinline__ bool better(double sa, int ia, double sb, int ib)
{
    return sa > sb || (sa == sb && ia < ib);
}

// one block per query
__global__ void __launch_bounds__(256)
k_argmax(const double *__restrict__ scores, Layout L, int *best, double *best_score, int *view_sel)
{
    __shared__ double s_s[256];
    __shared__ int s_i[256];
    const int q = blockIdx.x;
    const int v0 = L.q_view[q], V = L.q_view[q + 1] - v0;
    double bs = -INFINITY;
    int bi = 0x7fffffff;
    for (int k = threadIdx.x; k < V; k += 256)
        if (better(scores[v0 + k], k, bs, bi)) { bs = scores[v0 + k]; bi = k; }
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
        const int b = s_i[0] < V ? s_i[0] : 0;
        best[q] = b;
        best_score[q] = s_s[0];
        view_sel[q] = v0 + b;
    }
}

cudaError_t launch_argmax(const double *scores, const Layout &L, int *best, double *best_score, int *view_sel,
                          cudaStream_t st)
{
    if (L.Q <= 0) return cudaSuccess;
    k_argmax<<<L.Q, 256, 0, st>>>(scores, L, best, best_score, view_sel);
    return cudaGetLastError();
}

}  // namespace reloc
