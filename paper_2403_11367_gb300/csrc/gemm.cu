// gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05, TMEM).
//
//   C[m][n] = sum_k A[m][k] * B[n][k]   (+ bias[n], ReLU, optional)
//
// A and B are row-major with K contiguous ("K-major"), BF16; the accumulator
// is FP32 in tensor memory; C is written as FP32 or BF16.  This is the dense
// contraction of the learned candidate proposal (convolutions via im2col and
// the MLP, forward and backward).
//
// One CTA of 128 threads computes a 128 x BN tile (BN in {16, 32, ..., 128}).
// Per K step of 64 the threads copy the A and B tiles into shared memory in
// the canonical no-swizzle K-major layout (8-row x 16-byte core matrices;
// core matrices adjacent in K are LBO bytes apart, adjacent in M/N 128 bytes
// apart), one elected thread issues four tcgen05.mma (K = 16 each) and commits
// them to an mbarrier, and every thread waits on it before the tiles are
// overwritten.  The epilogue reads the accumulator with tcgen05.ld (each warp
// its 32 TMEM lanes) and applies bias and ReLU.  With split_k > 1, CTA z
// covers the K range [z*Ks, (z+1)*Ks) and writes FP32 partials
// C[z][M][N], summed later in a fixed order.
//
// Every mbarrier wait is bounded: past the limit the CTA records an error in
// *status, stops issuing MMAs, and still frees its tensor memory.
#include "internal.cuh"

namespace reloc {

constexpr int GEMM_THREADS = 128;
constexpr int GEMM_BM = 128;
constexpr int GEMM_BK = 64;
constexpr int GEMM_BN_MAX = 128;
constexpr unsigned GEMM_WAIT_LIMIT = 1u << 22;   // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle, K-major (tcgen05 format:
// start >> 4 in bits 0-13, leading byte offset >> 4 in 16-29, stride byte
// offset >> 4 in 32-45, version 1 in 46-47, layout type 0 in 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (unsigned it = 0; it < GEMM_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

struct GemmArgs {
    const __nv_bfloat16 *A, *B;
    const float *bias;          // [N] or null
    float *Cf;                  // FP32 output (or split-K partials) or null
    __nv_bfloat16 *Cb;          // BF16 output or null
    int M, N, K;                // K multiple of 64
    int lda, ldb, ldc;          // row strides (elements)
    int relu;
    int split_k;                // >= 1; > 1 writes partials Cf[z][M][ldc]
    int *status;                // error flag (1: an mbarrier wait gave up)
};

template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm_bf16(GemmArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    // A tile: 8 K-chunks x (128/8) row blocks x 128 B; B tile: 8 x (BN/8) x 128 B
    uint8_t *sA = smem;
    uint8_t *sB = smem + GEMM_BM * GEMM_BK * 2;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * GEMM_BM, n0 = blockIdx.y * BN;
    const int kz = blockIdx.z;
    const int k_per = g.K / g.split_k;                  // multiple of 64 by construction
    const int kbeg = kz * k_per, kend = kbeg + k_per;
    constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;   // power of two >= 32
    constexpr uint32_t LBO_A = (GEMM_BM / 8) * 128, LBO_B = (BN / 8) * 128, SBO = 128;
    constexpr uint32_t IDESC = instr_desc_bf16(GEMM_BM, BN);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        abort_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s;
    const uint32_t aA = smem_u32(sA), aB = smem_u32(sB), mb = smem_u32(&mbar);

    uint32_t phase = 0;
    bool any = false;
    for (int k0 = kbeg; k0 < kend; k0 += GEMM_BK) {
        // ---- stage A (128 x 64) and B (BN x 64) as 16-byte core-matrix rows
        for (int c = tid; c < GEMM_BM * (GEMM_BK / 8); c += GEMM_THREADS) {
            const int r = c / (GEMM_BK / 8), kc = c % (GEMM_BK / 8);
            uint4 v = make_uint4(0, 0, 0, 0);
            if (m0 + r < g.M) v = *reinterpret_cast<const uint4 *>(g.A + (int64_t)(m0 + r) * g.lda + k0 + kc * 8);
            *reinterpret_cast<uint4 *>(sA + kc * LBO_A + (r >> 3) * SBO + (r & 7) * 16) = v;
        }
        for (int c = tid; c < BN * (GEMM_BK / 8); c += GEMM_THREADS) {
            const int r = c / (GEMM_BK / 8), kc = c % (GEMM_BK / 8);
            uint4 v = make_uint4(0, 0, 0, 0);
            if (n0 + r < g.N) v = *reinterpret_cast<const uint4 *>(g.B + (int64_t)(n0 + r) * g.ldb + k0 + kc * 8);
            *reinterpret_cast<uint4 *>(sB + kc * LBO_B + (r >> 3) * SBO + (r & 7) * 16) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (abort_s) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int j = 0; j < GEMM_BK / 16; ++j) {
                // K step j covers two core-matrix columns: advance by 2 * LBO
                const uint64_t da = smem_desc(aA + 2 * j * LBO_A, LBO_A, SBO);
                const uint64_t db = smem_desc(aB + 2 * j * LBO_B, LBO_B, SBO);
                const uint32_t acc = (any || j > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\t"
                             "setp.ne.u32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(da), "l"(db), "r"(IDESC), "r"(acc)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                         : "memory");
        }
        any = true;
        // every thread waits until the MMAs have consumed this stage
        if (!mbar_wait(mb, phase)) {
            abort_s = 1;
            if (g.status) atomicExch(g.status, 1);
        }
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (abort_s) break;
    }

    // ---- epilogue: TMEM -> registers -> global ------------------------------
    if (!abort_s) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(lane_addr + c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < g.M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = n0 + c0 + i;
                    if (col >= g.N) continue;
                    float v = any ? __uint_as_float(r[i]) : 0.f;
                    if (g.split_k > 1) {
                        g.Cf[((int64_t)kz * g.M + row) * g.ldc + col] = v;
                        continue;
                    }
                    if (g.bias) v += g.bias[col];
                    if (g.relu) v = fmaxf(v, 0.f);
                    if (g.Cf) g.Cf[(int64_t)row * g.ldc + col] = v;
                    if (g.Cb) g.Cb[(int64_t)row * g.ldc + col] = __float2bfloat16_rn(v);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Sum split-K partials in a fixed order and apply the epilogue.
__global__ void k_gemm_reduce(const float *__restrict__ part, int split, int M, int N, int ldc,
                              const float *__restrict__ bias, int relu, float *__restrict__ Cf,
                              __nv_bfloat16 *__restrict__ Cb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * N) return;
    const int row = (int)(i / N), col = (int)(i % N);
    float v = 0.f;
    for (int z = 0; z < split; ++z) v += part[((int64_t)z * M + row) * ldc + col];
    if (bias) v += bias[col];
    if (relu) v = fmaxf(v, 0.f);
    if (Cf) Cf[(int64_t)row * ldc + col] = v;
    if (Cb) Cb[(int64_t)row * ldc + col] = __float2bfloat16_rn(v);
}

template <int BN>
static cudaError_t gemm_t(const GemmArgs &g, cudaStream_t st)
{
    // 96 KB of dynamic shared memory keeps at most two CTAs per SM, so their
    // tensor memory (<= 2 x 128 columns) always fits the SM's 512 columns.
    constexpr size_t SMEM = 96 * 1024;
    static_assert((GEMM_BM + BN) * GEMM_BK * 2 <= SMEM, "tiles fit");
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)ceil_div(g.M, GEMM_BM), (unsigned)ceil_div(g.N, BN), (unsigned)g.split_k);
    k_gemm_bf16<BN><<<grid, GEMM_THREADS, SMEM, st>>>(g);
    return cudaGetLastError();
}

// C = A B^T (+ bias, ReLU).  Requirements: K % 64 == 0, K / split_k % 64 == 0,
// lda, ldb multiples of 8 (16-byte rows), 16-byte aligned A and B.
// split_k > 1 needs `partials` (split_k * M * ldc floats).
cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias, float *Cf,
                             __nv_bfloat16 *Cb, int M, int N, int K, int lda, int ldb, int ldc, int relu, int split_k,
                             float *partials, int *status, cudaStream_t st)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (K % GEMM_BK || split_k < 1 || (K / split_k) % GEMM_BK || (lda % 8) || (ldb % 8) ||
        ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || (split_k > 1 && !partials))
        return cudaErrorInvalidValue;
    GemmArgs g{A, B, bias, Cf, Cb, M, N, K, lda, ldb, ldc, relu, split_k, status};
    if (split_k > 1) {
        g.Cf = partials;
        g.Cb = nullptr;
        g.bias = nullptr;
        g.relu = 0;
    }
    const int BN = N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : 128;
    cudaError_t e;
    switch (BN) {
    case 16: e = gemm_t<16>(g, st); break;
    case 32: e = gemm_t<32>(g, st); break;
    case 64: e = gemm_t<64>(g, st); break;
    default: e = gemm_t<128>(g, st); break;
    }
    if (e != cudaSuccess || split_k == 1) return e;
    const int64_t n = (int64_t)M * N;
    k_gemm_reduce<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(partials, split_k, M, N, ldc, bias, relu, Cf, Cb);
    return cudaGetLastError();
}

}  // namespace reloc
