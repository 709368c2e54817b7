// gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05, TMEM).
//
//   C[m][n] = sum_k A[m][k] * B[n][k]   (+ bias[n], ReLU, optional)
//
// A and B are row-major with K contiguous ("K-major"), BF16; the accumulator
// is FP32 in tensor memory; C is written as FP32 or BF16.  This is the dense
// contraction of the learned candidate proposal (convolutions via im2col and
// the MLP, forward and backward).
//
// One CTA of 128 threads computes a 128 x BN tile (BN in {16, 32, ..., 256}),
// warp-specialised over a ring of GEMM_STAGES shared-memory stages:
//   - one lane of warp 0 loads the A (128 x 64) and B (BN x 64) tiles of each
//     K step with TMA (cp.async.bulk.tensor, one box per operand: 64 BF16 =
//     128 bytes of K by the tile's rows, 128-byte swizzle, so the tiles land
//     in the canonical K-major SWIZZLE_128B layout: 128-byte rows whose 16-byte
//     chunks are XOR-permuted by the row within each 8-row, 1024-byte group)
//     and signals the stage's "full" mbarrier through the copies'
//     transaction count;
//   - one lane of warp 1 waits for a full stage, issues its four
//     tcgen05.mma (K = 16 each) into the TMEM accumulator and commits them to
//     the stage's "empty" mbarrier, which releases the stage to the loader
//     once the MMAs have read it; after the last K step it commits to a
//     "done" mbarrier;
//   - all four warps wait for "done" and read the accumulator with
//     tcgen05.ld (each warp its 32 TMEM lanes), applying bias and ReLU.
// So the loads of the next stages are in flight while the tensor cores work
// on the current one.  With split_k > 1, CTA z covers the K range
// [z*Ks, (z+1)*Ks) and writes FP32 partials C[z][M][N], summed later in a
// fixed order.
//
// Every mbarrier wait is bounded (GEMM_WAIT_NS of the global timer): past it
// the CTA records an error in *status and stops issuing; the loader then
// waits (bounded) for its own copies in flight, the MMA lane commits "done"
// (which tracks every MMA it issued) and all threads wait for it (bounded)
// before the tensor memory is freed, so nothing the CTA started still writes
// shared or tensor memory when it exits.
#include "internal.cuh"

#include <cuda.h>

namespace reloc {

constexpr int GEMM_THREADS = 128;
constexpr int GEMM_BM = 128;
constexpr int GEMM_BK = 64;
constexpr int GEMM_STAGES = 4;
constexpr unsigned long long GEMM_WAIT_NS = 1000000000ull;   // 1 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor of a K-major SWIZZLE_128B tile (tcgen05
// format: start >> 4 in bits 0-13, leading byte offset >> 4 in 16-29 (unused
// for swizzled K-major tiles whose K step fits the 128-byte row; 16), stride
// byte offset >> 4 in 32-45 (1024: from one 8-row group to the next), the
// fixed 0b001 in 46-48, base offset 0 (tiles start on 1024-byte
// boundaries), layout type 2 = 128-byte swizzle in 61-63).  A K step of 16
// BF16 inside the row advances the start by 32 bytes; the swizzle is applied
// to the resulting addresses.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Wait until the phase of the given parity has completed, or GEMM_WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    const unsigned long long deadline = global_ns() + GEMM_WAIT_NS;
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (global_ns() > deadline) return false;
    }
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// 2D TMA load of one box at (x, y) into shared memory, completing on mbar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(mbar)
                 : "memory");
}

struct GemmArgs {
    const float *bias;          // [N] or null
    float *Cf;                  // FP32 output (or split-K partials) or null
    __nv_bfloat16 *Cb;          // BF16 output or null
    int M, N, K;                // K multiple of 64
    int ldc;                    // row stride of C (elements)
    int relu;
    int split_k;                // >= 1; > 1 writes partials Cf[z][M][ldc]
    int inject;                 // test only: the MMA lane waits on a barrier nothing arrives at
    int *status;                // error flag (1: an mbarrier wait gave up)
};

template <int BN>
struct GemmSmem {
    static constexpr uint32_t A_BYTES = GEMM_BM * GEMM_BK * 2;
    static constexpr uint32_t B_BYTES = BN * GEMM_BK * 2;
    static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    static constexpr size_t TOTAL = (size_t)GEMM_STAGES * STAGE + 1024;   // + alignment slack
};

template <int BN>
__global__ void __launch_bounds__(GEMM_THREADS)
k_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs g)
{
    using SM = GemmSmem<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar_full[GEMM_STAGES], bar_empty[GEMM_STAGES], bar_done, bar_never;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * GEMM_BM, n0 = blockIdx.y * BN;
    const int kz = blockIdx.z;
    const int k_per = g.K / g.split_k;                  // multiple of 64 by construction
    const int kbeg = kz * k_per;
    const int n_k = k_per / GEMM_BK;
    constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;   // power of two >= 32
    constexpr uint32_t IDESC = instr_desc_bf16(GEMM_BM, BN);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        abort_s = 0;
        for (int s = 0; s < GEMM_STAGES; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_done), 1);
        mbar_init(smem_u32(&bar_never), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s;
    const uint32_t sbase = smem_u32(smem);

    if (tid == 0) {
        // ---- loader: K step it into stage it % GEMM_STAGES ------------------
        int issued = 0;
        for (int it = 0; it < n_k; ++it) {
            const int s = it % GEMM_STAGES;
            const uint32_t ph = (uint32_t)(it / GEMM_STAGES) & 1u;
            // the stage is free once the MMAs of K step it - GEMM_STAGES have read it
            if (it >= GEMM_STAGES && !mbar_wait(smem_u32(&bar_empty[s]), ph ^ 1u)) {
                abort_s = 1;
                if (g.status) atomicExch(g.status, 1);
                break;
            }
            if (abort_s) break;
            const uint32_t sa = sbase + s * SM::STAGE, sb = sa + SM::A_BYTES;
            const uint32_t fb = smem_u32(&bar_full[s]);
            mbar_expect_tx(fb, SM::STAGE);
            const int k0 = kbeg + it * GEMM_BK;
            tma_load_2d(sa, &tmA, k0, m0, fb);
            tma_load_2d(sb, &tmB, k0, n0, fb);
            ++issued;
        }
        // copies still in flight land before the CTA may exit: the last one
        // issued on each stage completes that stage's current phase
        for (int it = issued - GEMM_STAGES < 0 ? 0 : issued - GEMM_STAGES; it < issued; ++it)
            if (!mbar_wait(smem_u32(&bar_full[it % GEMM_STAGES]), (uint32_t)(it / GEMM_STAGES) & 1u) && g.status)
                atomicExch(g.status, 1);
    } else if (tid == 32) {
        // ---- MMA issuer ----------------------------------------------------------
        if (g.inject) {
            // test only: a wait that nothing completes runs out
            if (!mbar_wait(smem_u32(&bar_never), 0u)) {
                abort_s = 1;
                if (g.status) atomicExch(g.status, 1);
            }
        }
        for (int it = 0; it < n_k && !abort_s; ++it) {
            const int s = it % GEMM_STAGES;
            const uint32_t ph = (uint32_t)(it / GEMM_STAGES) & 1u;
            if (!mbar_wait(smem_u32(&bar_full[s]), ph)) {
                abort_s = 1;
                if (g.status) atomicExch(g.status, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = sbase + s * SM::STAGE, sb = sa + SM::A_BYTES;
#pragma unroll
            for (int j = 0; j < GEMM_BK / 16; ++j) {
                // K step j: 16 BF16 = 32 bytes further along the 128-byte rows
                const uint64_t da = smem_desc_sw128(sa + 32 * j);
                const uint64_t db = smem_desc_sw128(sb + 32 * j);
                const uint32_t acc = (it > 0 || j > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\t"
                             "setp.ne.u32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(da), "l"(db), "r"(IDESC), "r"(acc)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&bar_empty[s]))
                         : "memory");
        }
        // "done" completes once every MMA this lane issued has finished
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&bar_done))
                     : "memory");
    }
    __syncwarp();
    __syncthreads();
    if (!mbar_wait(smem_u32(&bar_done), 0u)) {
        abort_s = 1;
        if (g.status) atomicExch(g.status, 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();

    // ---- epilogue: TMEM -> registers -> global ------------------------------
    if (!abort_s) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        const bool any = n_k > 0;
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

// ---- tensor maps ---------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// Row-major BF16 matrix [rows][ld] (K = cols used), boxes of 64 K-elements
// (128 bytes) by box_rows rows, 128-byte swizzle; rows beyond `rows` read 0.
static cudaError_t make_map(CUtensorMap *map, const __nv_bfloat16 *base, int rows, int cols, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t stride[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    const cuuint32_t estride[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dim, stride, box, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN>
static cudaError_t gemm_t(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int lda, int ldb, const GemmArgs &g,
                          cudaStream_t st)
{
    CUtensorMap ma, mb;
    cudaError_t e = make_map(&ma, A, g.M, g.K, lda, GEMM_BM);
    if (e == cudaSuccess) e = make_map(&mb, B, g.N, g.K, ldb, BN);
    if (e != cudaSuccess) return e;
    constexpr size_t SMEM = GemmSmem<BN>::TOTAL;
    e = cudaFuncSetAttribute(k_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)ceil_div(g.M, GEMM_BM), (unsigned)ceil_div(g.N, BN), (unsigned)g.split_k);
    k_gemm_bf16<BN><<<grid, GEMM_THREADS, SMEM, st>>>(ma, mb, g);
    return cudaGetLastError();
}

// C = A B^T (+ bias, ReLU).  Requirements: K % 64 == 0, K / split_k % 64 == 0,
// lda, ldb multiples of 8 (16-byte rows), 16-byte aligned A and B.
// split_k > 1 needs `partials` (split_k * M * ldc floats).  inject != 0, or a
// pending FAULT_GEMM_WAIT injection (tests only), makes the CTAs' MMA lanes
// wait on a barrier nothing completes: every CTA gives up after the wait
// limit, issues no MMA and sets *status.
cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias, float *Cf,
                             __nv_bfloat16 *Cb, int M, int N, int K, int lda, int ldb, int ldc, int relu, int split_k,
                             float *partials, int *status, cudaStream_t st, int inject)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (K % GEMM_BK || split_k < 1 || (K / split_k) % GEMM_BK || (lda % 8) || (ldb % 8) ||
        ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || (split_k > 1 && !partials))
        return cudaErrorInvalidValue;
    if (take_fault(FAULT_GEMM_WAIT)) inject = 1;
    GemmArgs g{bias, Cf, Cb, M, N, K, ldc, relu, split_k, inject, status};
    if (split_k > 1) {
        g.Cf = partials;
        g.Cb = nullptr;
        g.bias = nullptr;
        g.relu = 0;
    }
    const int BN = N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
    cudaError_t e;
    switch (BN) {
    case 16: e = gemm_t<16>(A, B, lda, ldb, g, st); break;
    case 32: e = gemm_t<32>(A, B, lda, ldb, g, st); break;
    case 64: e = gemm_t<64>(A, B, lda, ldb, g, st); break;
    case 128: e = gemm_t<128>(A, B, lda, ldb, g, st); break;
    default: e = gemm_t<256>(A, B, lda, ldb, g, st); break;
    }
    if (e != cudaSuccess || split_k == 1) return e;
    const int64_t n = (int64_t)M * N;
    k_gemm_reduce<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(partials, split_k, M, N, ldc, bias, relu, Cf, Cb);
    return cudaGetLastError();
}

}  // namespace reloc
