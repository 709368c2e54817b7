// noalloc.cu -- NCC scoring of images the caller has already rendered, for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: a relocalization
// loop on a robot that reserves all device memory at start-up and then runs
// under a real-time budget (cudaMalloc and cudaFree may synchronise the whole
// device and take milliseconds), or a host process whose device memory is
// owned by another framework's pool.  reloc_ncc_images_noalloc serves them:
// it computes the same NCC (all 3*H*W samples, FP64 sums) as the scoring
// stage of reloc_score, but its only scratch is the file-scope device array
// below, so the call allocates nothing.
//
// The array is fixed at load time and every GPU that loads the library holds
// it until the process exits.  Its device address is looked up once per
// device (cudaGetSymbolAddress with that device current) on the first call
// made on that device; that first call should therefore come before any
// stream capture.  Every call overwrites the slots it reads before reading
// them, so nothing needs clearing between calls, but all calls share the one
// array: calls whose kernels overlap on the GPU (different streams, or
// different host threads on the same device) race on it and must be ordered
// by the caller.
#include <mutex>

#include "internal.cuh"
#include "reloc.h"

namespace reloc {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_BLOCKS = 32;                         // partial sums per image
constexpr int64_t NOALLOC_SCRATCH_DOUBLES =
    (int64_t)RELOC_NOALLOC_MAX_VIEWS * NOALLOC_BLOCKS * 3 + NOALLOC_BLOCKS * 2;

// 393,728 bytes: [view][block][S_r, S_rr, S_rq], then [block][S_q, S_qq].
static __device__ __align__(256) double g_ncc_scratch[NOALLOC_SCRATCH_DOUBLES];

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// grid (NOALLOC_BLOCKS, V + 1): row v < V sums image v against the query,
// row V sums the query alone.  Fixed grid and reduction order: deterministic.
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_ncc_partials_noalloc(const float *__restrict__ images, const float *__restrict__ query, int V, int64_t n,
                       double *__restrict__ scratch)
{
    __shared__ double s[3][NOALLOC_THREADS / 32];
    const int v = blockIdx.y;
    const bool is_query = v == V;
    const float *img = images + (int64_t)(is_query ? 0 : v) * n;
    double a = 0, b = 0, c = 0;
    for (int64_t j = (int64_t)blockIdx.x * NOALLOC_THREADS + threadIdx.x; j < n;
         j += (int64_t)NOALLOC_BLOCKS * NOALLOC_THREADS) {
        const double q = query[j];
        if (is_query) {
            a += q;
            b += q * q;
        } else {
            const double r = img[j];
            a += r;
            b += r * r;
            c += r * q;
        }
    }
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s[0][w] = a; s[1][w] = b; s[2][w] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0, B = 0, Cc = 0;
        for (int k = 0; k < NOALLOC_THREADS / 32; ++k) { A += s[0][k]; B += s[1][k]; Cc += s[2][k]; }
        if (is_query) {
            double *o = scratch + (int64_t)RELOC_NOALLOC_MAX_VIEWS * NOALLOC_BLOCKS * 3 + 2 * blockIdx.x;
            o[0] = A;
            o[1] = B;
        } else {
            double *o = scratch + ((int64_t)v * NOALLOC_BLOCKS + blockIdx.x) * 3;
            o[0] = A;
            o[1] = B;
            o[2] = Cc;
        }
    }
}

__global__ void k_ncc_final_noalloc(const double *__restrict__ scratch, int V, int64_t n, double *__restrict__ scores,
                                    int *__restrict__ degenerate)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const double *qp = scratch + (int64_t)RELOC_NOALLOC_MAX_VIEWS * NOALLOC_BLOCKS * 3;
    double Sq = 0, Sqq = 0, Sr = 0, Srr = 0, Srq = 0;
    for (int k = 0; k < NOALLOC_BLOCKS; ++k) {
        Sq += qp[2 * k];
        Sqq += qp[2 * k + 1];
        const double *p = scratch + ((int64_t)v * NOALLOC_BLOCKS + k) * 3;
        Sr += p[0];
        Srr += p[1];
        Srq += p[2];
    }
    const double nn = (double)n;
    const double cov = Srq - Sr * Sq / nn;
    const double vr = Srr - Sr * Sr / nn;
    const double vq = Sqq - Sq * Sq / nn;
    const bool dg = !(vr > 1e-12 * nn) || !(vq > 1e-12 * nn);
    scores[v] = dg ? 0.0 : cov / (sqrt(vr) * sqrt(vq));
    if (degenerate) degenerate[v] = dg ? 1 : 0;
}

// Device address of g_ncc_scratch, looked up once per device.
static double *scratch_address(int device, cudaError_t *err)
{
    static std::mutex mu;
    static double *addr[256] = {};
    std::lock_guard<std::mutex> lock(mu);
    *err = cudaSuccess;
    if (device < 0 || device >= 256) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    if (!addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_ncc_scratch);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        addr[device] = (double *)p;
    }
    return addr[device];
}

}  // namespace reloc

using namespace reloc;

extern "C" reloc_status reloc_ncc_images_noalloc(const float *images_dev, int n_views, int height, int width,
                                                 const float *query_dev, double *scores_dev, int *degenerate_dev,
                                                 void *stream)
{
    if (!images_dev || !query_dev || !scores_dev)
        return reloc_internal_fail(RELOC_EINVAL, "reloc_ncc_images_noalloc: NULL image, query or score pointer");
    if (n_views < 1 || n_views > RELOC_NOALLOC_MAX_VIEWS)
        return reloc_internal_fail(RELOC_EINVAL, "reloc_ncc_images_noalloc: n_views must be in 1..RELOC_NOALLOC_MAX_VIEWS (512)");
    if (height < 1 || width < 1 || height > 16383 || width > 16383)
        return reloc_internal_fail(RELOC_EINVAL, "reloc_ncc_images_noalloc: image size out of range");
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return reloc_internal_fail(RELOC_ECUDA, cudaGetErrorString(e));
    double *scratch = scratch_address(device, &e);
    if (!scratch) return reloc_internal_fail(RELOC_ECUDA, cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = 3 * (int64_t)height * width;
    k_ncc_partials_noalloc<<<dim3(NOALLOC_BLOCKS, n_views + 1), NOALLOC_THREADS, 0, st>>>(images_dev, query_dev,
                                                                                      n_views, n, scratch);
    k_ncc_final_noalloc<<<(n_views + 127) / 128, 128, 0, st>>>(scratch, n_views, n, scores_dev, degenerate_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return reloc_internal_fail(RELOC_ECUDA, cudaGetErrorString(e));
    return RELOC_OK;
}
