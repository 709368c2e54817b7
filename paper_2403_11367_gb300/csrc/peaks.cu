// peaks.cu -- measured FP32 and exponential throughput of this GPU, the
// denominators of the blend's and projection's rooflines (their work is FP32
// arithmetic and exponentials, not memory traffic or tensor-core math).
//
// Each kernel keeps a set of independent register-resident dependency chains
// per thread, long enough that launch and tail effects are below 1%, on a
// grid of several waves of the SM count.  Results are written only when an
// impossible value appears, so the compiler keeps the arithmetic.
#include "internal.cuh"

namespace reloc {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_ITERS = 4096;

__global__ void __launch_bounds__(PEAK_THREADS) k_peak_ffma(float b, float c, float *sink)
{
    float a[PEAK_CHAINS];
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int it = 0; it < PEAK_ITERS; ++it) {
#pragma unroll
        for (int j = 0; j < PEAK_CHAINS; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) s += a[j];
    if (s == -1.f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) k_peak_ffma2(float b, float c, float *sink)
{
    unsigned long long a[PEAK_CHAINS], bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) {
        const float x = (float)(threadIdx.x + j) * 1e-3f;
        asm("mov.b64 %0, {%1, %1};" : "=l"(a[j]) : "f"(x));
    }
    for (int it = 0; it < PEAK_ITERS; ++it) {
#pragma unroll
        for (int j = 0; j < PEAK_CHAINS; ++j) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[j]));
        s += lo + hi;
    }
    if (s == -1.f) sink[threadIdx.x] = s;
}

// x <- 2^x - 1 keeps x in [-1, 0]: one ex2.approx and one add per step.
__global__ void __launch_bounds__(PEAK_THREADS) k_peak_ex2(float *sink)
{
    float a[PEAK_CHAINS];
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) a[j] = -(float)((threadIdx.x + j) & 63) * (1.f / 64.f);
    for (int it = 0; it < PEAK_ITERS / 4; ++it) {
#pragma unroll
        for (int j = 0; j < PEAK_CHAINS; ++j) {
            float y;
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[j]));
            a[j] = y - 1.f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) s += a[j];
    if (s == 1e30f) sink[threadIdx.x] = s;
}

cudaError_t measure_peaks(double *fp32_scalar_tflops, double *fp32_packed_tflops, double *ex2_gops)
{
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    float *sink = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaMalloc(&sink, PEAK_THREADS * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks = n_sm * 8 * 4;                        // four waves of 8 blocks per SM
    const double threads = (double)blocks * PEAK_THREADS;
    auto timed = [&](int which, double ops_per_thread, double *out) {
        if (e != cudaSuccess) return;
        for (int rep = 0; rep < 2; ++rep) {                 // first launch warms up
            cudaEventRecord(t0);
            if (which == 0) k_peak_ffma<<<blocks, PEAK_THREADS>>>(0.999f, 1e-3f, sink);
            else if (which == 1) k_peak_ffma2<<<blocks, PEAK_THREADS>>>(0.999f, 1e-3f, sink);
            else k_peak_ex2<<<blocks, PEAK_THREADS>>>(sink);
            cudaEventRecord(t1);
            e = cudaEventSynchronize(t1);
            if (e != cudaSuccess) return;
        }
        e = cudaGetLastError();
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && out) *out = threads * ops_per_thread / (ms * 1e-3);
    };
    double f1 = 0, f2 = 0, x = 0;
    timed(0, 2.0 * PEAK_CHAINS * PEAK_ITERS, &f1);          // 2 flop per FMA
    timed(1, 4.0 * PEAK_CHAINS * PEAK_ITERS, &f2);          // 2 lanes x 2 flop per packed FMA
    timed(2, (double)PEAK_CHAINS * (PEAK_ITERS / 4), &x);   // one exponential per step
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return e;
    if (fp32_scalar_tflops) *fp32_scalar_tflops = f1 * 1e-12;
    if (fp32_packed_tflops) *fp32_packed_tflops = f2 * 1e-12;
    if (ex2_gops) *ex2_gops = x * 1e-9;
    return cudaSuccess;
}

}  // namespace reloc
