// kpx_peak.cu -- FP32 fused multiply-add throughput of the device, measured
// (the denominator of the planner kernels' FP32 roofline beside the one
// derived from unit counts and the clock).
//
// Every thread runs 16 independent FMA chains, so that four warps per SM
// sub-partition cover the FMA latency; the grid is 4 blocks of 256 threads
// per SM (32 warps per SM).  The chains' results are kept alive by a store
// to a file-scope device word that runs only when their sum is exactly zero
// (never, for these inputs); nothing is allocated.
#include <cuda_runtime.h>

#include <cstdint>

#include "kpx.h"

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 4;
constexpr int PEAK_CHAINS = 16;

__device__ float g_fma_sink;

__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(int iters) {
    float a[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = 1.0f + 1e-3f * (float)(threadIdx.x + c);
    const float b = 0.999999f, d = 1e-6f;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; ++c) a[c] = fmaf(a[c], b, d);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += a[c];
    if (s == 0.0f) g_fma_sink = s;
}

}  // namespace

extern "C" kpx_status kpx_fp32_fma_rate(int32_t iters, double* tflops, void* cuda_stream) {
    if (!tflops || iters < 1 || iters > (1 << 20)) return KPX_E_INVALID;
    *tflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return KPX_E_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int blocks = sms * PEAK_BLOCKS_PER_SM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fma_peak<<<blocks, PEAK_THREADS, 0, s>>>(iters);  // warm-up (clocks, instruction cache)
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        k_fma_peak<<<blocks, PEAK_THREADS, 0, s>>>(iters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess || !(ms > 0.0f)) return KPX_E_CUDA;
    const double flops = 2.0 * PEAK_CHAINS * (double)iters * blocks * PEAK_THREADS;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return KPX_OK;
}
