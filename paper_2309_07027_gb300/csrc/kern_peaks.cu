// Issue-rate microbenchmark for the FP64 and FP32 fused multiply-add pipes.
//
// Every thread runs 8 independent FMA chains (enough independent work to
// keep the pipe busy at full occupancy); the grid fills every SM 8 CTAs
// deep.  The best of three timed runs (CUDA events) gives lane-FMAs per
// second, the denominator of the walk kernels' ALU roofline (2 flops per
// FMA).
#include <cuda_runtime.h>
#include "kernels.h"

namespace bs {

constexpr int kChains = 8;
constexpr int kInner = 8;

template <typename T>
__global__ void fma_rate_kernel(T* out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x * 1e-3) + (T)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kInner; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    // never true for these inputs; keeps the chains live
    if (s == (T)-1234.5) out[0] = s;
}

int sm_count(int device) {
    static int cached[64] = {0};
    if (device >= 0 && device < 64 && cached[device] > 0) return cached[device];
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
    if (n < 1) n = 1;
    if (device >= 0 && device < 64) cached[device] = n;
    return n;
}

template <typename T>
static cudaError_t time_rate(int iters, double* rate) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int threads = 256;
    const int blocks = sm_count(dev) * 8;
    T* out = nullptr;
    cudaError_t e = cudaMalloc(&out, 64);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_rate_kernel<T><<<blocks, threads>>>(out, iters / 8 + 1, (T)0.9999, (T)1e-4);
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0);
        fma_rate_kernel<T><<<blocks, threads>>>(out, iters, (T)0.9999, (T)1e-4);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    double ops = (double)threads * blocks * (double)iters * kInner * kChains;
    *rate = ops / (best * 1e-3);
    return cudaSuccess;
}

cudaError_t measure_fma_rates(int device, double* fp64_per_s, double* fp32_per_s) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    e = time_rate<double>(3000, fp64_per_s);
    if (e != cudaSuccess) return e;
    return time_rate<float>(150000, fp32_per_s);
}

}  // namespace bs
