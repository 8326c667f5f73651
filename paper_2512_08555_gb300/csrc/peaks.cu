// Arithmetic peak of the current device, measured: the FP64 (or FP32) FMA
// throughput that bounds the plain FP64 stencil kernels, whose flops per
// byte sit far above the FP64 ridge of this GPU.  Each thread runs 8
// independent FMA chains (enough to cover the FMA pipe latency); the grid
// fills every SM several times over.  Timed with CUDA events, best of 3.
#include "mrp_internal.h"

namespace mrp {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* __restrict__ sink, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == T(-1)) sink[blockIdx.x] = s;      // never true: keeps the chains live
}

template <typename T>
static int fma_peak(double* tflops, cudaStream_t s) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MRP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MRP_ERR_CUDA;
    const int blocks = nsm * 8, threads = 256;
    const int iters = sizeof(T) == 8 ? 4096 : 65536;
    T* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return MRP_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = T(0.999999), b = T(1e-7);
    k_fma_chains<T><<<blocks, threads, 0, s>>>(sink, iters, a, b);
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, s);
        k_fma_chains<T><<<blocks, threads, 0, s>>>(sink, iters, a, b);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (cudaGetLastError() != cudaSuccess || best >= 1e30f) return MRP_ERR_CUDA;
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return MRP_OK;
}

}  // namespace mrp

extern "C" int mrp_fma_peak(int32_t precision, double* tflops, void* stream) {
    if (!tflops || (precision != MRP_FP64 && precision != MRP_MIXED)) return MRP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == MRP_FP64 ? mrp::fma_peak<double>(tflops, s) : mrp::fma_peak<float>(tflops, s);
}
