// Peak arithmetic throughput of the SIMT pipes, measured (the roofline
// denominators of the element-integral kernels, which are bound by FP32
// fused multiply-adds, and of the FP64 forms).
//
// Every thread runs kChains independent FMA chains x = x * a + b for `iters`
// rounds; the chains keep the pipe busy without memory traffic.  The grid is
// blocks_per_sm x the SM count; 2 flop per FMA.
#include <algorithm>

#include "internal.h"

namespace dnnmg {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T a, T b, T* __restrict__ sink) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink[int64_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t probe(int iters, int blocks_per_sm, double* tflops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * blocks_per_sm, threads = 256;
    T* sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(&sink, size_t(blocks) * threads * sizeof(T))) != cudaSuccess) return e;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    // a value near 1 keeps the chains finite; b != 0 keeps them from folding
    const T a = T(0.999999), b = T(1e-7);
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {   // the first is a warm-up
        cudaEventRecord(e0, s);
        fma_probe_kernel<T><<<blocks, threads, 0, s>>>(iters, a, b, sink);
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) {
        const double flop = 2.0 * kChains * double(iters) * double(blocks) * threads;
        *tflops = flop / (double(best) * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    return e;
}

}  // namespace
}  // namespace dnnmg

extern "C" dnnmg_status dnnmg_probe_fma(int32_t precision, int32_t iters, int32_t blocks_per_sm, double* tflops) {
    if (!tflops || iters <= 0 || blocks_per_sm <= 0 || blocks_per_sm > 64 ||
        (precision != DNNMG_FP64 && precision != DNNMG_FP32))
        return DNNMG_EINVAL;
    cudaError_t e = precision == DNNMG_FP64 ? dnnmg::probe<double>(iters, blocks_per_sm, tflops)
                                            : dnnmg::probe<float>(iters, blocks_per_sm, tflops);
    return e == cudaSuccess ? DNNMG_OK : (e == cudaErrorMemoryAllocation ? DNNMG_ENOMEM : DNNMG_ECUDA);
}
