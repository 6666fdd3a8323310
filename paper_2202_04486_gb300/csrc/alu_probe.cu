// FMA throughput probes: the FP32 and FP64 arithmetic peaks of the device, measured rather than
// derived from lane counts and the nominal clock.  The FP32 figure is the denominator of the step
// roofline of the FP32 path (its FFTs and FMA products run on the CUDA cores); the FP64 figure is what
// decided that the set-up's power iteration takes its products in FP32 and only its norms in FP64.
//
// Each thread runs kChains independent multiply-add chains a <- a*b + c with |b| < 1, so the values
// stay normal and bounded, and writes the sum of its chains to sink[thread] so the compiler keeps every
// operation.  One launch performs blocks * kThreads * kChains * iters multiply-adds, two flops each.
#include <cstdint>

#include "smdd_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <typename T>
__device__ __forceinline__ T fma_op(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_op<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_op<double>(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(T *sink, int iters, T b, T c) {
    const int gid = blockIdx.x * kThreads + threadIdx.x;
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = T(gid & 1023) * T(1e-3) + T(i);
    // iters is a multiple of 16 (checked on the host): 16 rounds of all chains per loop trip keep the
    // loop's own instructions a few per cent of the issue slots
    for (int it = 0; it < iters; it += 16) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fma_op(a[i], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    sink[gid] = s;
}

}  // namespace

extern "C" int mdc_alu_probe(int kind, int blocks, int iters, void *sink, double *flops, void *stream) {
    if (kind < 0 || kind > 1 || blocks < 1 || iters < 16 || iters % 16 != 0 || !sink)
        return MDC_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (kind == 0)
        k_fma_probe<float><<<blocks, kThreads, 0, st>>>(static_cast<float *>(sink), iters, 0.9990234375f, 1e-3f);
    else
        k_fma_probe<double><<<blocks, kThreads, 0, st>>>(static_cast<double *>(sink), iters, 0.9990234375, 1e-3);
    if (cudaGetLastError() != cudaSuccess) return MDC_ERR_CUDA;
    if (flops) *flops = 2.0 * double(blocks) * kThreads * kChains * double(iters);
    return MDC_OK;
}
