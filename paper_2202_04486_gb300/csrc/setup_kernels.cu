// Step-size setup (Appendix B): the largest singular value of the MDC operator equals that of its
// frequency-domain kernel, so sigma^2_max = max_f lambda_max(Dh_f^H Dh_f), Dh_f the ns x nr matrix of
// the down-going spectrum at bin f.  One CTA runs a power iteration per bin (FP32 products, FP64 norms);
// the Rayleigh quotient ||Dh_f v||^2 / ||v||^2 of the last iterate is a lower bound that converges to
// lambda_max as the iteration count grows.
#include "smdd_fft.cuh"
#include "smdd_internal.h"

namespace smdd {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of v; every thread gets the result (red holds 32 doubles)
__device__ __forceinline__ double block_allsum(double v, double *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += red[i];
    return s;
}

constexpr int PI_THREADS = 256;

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The matrix-vector products run in FP32 (the FP64 units of this GPU are a small fraction of its FP32
// rate); the norms and the Rayleigh quotient are accumulated in FP64.  FP32 rounding changes the
// quotient by ~1e-6 relative, far below what the step size needs.
__global__ void __launch_bounds__(PI_THREADS) k_power_iter(const float2 *__restrict__ Dh, int ns, int nr, int ldr,
                                                           long long sDf, int n_iter, double *lam) {
    extern __shared__ float2 pvs[];
    __shared__ double red[32];
    float2 *v = pvs, *u = pvs + nr, *w = pvs + 2 * nr;
    const int f = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = PI_THREADS / 32;
    const float2 *Df = Dh + (long long)f * sDf;

    // deterministic start vector with no special structure
    for (int r = tid; r < nr; r += PI_THREADS) v[r] = make_float2(1.0f + 0.1f * (r % 7), 0.05f * (r % 5));
    __syncthreads();
    double vv = 0.0;
    for (int r = tid; r < nr; r += PI_THREADS) vv += (double)v[r].x * v[r].x + (double)v[r].y * v[r].y;
    vv = block_allsum(vv, red);

    double result = 0.0;
    for (int it = 0; it < n_iter; ++it) {
        // w = Dh_f v  (warp per row s, lanes along r)
        for (int s = warp; s < ns; s += nwarp) {
            float re = 0.f, im = 0.f;
            const float2 *row = Df + (long long)s * ldr;
            for (int r = lane; r < nr; r += 32) {
                const float2 d = __ldg(row + r);
                const float2 x = v[r];
                re = fmaf(d.x, x.x, fmaf(-d.y, x.y, re));
                im = fmaf(d.x, x.y, fmaf(d.y, x.x, im));
            }
            re = warp_sumf(re);
            im = warp_sumf(im);
            if (lane == 0) w[s] = make_float2(re, im);
        }
        __syncthreads();
        // u = Dh_f^H w  (thread per column r, rows streamed: coalesced across the warp)
        for (int r = tid; r < nr; r += PI_THREADS) {
            float re = 0.f, im = 0.f;
            for (int s = 0; s < ns; ++s) {
                const float2 d = __ldg(Df + (long long)s * ldr + r);
                const float2 y = w[s];
                re = fmaf(d.x, y.x, fmaf(d.y, y.y, re));   // conj(d) * y
                im = fmaf(d.x, y.y, fmaf(-d.y, y.x, im));
            }
            u[r] = make_float2(re, im);
        }
        double ww = 0.0;
        for (int s = tid; s < ns; s += PI_THREADS) ww += (double)w[s].x * w[s].x + (double)w[s].y * w[s].y;
        ww = block_allsum(ww, red);   // includes the barrier that publishes u
        double uu = 0.0;
        for (int r = tid; r < nr; r += PI_THREADS) uu += (double)u[r].x * u[r].x + (double)u[r].y * u[r].y;
        uu = block_allsum(uu, red);
        result = (vv > 0.0) ? ww / vv : 0.0;
        if (!(uu > 0.0)) break;
        const double inv = 1.0 / sqrt(uu);
        double nv2 = 0.0;
        for (int r = tid; r < nr; r += PI_THREADS) {
            const float2 x = make_float2((float)(u[r].x * inv), (float)(u[r].y * inv));
            v[r] = x;
            nv2 += (double)x.x * x.x + (double)x.y * x.y;
        }
        vv = block_allsum(nv2, red);   // the norm of the rounded iterate; includes the barrier publishing v
    }
    if (tid == 0) lam[f] = result;
}

__global__ void k_max_reduce(const double *__restrict__ x, int n, double *out) {
    __shared__ double red[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, x[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) r = fmax(r, red[i]);
        *out = r;
    }
}

cudaError_t launch_power_iter(const float2 *Dh, int ns, int nr, int ldr, long long sDf, int nf, int n_iter,
                              double *lam, cudaStream_t st) {
    const size_t smem = (size_t)(2 * nr + ns) * sizeof(float2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_power_iter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_power_iter<<<nf, PI_THREADS, smem, st>>>(Dh, ns, nr, ldr, sDf, n_iter, lam);
    return cudaGetLastError();
}

cudaError_t launch_max_reduce(const double *lam, int n, double *out, cudaStream_t st) {
    k_max_reduce<<<1, 1024, 0, st>>>(lam, n, out);
    return cudaGetLastError();
}

}  // namespace smdd
