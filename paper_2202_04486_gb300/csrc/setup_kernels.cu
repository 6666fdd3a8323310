// Step-size setup (Appendix B): the largest singular value of the MDC operator equals that of its
// frequency-domain kernel, so sigma^2_max = max_f lambda_max(Dh_f^H Dh_f), Dh_f the ns x nr matrix of
// the down-going spectrum at bin f.  One CTA runs a power iteration per bin with FP64 accumulation;
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

__global__ void __launch_bounds__(PI_THREADS) k_power_iter(const float2 *__restrict__ Dh, int ns, int nr, int ldr,
                                                           long long sDf, int n_iter, double *lam) {
    extern __shared__ double2 psm[];
    __shared__ double red[32];
    double2 *v = psm, *u = psm + nr, *w = psm + 2 * nr;
    const int f = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = PI_THREADS / 32;
    const float2 *Df = Dh + (long long)f * sDf;

    // deterministic start vector with no special structure
    for (int r = tid; r < nr; r += PI_THREADS) v[r] = make_double2(1.0 + 0.1 * (r % 7), 0.05 * (r % 5));
    __syncthreads();
    double vv = 0.0;
    for (int r = tid; r < nr; r += PI_THREADS) vv += v[r].x * v[r].x + v[r].y * v[r].y;
    vv = block_allsum(vv, red);

    double result = 0.0;
    for (int it = 0; it < n_iter; ++it) {
        // w = Dh_f v  (warp per row s, lanes along r)
        for (int s = warp; s < ns; s += nwarp) {
            double re = 0.0, im = 0.0;
            const float2 *row = Df + (long long)s * ldr;
            for (int r = lane; r < nr; r += 32) {
                const float2 d = row[r];
                const double2 x = v[r];
                re += (double)d.x * x.x - (double)d.y * x.y;
                im += (double)d.x * x.y + (double)d.y * x.x;
            }
            re = warp_sum(re);
            im = warp_sum(im);
            if (lane == 0) w[s] = make_double2(re, im);
        }
        __syncthreads();
        // u = Dh_f^H w  (thread per column r, rows streamed: coalesced across the warp)
        for (int r = tid; r < nr; r += PI_THREADS) {
            double re = 0.0, im = 0.0;
            for (int s = 0; s < ns; ++s) {
                const float2 d = Df[(long long)s * ldr + r];
                const double2 y = w[s];
                re += (double)d.x * y.x + (double)d.y * y.y;   // conj(d) * y
                im += (double)d.x * y.y - (double)d.y * y.x;
            }
            u[r] = make_double2(re, im);
        }
        double ww = 0.0;
        for (int s = tid; s < ns; s += PI_THREADS) ww += w[s].x * w[s].x + w[s].y * w[s].y;
        ww = block_allsum(ww, red);   // includes the barrier that publishes u
        double uu = 0.0;
        for (int r = tid; r < nr; r += PI_THREADS) uu += u[r].x * u[r].x + u[r].y * u[r].y;
        uu = block_allsum(uu, red);
        result = (vv > 0.0) ? ww / vv : 0.0;
        if (!(uu > 0.0)) break;
        const double inv = 1.0 / sqrt(uu);
        for (int r = tid; r < nr; r += PI_THREADS) v[r] = make_double2(u[r].x * inv, u[r].y * inv);
        vv = 1.0;
        __syncthreads();
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
    const size_t smem = (size_t)(2 * nr + ns) * sizeof(double2);
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
