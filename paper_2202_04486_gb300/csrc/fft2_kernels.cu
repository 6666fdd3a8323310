// The trace kernels of fft_kernels.cu (rfft, irfft with window, residual step, update step) on the
// register FFTs of radix-order variant 2: the two-pass FFT of smdd_fft2.cuh (128 <= M <= 1024; a team of
// M/32 threads per trace, 32 values per thread, one shared-memory exchange per transform) and the
// three-pass FFT of smdd_fft3.cuh (M = 1536; a warp per trace, 48 values per thread, two exchanges).
// Same arguments, same results as the radix kernels; the real-signal post-processing through warp
// shuffles.
//
// Time samples: thread t of a team holds z[n] = (x[2n], x[2n+1]) for n = t + T m, so for every m the
// team reads / writes 2T consecutive samples.
#include <cmath>
#include <vector>

#include "smdd_fft2.cuh"
#include "smdd_fft3.cuh"
#include "smdd_internal.h"
#include "work_queue.cuh"

namespace smdd {

namespace {

// Traits of the register FFTs: P values per thread, T threads per trace, TR traces per CTA; fwd / inv
// run the real transforms between the registers (time samples z[n], n = t + T m, m < P / 2) and the
// trace's shared-memory spectrum.  PREFETCH: the time-domain operand of the update / residual is loaded
// into registers before the inverse transform (where the registers allow it), else right after it.
template <int M>
struct RegFft {
    using F = Fft2<M>;
    static constexpr int P = F::P, T = F::T, TR = F::TR, THREADS = F::THREADS, STRIDE = F::STRIDE;
    static constexpr size_t SMEM = F::SMEM;
    static constexpr bool PREFETCH = true;
    __device__ static void fwd(float2 (&a)[P], float2 *buf, int t, const float2 *tw, const float2 *twN) {
        rfft2_regs_to_smem<M>(a, buf, t, tw, twN);
    }
    __device__ static void inv(float2 (&a)[P], float2 *buf, int t, const float2 *tw, const float2 *twN) {
        irfft2_smem_to_regs<M>(a, buf, t, tw, twN);
    }
};

template <>
struct RegFft<1536> {
    using F = Fft3;
    static constexpr int P = F::P, T = F::T, TR = F::TR, THREADS = F::THREADS, STRIDE = F::STRIDE;
    static constexpr size_t SMEM = F::SMEM;
    static constexpr bool PREFETCH = false;   // 48 values per thread already fill most of the registers
    __device__ static void fwd(float2 (&a)[P], float2 *buf, int t, const float2 *tw, const float2 *twN) {
        rfft3_regs_to_smem(a, buf, t, tw, twN);
    }
    __device__ static void inv(float2 (&a)[P], float2 *buf, int t, const float2 *tw, const float2 *twN) {
        irfft3_smem_to_regs(a, buf, t, tw, twN);
    }
};

struct TileCoord2 {
    int i, j;
    bool valid;
};

// tile bid of the grid (blockIdx.x in a plain launch, the dequeued tile in a work-queue launch)
template <int M>
__device__ __forceinline__ TileCoord2 coord2_of(const TraceGrid &g, int tr, int bid) {
    constexpr int TR = RegFft<M>::TR;
    const int ti = 1 << g.ti_log2;
    const int tj = TR >> g.ti_log2;
    const int ntile_i = (g.ni + ti - 1) / ti;
    const int bi = bid % ntile_i, bj = bid / ntile_i;
    TileCoord2 c;
    c.i = bi * ti + (tr & (ti - 1));
    c.j = bj * tj + (tr >> g.ti_log2);
    c.valid = c.i < g.ni && c.j < g.nj;
    return c;
}

// spectra of the CTA's traces -> shared memory (slot 0 = (Re X[0], Re X[M])); thread binding: trace
// tr = tid % TR, bins f = tid / TR + it * (THREADS / TR)
template <int M>
__device__ __forceinline__ void tile2_load(float2 *sm, const float2 *__restrict__ spec, const TraceGrid &g, int bid) {
    using F = RegFft<M>;
    constexpr int TR = F::TR, STR = F::STRIDE, STEP = F::THREADS / TR, NIT = M / STEP;
    const int tr = threadIdx.x % TR, f0 = threadIdx.x / TR;
    const TileCoord2 c = coord2_of<M>(g, tr, bid);
    float2 v[NIT];
    float nyq = 0.f;
    if (c.valid) {
        const float2 *s = spec + (long long)c.i * g.ssi + (long long)c.j * g.ssj;
#pragma unroll
        for (int it = 0; it < NIT; ++it) v[it] = __ldcs(s + (long long)(f0 + it * STEP) * g.ssf);
        if (f0 == 0) nyq = __ldcs(s + (long long)M * g.ssf).x;
    } else {
#pragma unroll
        for (int it = 0; it < NIT; ++it) v[it] = make_float2(0.f, 0.f);
    }
    float2 *b = sm + tr * STR;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int f = f0 + it * STEP;
        b[pad2(f)] = (f == 0) ? make_float2(v[it].x, nyq) : v[it];
    }
}

template <int M>
__device__ __forceinline__ void tile2_store(const float2 *sm, float2 *__restrict__ spec, const TraceGrid &g, int bid) {
    using F = RegFft<M>;
    constexpr int TR = F::TR, STR = F::STRIDE, STEP = F::THREADS / TR, NIT = M / STEP;
    const int tr = threadIdx.x % TR, f0 = threadIdx.x / TR;
    const TileCoord2 c = coord2_of<M>(g, tr, bid);
    if (!c.valid) return;
    const float2 *b = sm + tr * STR;
    float2 *s = spec + (long long)c.i * g.ssi + (long long)c.j * g.ssj;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int f = f0 + it * STEP;
        const float2 v = b[pad2(f)];
        s[(long long)f * g.ssf] = (f == 0) ? make_float2(v.x, 0.f) : v;
    }
    if (f0 == 0) s[(long long)M * g.ssf] = make_float2(b[0].y, 0.f);
}

// the two samples of element n (window [0, nt)); vec: the trace may be read as float2
__device__ __forceinline__ float2 load_z(const float *x, int n, int nt, bool vec) {
    const int i0 = 2 * n;
    if (vec && i0 + 1 < nt) return __ldcs(reinterpret_cast<const float2 *>(x + i0));
    float2 z = make_float2(0.f, 0.f);
    if (i0 < nt) z.x = x[i0];
    if (i0 + 1 < nt) z.y = x[i0 + 1];
    return z;
}
__device__ __forceinline__ void store_z(float *y, int n, int nt, bool vec, float2 z) {
    const int i0 = 2 * n;
    if (vec && i0 + 1 < nt) {
        *reinterpret_cast<float2 *>(y + i0) = z;
    } else {
        if (i0 < nt) y[i0] = z.x;
        if (i0 + 1 < nt) y[i0 + 1] = z.y;
    }
}

template <int M>
__device__ __forceinline__ void rfft2_body(const FftArgs &a, int bid) {
    extern __shared__ __align__(16) float2 sm[];
    using F = RegFft<M>;
    constexpr int T = F::T, P = F::P;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    const TileCoord2 c = coord2_of<M>(a.g, tr, bid);
    float2 *buf = sm + tr * F::STRIDE;
    const float *x = a.tin + (c.valid ? (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj : 0);
    float2 v[P];
#pragma unroll
    for (int m = 0; m < P; ++m) v[m] = (m < P / 2 && c.valid) ? load_z(x, t + T * m, a.nt, a.vec) : make_float2(0.f, 0.f);
    F::fwd(v, buf, t, a.tw, a.twN);
    __syncthreads();
    tile2_store<M>(sm, a.spec, a.g, bid);
}

template <int M>
__global__ void __launch_bounds__(RegFft<M>::THREADS, 2) k2_rfft(FftArgs a) {
    rfft2_body<M>(a, blockIdx.x);
}

template <int M>
__global__ void __launch_bounds__(RegFft<M>::THREADS, 2) k2_irfft_out(FftArgs a) {
    const int bid = blockIdx.x;
    extern __shared__ __align__(16) float2 sm[];
    using F = RegFft<M>;
    constexpr int T = F::T, P = F::P;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    tile2_load<M>(sm, a.spec, a.g, bid);
    __syncthreads();
    const TileCoord2 c = coord2_of<M>(a.g, tr, bid);
    float2 *buf = sm + tr * F::STRIDE;
    float2 v[P];
    F::inv(v, buf, t, a.tw, a.twN);
    if (!c.valid) return;   // no barrier follows
    float *y = a.tout + (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj;
#pragma unroll
    for (int m = 0; m < P / 2; ++m) store_z(y, t + T * m, a.nt, a.vec, make_float2(v[m].x * a.s, v[m].y * a.s));
}

__device__ __forceinline__ double block_sum2(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();   // red may still be read by a previous call
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) s += red[i];
    return s;   // valid in thread 0
}

// residual step: R = s * irfft(Uh)[0:nt] - U_obs[row], FP64 loss partials, Rh = rfft(R) in place
template <int M>
__device__ __forceinline__ void residual2_body(const FftArgs &a, int bid, int nblk) {
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[32];
    __shared__ bool am_last;
    using F = RegFft<M>;
    constexpr int T = F::T, P = F::P;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    const TileCoord2 c = coord2_of<M>(a.g, tr, bid);
    const float *uo = nullptr;
    if (c.valid) {
        int row = c.i;
        if (!a.gathered) {
            row = a.idx[c.i];
            if (row < 0 || row >= a.ns) {
                atomicOr(a.status, 1);
                row = -1;
            }
        }
        if (row >= 0) uo = a.uobs + (long long)row * a.uo_si + (long long)c.j * a.uo_sj;
    }
    float2 o[P / 2];
    if constexpr (F::PREFETCH) {
#pragma unroll
        for (int m = 0; m < P / 2; ++m) o[m] = uo ? load_z(uo, t + T * m, a.nt, a.vec) : make_float2(0.f, 0.f);
    }
    tile2_load<M>(sm, a.spec, a.g, bid);
    __syncthreads();
    float2 *buf = sm + tr * F::STRIDE;
    float2 v[P];
    F::inv(v, buf, t, a.tw, a.twN);
    if constexpr (!F::PREFETCH) {
#pragma unroll
        for (int m = 0; m < P / 2; ++m) o[m] = uo ? load_z(uo, t + T * m, a.nt, a.vec) : make_float2(0.f, 0.f);
    }
    double l2 = 0.0;
#pragma unroll
    for (int m = 0; m < P; ++m) {
        if (m < P / 2) {
            const int i0 = 2 * (t + T * m);
            float2 q = make_float2(0.f, 0.f);
            if (c.valid) {
                q.x = (i0 < a.nt) ? fmaf(v[m].x, a.s, -o[m].x) : 0.f;
                q.y = (i0 + 1 < a.nt) ? fmaf(v[m].y, a.s, -o[m].y) : 0.f;
                l2 += (double)q.x * q.x + (double)q.y * q.y;
            }
            v[m] = q;
        } else {
            v[m] = make_float2(0.f, 0.f);
        }
    }
    F::fwd(v, buf, t, a.tw, a.twN);
    __syncthreads();
    tile2_store<M>(sm, a.spec, a.g, bid);

    const double bs = block_sum2(l2, red);
    if (threadIdx.x == 0) {
        a.partials[bid] = bs;
        __threadfence();
        const unsigned prev = atomicAdd(a.counter, 1u);
        am_last = (prev == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (am_last) {   // block-uniform
        __threadfence();
        double s = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += __ldcg(&a.partials[b]);
        s = block_sum2(s, red);   // fixed assignment and order: deterministic
        if (threadIdx.x == 0) {
            if (a.loss) *a.loss = 0.5 * s;
            *a.counter = 0u;
        }
    }
}

template <int M>
__global__ void __launch_bounds__(RegFft<M>::THREADS, 2) k2_residual(FftArgs a) {
    residual2_body<M>(a, blockIdx.x, gridDim.x);
}

// update step: g = s * irfft(Gh)[0:nt]; X <- X - alpha g; optionally Gh <- rfft(X_new) in place
template <int M, bool KEEP>
__device__ __forceinline__ void update2_body(const FftArgs &a, int bid) {
    extern __shared__ __align__(16) float2 sm[];
    using F = RegFft<M>;
    constexpr int T = F::T, P = F::P;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    const TileCoord2 c = coord2_of<M>(a.g, tr, bid);
    float *x = a.tout + (c.valid ? (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj : 0);
    float2 xo[P / 2];
    if constexpr (F::PREFETCH) {
#pragma unroll
        for (int m = 0; m < P / 2; ++m) xo[m] = c.valid ? load_z(x, t + T * m, a.nt, a.vec) : make_float2(0.f, 0.f);
    }
    tile2_load<M>(sm, a.spec, a.g, bid);
    __syncthreads();
    float2 *buf = sm + tr * F::STRIDE;
    float2 v[P];
    F::inv(v, buf, t, a.tw, a.twN);
    if constexpr (!F::PREFETCH) {
#pragma unroll
        for (int m = 0; m < P / 2; ++m) xo[m] = c.valid ? load_z(x, t + T * m, a.nt, a.vec) : make_float2(0.f, 0.f);
    }
    const float nas = -a.alpha * a.s;
#pragma unroll
    for (int m = 0; m < P; ++m) {
        if (m < P / 2) {
            const int n = t + T * m, i0 = 2 * n;
            float2 z;
            z.x = (i0 < a.nt) ? fmaf(nas, v[m].x, xo[m].x) : 0.f;
            z.y = (i0 + 1 < a.nt) ? fmaf(nas, v[m].y, xo[m].y) : 0.f;
            if (c.valid) store_z(x, n, a.nt, a.vec, z);
            v[m] = z;
        } else {
            v[m] = make_float2(0.f, 0.f);
        }
    }
    if constexpr (KEEP) {
        F::fwd(v, buf, t, a.tw, a.twN);
        __syncthreads();
        tile2_store<M>(sm, a.spec, a.g, bid);
    }
}

template <int M, bool KEEP>
__global__ void __launch_bounds__(RegFft<M>::THREADS, 2) k2_update(FftArgs a) {
    update2_body<M, KEEP>(a, blockIdx.x);
}

// work-queue forms: persistent CTAs taking (problem, tile) items until the queue is empty
template <int M>
__global__ void __launch_bounds__(RegFft<M>::THREADS, 2) k2_rfft_q(WorkQueue q) {
    const FftArgs *args = static_cast<const FftArgs *>(q.args);
    int m = 0, tile = 0;
    __shared__ FftArgs sa;
    while (queue_next(q, m, tile) >= 0) {
        queue_args(args + m, sa);
        __syncthreads();
        rfft2_body<M>(sa, tile);
    }
}

template <int M>
__global__ void __launch_bounds__(RegFft<M>::THREADS, 2) k2_residual_q(WorkQueue q) {
    const FftArgs *args = static_cast<const FftArgs *>(q.args);
    int m = 0, tile = 0;
    __shared__ FftArgs sa;
    while (queue_next(q, m, tile) >= 0) {
        queue_args(args + m, sa);
        __syncthreads();
        residual2_body<M>(sa, tile, __ldg(q.start + m + 1) - __ldg(q.start + m));
    }
}

template <int M>
__global__ void __launch_bounds__(RegFft<M>::THREADS, 2) k2_update_q(WorkQueue q) {
    const FftArgs *args = static_cast<const FftArgs *>(q.args);
    int m = 0, tile = 0;
    __shared__ FftArgs sa;
    while (queue_next(q, m, tile) >= 0) {
        queue_args(args + m, sa);
        __syncthreads();
        update2_body<M, true>(sa, tile);
    }
}

template <int M>
int blocks2_for(const TraceGrid &g) {
    // -1: the grid was laid out for CTAs of another trace count (more traces along i than a CTA holds)
    const int ti = 1 << g.ti_log2, tj = RegFft<M>::TR >> g.ti_log2;
    if (tj < 1) return -1;
    return ((g.ni + ti - 1) / ti) * ((g.nj + tj - 1) / tj);
}

#define SMDD_SWITCH_M2(M_, ...)                                      \
    switch (M_) {                                                    \
        case 128: { constexpr int MM = 128; __VA_ARGS__; } break;    \
        case 256: { constexpr int MM = 256; __VA_ARGS__; } break;    \
        case 512: { constexpr int MM = 512; __VA_ARGS__; } break;    \
        case 1024: { constexpr int MM = 1024; __VA_ARGS__; } break;  \
        case 1536: { constexpr int MM = 1536; __VA_ARGS__; } break;  \
        default: return cudaErrorInvalidValue;                       \
    }

}  // namespace

bool fft2_supported(int M) { return (M >= 128 && M <= 1024) || M == 1536; }

int fft2_traces_per_cta(int M) {
    switch (M) {
        case 128: return Fft2<128>::TR;
        case 256: return Fft2<256>::TR;
        case 512: return Fft2<512>::TR;
        case 1024: return Fft2<1024>::TR;
        case 1536: return Fft3::TR;
    }
    return 0;
}

int fft2_blocks(int M, const TraceGrid &g) {
    switch (M) {
        case 128: return blocks2_for<128>(g);
        case 256: return blocks2_for<256>(g);
        case 512: return blocks2_for<512>(g);
        case 1024: return blocks2_for<1024>(g);
        case 1536: return blocks2_for<1536>(g);
    }
    return 0;
}

int fft2_tw_size(int M) { return M == 1536 ? Fft3::TW_SIZE : M; }

// M <= 1024: the pass-2 table [r][j'] = w_M^{r j'} (r < M/32, j' < 32); M = 1536: the pass-2 table
// [r][k] = w_192^{r k} (r < 4, k < 48) followed by the pass-3 table [r][j] = w_1536^{r j} (r < 8,
// j < 192); double precision rounded once
void fft2_tw_fill(int M, std::vector<float2> &tw) {
    const double pi = 3.14159265358979323846;
    tw.assign(fft2_tw_size(M), make_float2(0.f, 0.f));
    auto put = [&](int i, long long num, long long den) {
        const double ang = 2.0 * pi * (double)num / (double)den;
        tw[i] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    };
    if (M == 1536) {
        for (int r = 0; r < 4; ++r)
            for (int k = 0; k < 48; ++k) put(r * 48 + k, (long long)r * k, 192);
        for (int r = 0; r < 8; ++r)
            for (int j = 0; j < 192; ++j) put(Fft3::TW2 + r * 192 + j, (long long)r * j, 1536);
        return;
    }
    for (int r = 0; r < M / 32; ++r)
        for (int j = 0; j < 32; ++j) put(r * 32 + j, (long long)r * j, M);
}

template <int M>
static cudaError_t prepare2_m() {
    const int sm = (int)RegFft<M>::SMEM;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_rfft<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_irfft_out<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_residual<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_update<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_update<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_rfft_q<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_residual_q<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_update_q<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return e;
}

cudaError_t fft2_prepare(int M) {
    SMDD_SWITCH_M2(M, { return prepare2_m<MM>(); });
    return cudaSuccess;
}

cudaError_t launch2_rfft(int M, const FftArgs &a, cudaStream_t st) {
    SMDD_SWITCH_M2(M, {
        const int nb = blocks2_for<MM>(a.g);
        if (nb < 0) return cudaErrorInvalidValue;
        if (nb == 0) return cudaSuccess;
        k2_rfft<MM><<<nb, RegFft<MM>::THREADS, RegFft<MM>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

cudaError_t launch2_irfft_out(int M, const FftArgs &a, cudaStream_t st) {
    SMDD_SWITCH_M2(M, {
        const int nb = blocks2_for<MM>(a.g);
        if (nb < 0) return cudaErrorInvalidValue;
        if (nb == 0) return cudaSuccess;
        k2_irfft_out<MM><<<nb, RegFft<MM>::THREADS, RegFft<MM>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

cudaError_t launch2_residual(int M, const FftArgs &a, int nblocks_expected, cudaStream_t st) {
    SMDD_SWITCH_M2(M, {
        const int nb = blocks2_for<MM>(a.g);
        if (nb <= 0 || nb > nblocks_expected) return cudaErrorInvalidValue;
        k2_residual<MM><<<nb, RegFft<MM>::THREADS, RegFft<MM>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

cudaError_t launch2_update(int M, bool keep, const FftArgs &a, cudaStream_t st) {
    SMDD_SWITCH_M2(M, {
        const int nb = blocks2_for<MM>(a.g);
        if (nb < 0) return cudaErrorInvalidValue;
        if (nb == 0) return cudaSuccess;
        if (keep) k2_update<MM, true><<<nb, RegFft<MM>::THREADS, RegFft<MM>::SMEM, st>>>(a);
        else k2_update<MM, false><<<nb, RegFft<MM>::THREADS, RegFft<MM>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

template <class KF>
static cudaError_t launch2_queue_kernel(KF kern, int threads, size_t smem, const WorkQueue &q, cudaStream_t st) {
    if (q.total <= 0) return cudaSuccess;
    kern<<<queue_grid(kern, threads, smem, q.total), threads, smem, st>>>(q);
    return cudaGetLastError();
}

cudaError_t launch2_queue_rfft(int M, const WorkQueue &q, cudaStream_t st) {
    SMDD_SWITCH_M2(M, { return launch2_queue_kernel(k2_rfft_q<MM>, RegFft<MM>::THREADS, RegFft<MM>::SMEM, q, st); });
    return cudaSuccess;
}

cudaError_t launch2_queue_residual(int M, const WorkQueue &q, cudaStream_t st) {
    SMDD_SWITCH_M2(M, { return launch2_queue_kernel(k2_residual_q<MM>, RegFft<MM>::THREADS, RegFft<MM>::SMEM, q, st); });
    return cudaSuccess;
}

cudaError_t launch2_queue_update(int M, const WorkQueue &q, cudaStream_t st) {
    SMDD_SWITCH_M2(M, { return launch2_queue_kernel(k2_update_q<MM>, RegFft<MM>::THREADS, RegFft<MM>::SMEM, q, st); });
    return cudaSuccess;
}

}  // namespace smdd
