// Trace-parallel FFT kernels of the MDC hot path: model / residual / kernel spectra (rfft), the
// residual step (inverse FFT, causal window, subtraction of the observed data, FP64 loss, forward FFT),
// the SGD update (inverse FFT of the gradient spectrum, window, X <- X - alpha g, optional forward FFT
// of the new model) and plain inverse transforms for the operator outputs.
//
// Appendix A: MDC = FFT along time -> batched per-frequency products -> inverse FFT.  The causal
// window keeps t in [0, nt) of the length-N result; with N >= 2 nt - 1 this equals the linear
// convolution (forward) and the linear cross-correlation at non-negative lags (adjoint, Eq. 6).
#include "smdd_fft.cuh"
#include "smdd_internal.h"

namespace smdd {

// ------------------------------------------------------------------------------------------------
// tile <-> shared memory
// ------------------------------------------------------------------------------------------------
struct TileCoord {
    int i, j;
    bool valid;
};

template <int M>
__device__ __forceinline__ TileCoord coord_of(const TraceGrid &g, int tr) {
    constexpr int TR = Team<M>::TR;
    const int ti = 1 << g.ti_log2;
    const int tj = TR >> g.ti_log2;
    const int ntile_i = (g.ni + ti - 1) / ti;
    const int bi = blockIdx.x % ntile_i, bj = blockIdx.x / ntile_i;
    TileCoord c;
    c.i = bi * ti + (tr & (ti - 1));
    c.j = bj * tj + (tr >> g.ti_log2);
    c.valid = c.i < g.ni && c.j < g.nj;
    return c;
}

// spectra of the CTA's traces -> shared memory (slot 0 of each trace holds (Re X[0], Re X[M]))
template <int M>
__device__ __forceinline__ void tile_load_spec(float2 *sm, const float2 *__restrict__ spec, const TraceGrid &g) {
    constexpr int TR = Team<M>::TR, STR = Team<M>::STRIDE;
    for (int e = threadIdx.x; e < (M + 1) * TR; e += blockDim.x) {
        const int f = e / TR, tr = e % TR;
        const TileCoord c = coord_of<M>(g, tr);
        float2 v = make_float2(0.f, 0.f);
        if (c.valid) v = spec[(long long)f * g.ssf + (long long)c.i * g.ssi + (long long)c.j * g.ssj];
        float2 *b = sm + tr * STR;
        if (f == 0) reinterpret_cast<float *>(b)[0] = v.x;
        else if (f == M) reinterpret_cast<float *>(b)[1] = v.x;
        else b[swz(f)] = v;
    }
}

template <int M>
__device__ __forceinline__ void tile_store_spec(const float2 *sm, float2 *__restrict__ spec, const TraceGrid &g) {
    constexpr int TR = Team<M>::TR, STR = Team<M>::STRIDE;
    for (int e = threadIdx.x; e < (M + 1) * TR; e += blockDim.x) {
        const int f = e / TR, tr = e % TR;
        const TileCoord c = coord_of<M>(g, tr);
        if (!c.valid) continue;
        const float2 *b = sm + tr * STR;
        float2 v;
        if (f == 0) v = make_float2(b[0].x, 0.f);
        else if (f == M) v = make_float2(b[0].y, 0.f);
        else v = b[swz(f)];
        spec[(long long)f * g.ssf + (long long)c.i * g.ssi + (long long)c.j * g.ssj] = v;
    }
}

// time trace -> registers in first-forward-pass order; samples past nt are the zero padding
template <int M>
__device__ __forceinline__ void load_time(const float *__restrict__ x, int nt, bool valid, bool vec, int t,
                                          float2 (&a)[16]) {
    constexpr int R = fft_radix(M, 0), T = M / 16, Q = 16 / R, S = M / R;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 v = make_float2(0.f, 0.f);
            if (r < R / 2 && valid) {   // n < M/2 <= ... ; n >= M/2 holds only padding since nt <= M
                const int i0 = 2 * (t + T * q + r * S);
                if (vec) {
                    if (i0 + 1 < nt) v = *reinterpret_cast<const float2 *>(x + i0);
                    else if (i0 < nt) v.x = x[i0];
                } else {
                    if (i0 < nt) v.x = x[i0];
                    if (i0 + 1 < nt) v.y = x[i0 + 1];
                }
            }
            a[q * R + r] = v;
        }
}

// ------------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(Team<M>::THREADS) k_rfft(FftArgs a) {
    extern __shared__ float2 sm[];
    constexpr int T = Team<M>::T;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    const TileCoord c = coord_of<M>(a.g, tr);
    float2 *buf = sm + tr * Team<M>::STRIDE;
    float2 v[16];
    const float *x = a.tin + (c.valid ? (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj : 0);
    load_time<M>(x, a.nt, c.valid, a.vec, t, v);
    fft_forward_regs_to_smem<M>(v, buf, t, a.twM);
    real_post<M>(buf, t, a.twN);
    __syncthreads();
    tile_store_spec<M>(sm, a.spec, a.g);
}

// spectra -> s * irfft, causal window [0, nt)
template <int M>
__global__ void __launch_bounds__(Team<M>::THREADS) k_irfft_out(FftArgs a) {
    extern __shared__ float2 sm[];
    constexpr int T = Team<M>::T, R = fft_radix(M, 0), Q = 16 / R, S = M / R;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    tile_load_spec<M>(sm, a.spec, a.g);
    __syncthreads();
    const TileCoord c = coord_of<M>(a.g, tr);
    float2 *buf = sm + tr * Team<M>::STRIDE;
    real_pre<M>(buf, t, a.twN);
    float2 v[16];
    fft_inverse_smem_to_regs<M>(v, buf, t, a.twM);
    if (!c.valid) return;   // no barrier follows
    float *y = a.tout + (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < R / 2; ++r) {
            const int i0 = 2 * (t + T * q + r * S);
            const float2 z = v[q * R + r];
            if (a.vec && i0 + 1 < a.nt) {
                *reinterpret_cast<float2 *>(y + i0) = make_float2(z.x * a.s, z.y * a.s);
            } else {
                if (i0 < a.nt) y[i0] = z.x * a.s;
                if (i0 + 1 < a.nt) y[i0 + 1] = z.y * a.s;
            }
        }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) s += red[i];
    return s;   // valid in thread 0
}

// Residual step: R = s * irfft(Uh)[0:nt] - U_obs[row], loss partial 1/2 sum R^2 (FP64), Rh = rfft(R)
// written in place over Uh.  Trace grid: i = batch entry b, j = virtual source v.
template <int M>
__global__ void __launch_bounds__(Team<M>::THREADS) k_residual(FftArgs a) {
    extern __shared__ float2 sm[];
    __shared__ double red[32];
    __shared__ bool am_last;
    constexpr int T = Team<M>::T, R = fft_radix(M, 0), Q = 16 / R, S = M / R;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    tile_load_spec<M>(sm, a.spec, a.g);
    __syncthreads();
    const TileCoord c = coord_of<M>(a.g, tr);
    float2 *buf = sm + tr * Team<M>::STRIDE;
    real_pre<M>(buf, t, a.twN);
    float2 v[16];
    fft_inverse_smem_to_regs<M>(v, buf, t, a.twM);

    // observed row for this trace
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
    double l2 = 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 z = make_float2(0.f, 0.f);
            if (r < R / 2 && c.valid) {
                const int i0 = 2 * (t + T * q + r * S);
                const float2 p = v[q * R + r];
                float2 o = make_float2(0.f, 0.f);
                if (uo) {
                    if (a.vec && i0 + 1 < a.nt) o = *reinterpret_cast<const float2 *>(uo + i0);
                    else {
                        if (i0 < a.nt) o.x = uo[i0];
                        if (i0 + 1 < a.nt) o.y = uo[i0 + 1];
                    }
                }
                if (i0 < a.nt) z.x = fmaf(p.x, a.s, -o.x);
                if (i0 + 1 < a.nt) z.y = fmaf(p.y, a.s, -o.y);
                l2 += (double)z.x * (double)z.x + (double)z.y * (double)z.y;
            }
            v[q * R + r] = z;
        }
    team_sync<T>();          // every thread of the team has finished reading buf
    fft_forward_regs_to_smem<M>(v, buf, t, a.twM);
    real_post<M>(buf, t, a.twN);
    __syncthreads();
    tile_store_spec<M>(sm, a.spec, a.g);

    // deterministic loss: per-block partials, summed in block order by the last block to finish
    const double bs = block_sum(l2, red);
    if (threadIdx.x == 0) {
        const int nblk = gridDim.x;
        a.partials[blockIdx.x] = bs;
        __threadfence();
        const unsigned prev = atomicAdd(a.counter, 1u);
        am_last = (prev == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (am_last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += *((volatile double *)&a.partials[b]);
        if (a.loss) *a.loss = 0.5 * s;
        *a.counter = 0u;
    }
}

// SGD update: g = s * irfft(Gh)[0:nt];  X <- X - alpha g;  optionally Gh <- rfft(X_new) (in place).
// Trace grid: i = receiver r, j = virtual source v (model layout [nv][nr][nt]).
template <int M, bool KEEP>
__global__ void __launch_bounds__(Team<M>::THREADS) k_update(FftArgs a) {
    extern __shared__ float2 sm[];
    constexpr int T = Team<M>::T, R = fft_radix(M, 0), Q = 16 / R, S = M / R;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    tile_load_spec<M>(sm, a.spec, a.g);
    __syncthreads();
    const TileCoord c = coord_of<M>(a.g, tr);
    float2 *buf = sm + tr * Team<M>::STRIDE;
    real_pre<M>(buf, t, a.twN);
    float2 v[16];
    fft_inverse_smem_to_regs<M>(v, buf, t, a.twM);
    float *x = a.tout + (c.valid ? (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj : 0);
    const float as = a.alpha * a.s;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 z = make_float2(0.f, 0.f);
            if (r < R / 2 && c.valid) {
                const int i0 = 2 * (t + T * q + r * S);
                const float2 g = v[q * R + r];
                if (a.vec && i0 + 1 < a.nt) {
                    const float2 xo = *reinterpret_cast<const float2 *>(x + i0);
                    z = make_float2(fmaf(-as, g.x, xo.x), fmaf(-as, g.y, xo.y));
                    *reinterpret_cast<float2 *>(x + i0) = z;
                } else {
                    if (i0 < a.nt) { z.x = fmaf(-as, g.x, x[i0]); x[i0] = z.x; }
                    if (i0 + 1 < a.nt) { z.y = fmaf(-as, g.y, x[i0 + 1]); x[i0 + 1] = z.y; }
                }
            }
            v[q * R + r] = z;
        }
    if constexpr (KEEP) {
        team_sync<T>();
        fft_forward_regs_to_smem<M>(v, buf, t, a.twM);
        real_post<M>(buf, t, a.twN);
        __syncthreads();
        tile_store_spec<M>(sm, a.spec, a.g);
    }
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
#define SMDD_SWITCH_M(M_, ...)              \
    switch (M_) {                            \
        case 32: { constexpr int MM = 32; __VA_ARGS__; } break;     \
        case 64: { constexpr int MM = 64; __VA_ARGS__; } break;     \
        case 128: { constexpr int MM = 128; __VA_ARGS__; } break;   \
        case 256: { constexpr int MM = 256; __VA_ARGS__; } break;   \
        case 512: { constexpr int MM = 512; __VA_ARGS__; } break;   \
        case 1024: { constexpr int MM = 1024; __VA_ARGS__; } break; \
        case 2048: { constexpr int MM = 2048; __VA_ARGS__; } break; \
        case 4096: { constexpr int MM = 4096; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;               \
    }

template <int M>
static int blocks_for(const TraceGrid &g) {
    const int ti = 1 << g.ti_log2, tj = Team<M>::TR >> g.ti_log2;
    return ((g.ni + ti - 1) / ti) * ((g.nj + tj - 1) / tj);
}

int fft_blocks(int M, const TraceGrid &g) {
    switch (M) {
        case 32: return blocks_for<32>(g);
        case 64: return blocks_for<64>(g);
        case 128: return blocks_for<128>(g);
        case 256: return blocks_for<256>(g);
        case 512: return blocks_for<512>(g);
        case 1024: return blocks_for<1024>(g);
        case 2048: return blocks_for<2048>(g);
        case 4096: return blocks_for<4096>(g);
    }
    return 0;
}

cudaError_t fft_prepare(int M) {
    SMDD_SWITCH_M(M, {
        const int sm = (int)Team<MM>::SMEM;
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_rfft<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
        if ((e = cudaFuncSetAttribute(k_irfft_out<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
        if ((e = cudaFuncSetAttribute(k_residual<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
        if ((e = cudaFuncSetAttribute(k_update<MM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
        if ((e = cudaFuncSetAttribute(k_update<MM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    });
    return cudaSuccess;
}

cudaError_t launch_rfft(int M, const FftArgs &a, cudaStream_t st) {
    SMDD_SWITCH_M(M, {
        const int nb = blocks_for<MM>(a.g);
        if (nb == 0) return cudaSuccess;
        k_rfft<MM><<<nb, Team<MM>::THREADS, Team<MM>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

cudaError_t launch_irfft_out(int M, const FftArgs &a, cudaStream_t st) {
    SMDD_SWITCH_M(M, {
        const int nb = blocks_for<MM>(a.g);
        if (nb == 0) return cudaSuccess;
        k_irfft_out<MM><<<nb, Team<MM>::THREADS, Team<MM>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

cudaError_t launch_residual(int M, const FftArgs &a, int nblocks_expected, cudaStream_t st) {
    SMDD_SWITCH_M(M, {
        const int nb = blocks_for<MM>(a.g);
        if (nb == 0 || nb > nblocks_expected) return cudaErrorInvalidValue;
        k_residual<MM><<<nb, Team<MM>::THREADS, Team<MM>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

cudaError_t launch_update(int M, bool keep, const FftArgs &a, cudaStream_t st) {
    SMDD_SWITCH_M(M, {
        const int nb = blocks_for<MM>(a.g);
        if (nb == 0) return cudaSuccess;
        if (keep) k_update<MM, true><<<nb, Team<MM>::THREADS, Team<MM>::SMEM, st>>>(a);
        else k_update<MM, false><<<nb, Team<MM>::THREADS, Team<MM>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

}  // namespace smdd
