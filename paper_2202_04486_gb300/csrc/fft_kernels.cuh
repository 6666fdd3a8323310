// Trace-parallel FFT kernels of the MDC hot path: model / residual / kernel spectra (rfft), the
// residual step (inverse FFT, causal window, subtraction of the observed data, FP64 loss, forward FFT),
// the SGD update (inverse FFT of the gradient spectrum, window, X <- X - alpha g, optional forward FFT
// of the new model) and plain inverse transforms for the operator outputs.
//
// Appendix A: MDC = FFT along time -> batched per-frequency products -> inverse FFT.  The causal
// window keeps t in [0, nt) of the length-N result; with N >= 2 nt - 1 this equals the linear
// convolution (forward) and the linear cross-correlation at non-negative lags (adjoint, Eq. 6).
//
// Memory behaviour: a CTA owns TR traces whose spectra are adjacent along the contiguous axis, so a
// frequency row of the tile is one contiguous segment of TR complex values.  Every thread of the tile
// loader is bound to one trace and issues all of its P global loads before any shared-memory store;
// time-domain inputs needed after an inverse FFT (the model for the update, the observed data for the
// residual) are loaded into registers before that FFT starts, so their latency overlaps the passes.
//
// This header holds the device code and the per-length launchers FftLaunch<M>; each complex length M is
// instantiated in a translation unit of its own (fft_m*.cu) so the library compiles in parallel, and
// fft_kernels.cu dispatches on M at run time.
#pragma once

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "smdd_fft.cuh"
#include "smdd_internal.h"
#include "work_queue.cuh"

namespace smdd {

struct TileCoord {
    int i, j;
    bool valid;
};

// tile bid of the grid (blockIdx.x in a plain launch, the dequeued tile in a work-queue launch)
template <int M>
__device__ __forceinline__ TileCoord coord_of(const TraceGrid &g, int tr, int bid) {
    constexpr int TR = Team<M>::TR;
    const int ti = 1 << g.ti_log2;
    const int tj = TR >> g.ti_log2;
    const int ntile_i = (g.ni + ti - 1) / ti;
    const int bi = bid % ntile_i, bj = bid / ntile_i;
    TileCoord c;
    c.i = bi * ti + (tr & (ti - 1));
    c.j = bj * tj + (tr >> g.ti_log2);
    c.valid = c.i < g.ni && c.j < g.nj;
    return c;
}

// Upper enumeration of a square grid (TraceGrid::sym): tile number bid -> the number of the same tile in
// the full enumeration (bi + nbi j).  Rows j = TR g .. TR g + TR - 1 form group g, each row holding the
// tiles bi = g .. nbi - 1, so group g starts at G(g) = TR (g nbi - g (g - 1) / 2).
__host__ __device__ __forceinline__ int sym_tile_to_full(const TraceGrid &g, int TR, int bid) {
    const int nbi = (g.ni + TR - 1) / TR;
    auto G = [&](long long q) { return (long long)TR * (q * nbi - q * (q - 1) / 2); };
    const float h = nbi + 0.5f;
    int q = (int)(h - sqrtf(fmaxf(h * h - 2.f * (float)bid / (float)TR, 0.f)));
    q = q < 0 ? 0 : (q > nbi - 1 ? nbi - 1 : q);
    while (q > 0 && G(q) > bid) --q;
    while (q + 1 < nbi && G(q + 1) <= bid) ++q;
    const int off = (int)(bid - G(q)), w = nbi - q;
    const int j = q * TR + off / w, bi = q + off % w;
    return j * nbi + bi;
}

#ifndef SMDD_FFT_PAIR_IO
#define SMDD_FFT_PAIR_IO 1   // spectrum tiles moved as 16-byte pairs of adjacent traces where the grid allows
#endif

// The CTA's traces come in pairs adjacent along the contiguous spectrum axis (2 or more consecutive i,
// an even TR): a thread then moves the bins of two traces with one 16-byte access.
template <int M>
__device__ __forceinline__ bool pair_io(const TraceGrid &g) {
    return SMDD_FFT_PAIR_IO && Team<M>::TR % 2 == 0 && g.ti_log2 >= 1 && g.ssi == 1 && (g.ssj % 2) == 0 &&
           (g.ssf % 2) == 0;
}

// Spectra of the CTA's traces -> shared memory, paired form: traces 2p, 2p+1 (p = tid % (TR/2)), bins
// f = tid / (TR/2) + it * 2T (it < P/2), plus f = M for tid < TR/2.
template <int M>
__device__ __forceinline__ void tile_load_spec_pair(float2 *sm, const float2 *__restrict__ spec, const TraceGrid &g, int bid) {
    constexpr int TR = Team<M>::TR, STR = Team<M>::STRIDE, P = Team<M>::P, T = Team<M>::T, H = TR / 2;
    const int pr = threadIdx.x % H, f0 = threadIdx.x / H;
    const TileCoord c0 = coord_of<M>(g, 2 * pr, bid), c1 = coord_of<M>(g, 2 * pr + 1, bid);
    float4 v[P / 2];
    float2 nyq = make_float2(0.f, 0.f);
    if (c0.valid) {
        // c0.i is even and the strides are even: 16-byte aligned; the second trace (c1.i = c0.i + 1) may lie
        // past ni, where the pair reads the padding column of the spectra (ldr is even) and drops it
        const float2 *s = spec + (long long)c0.i * g.ssi + (long long)c0.j * g.ssj;
#pragma unroll
        for (int it = 0; it < P / 2; ++it) v[it] = __ldcs(reinterpret_cast<const float4 *>(s + (long long)(f0 + it * 2 * T) * g.ssf));
        if (f0 == 0) {
            const float4 w = __ldcs(reinterpret_cast<const float4 *>(s + (long long)M * g.ssf));
            nyq = make_float2(w.x, w.z);
        }
    } else {
#pragma unroll
        for (int it = 0; it < P / 2; ++it) v[it] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const bool ok1 = c1.valid;
    float2 *b0 = sm + (2 * pr) * STR, *b1 = b0 + STR;
#pragma unroll
    for (int it = 0; it < P / 2; ++it) {
        const int f = f0 + it * 2 * T;
        const float2 x0 = make_float2(v[it].x, v[it].y), x1 = ok1 ? make_float2(v[it].z, v[it].w) : make_float2(0.f, 0.f);
        if (f == 0) {
            b0[0] = make_float2(x0.x, nyq.x);
            b1[0] = make_float2(x1.x, ok1 ? nyq.y : 0.f);
        } else {
            b0[padi(f)] = x0;
            b1[padi(f)] = x1;
        }
    }
}

template <int M>
__device__ __forceinline__ void tile_store_spec_pair(const float2 *sm, float2 *__restrict__ spec, const TraceGrid &g, int bid) {
    constexpr int TR = Team<M>::TR, STR = Team<M>::STRIDE, P = Team<M>::P, T = Team<M>::T, H = TR / 2;
    const int pr = threadIdx.x % H, f0 = threadIdx.x / H;
    const TileCoord c0 = coord_of<M>(g, 2 * pr, bid), c1 = coord_of<M>(g, 2 * pr + 1, bid);
    if (!c0.valid) return;
    const float2 *b0 = sm + (2 * pr) * STR, *b1 = b0 + STR;
    float2 *s = spec + (long long)c0.i * g.ssi + (long long)c0.j * g.ssj;
    if (c1.valid) {
#pragma unroll
        for (int it = 0; it < P / 2; ++it) {
            const int f = f0 + it * 2 * T;
            const float2 x0 = (f == 0) ? make_float2(b0[0].x, 0.f) : b0[padi(f)];
            const float2 x1 = (f == 0) ? make_float2(b1[0].x, 0.f) : b1[padi(f)];
            *reinterpret_cast<float4 *>(s + (long long)f * g.ssf) = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
        if (f0 == 0) *reinterpret_cast<float4 *>(s + (long long)M * g.ssf) = make_float4(b0[0].y, 0.f, b1[0].y, 0.f);
    } else {   // the second trace lies past ni: its slot of the spectra is left untouched
#pragma unroll
        for (int it = 0; it < P / 2; ++it) {
            const int f = f0 + it * 2 * T;
            s[(long long)f * g.ssf] = (f == 0) ? make_float2(b0[0].x, 0.f) : b0[padi(f)];
        }
        if (f0 == 0) s[(long long)M * g.ssf] = make_float2(b0[0].y, 0.f);
    }
}

// Spectra of the CTA's traces -> shared memory.  Slot 0 of each trace holds (Re X[0], Re X[M]).
// Thread binding: trace tr = tid % TR, bins f = tid / TR + it * T (it < P), plus f = M for tid < TR.
template <int M>
__device__ __forceinline__ void tile_load_spec(float2 *sm, const float2 *__restrict__ spec, const TraceGrid &g, int bid) {
    if (pair_io<M>(g)) {
        tile_load_spec_pair<M>(sm, spec, g, bid);
        return;
    }
    constexpr int TR = Team<M>::TR, STR = Team<M>::STRIDE, P = Team<M>::P, T = Team<M>::T;
    const int tr = threadIdx.x % TR, f0 = threadIdx.x / TR;
    const TileCoord c = coord_of<M>(g, tr, bid);
    float2 v[P];
    float nyq = 0.f;
    if (c.valid) {
        const float2 *s = spec + (long long)c.i * g.ssi + (long long)c.j * g.ssj;
#pragma unroll
        for (int it = 0; it < P; ++it) v[it] = __ldcs(s + (long long)(f0 + it * T) * g.ssf);
        if (f0 == 0) nyq = __ldcs(s + (long long)M * g.ssf).x;
    } else {
#pragma unroll
        for (int it = 0; it < P; ++it) v[it] = make_float2(0.f, 0.f);
    }
    float2 *b = sm + tr * STR;
#pragma unroll
    for (int it = 0; it < P; ++it) {
        const int f = f0 + it * T;
        if (f == 0) b[0] = make_float2(v[it].x, nyq);
        else b[padi(f)] = v[it];
    }
}

template <int M>
__device__ __forceinline__ void tile_store_spec(const float2 *sm, float2 *__restrict__ spec, const TraceGrid &g, int bid) {
    if (pair_io<M>(g)) {
        tile_store_spec_pair<M>(sm, spec, g, bid);
        return;
    }
    constexpr int TR = Team<M>::TR, STR = Team<M>::STRIDE, P = Team<M>::P, T = Team<M>::T;
    const int tr = threadIdx.x % TR, f0 = threadIdx.x / TR;
    const TileCoord c = coord_of<M>(g, tr, bid);
    if (!c.valid) return;
    const float2 *b = sm + tr * STR;
    float2 *s = spec + (long long)c.i * g.ssi + (long long)c.j * g.ssj;
#pragma unroll
    for (int it = 0; it < P; ++it) {
        const int f = f0 + it * T;
        const float2 v = (f == 0) ? make_float2(b[0].x, 0.f) : b[padi(f)];
        s[(long long)f * g.ssf] = v;
    }
    if (f0 == 0) s[(long long)M * g.ssf] = make_float2(b[0].y, 0.f);
}

// Time samples for the first-forward-pass positions: register pair (2qq, 2qq+1) x r holds
// z[n], z[n+1] = (x[2n], x[2n+1]), (x[2n+2], x[2n+3]) with n = 2t + 2T qq + r M/R_1.  Only r < R_1/2 can
// hold samples (the upper half is the zero padding since nt <= M).  Slot h = qq * (R_1/2) + r.
constexpr int NPAIR = FFT_P / 4;   // float4 slots per thread

template <int M, int V>
__device__ __forceinline__ void load_pairs(const float *__restrict__ x, int nt, bool valid, bool vec, int t,
                                           float4 (&h)[NPAIR]) {
    constexpr int R = fft_radix(M, 0, V), T = M / FFT_P, QQ = FFT_P / R / 2, S = M / R;
#pragma unroll
    for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
        for (int r = 0; r < R / 2; ++r) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            const int i0 = 2 * (2 * t + 2 * T * qq + r * S);
            if (valid) {
                if (vec && i0 + 3 < nt) {
                    v = __ldcs(reinterpret_cast<const float4 *>(x + i0));
                } else {
                    if (i0 < nt) v.x = x[i0];
                    if (i0 + 1 < nt) v.y = x[i0 + 1];
                    if (i0 + 2 < nt) v.z = x[i0 + 2];
                    if (i0 + 3 < nt) v.w = x[i0 + 3];
                }
            }
            h[qq * (R / 2) + r] = v;
        }
}

// pairs -> first-forward-pass registers (upper half of every butterfly is zero padding)
template <int M, int V>
__device__ __forceinline__ void pairs_to_regs(const float4 (&h)[NPAIR], float2 (&a)[FFT_P]) {
    constexpr int R = fft_radix(M, 0, V), QQ = FFT_P / R / 2;
#pragma unroll
    for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 v = (r < R / 2) ? h[qq * (R / 2) + r] : make_float4(0.f, 0.f, 0.f, 0.f);
            a[(2 * qq) * R + r] = make_float2(v.x, v.y);
            a[(2 * qq + 1) * R + r] = make_float2(v.z, v.w);
        }
}

// read 4 time samples starting at i0 (zero outside [0, nt))
__device__ __forceinline__ float4 load_quad(const float *y, int i0, int nt, bool vec) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vec && i0 + 3 < nt) {
        v = *reinterpret_cast<const float4 *>(y + i0);
    } else {
        if (i0 < nt) v.x = y[i0];
        if (i0 + 1 < nt) v.y = y[i0 + 1];
        if (i0 + 2 < nt) v.z = y[i0 + 2];
        if (i0 + 3 < nt) v.w = y[i0 + 3];
    }
    return v;
}

// write 4 time samples starting at i0 (window [0, nt))
__device__ __forceinline__ void store_quad(float *y, int i0, int nt, bool vec, float4 v) {
    if (vec && i0 + 3 < nt) {
        *reinterpret_cast<float4 *>(y + i0) = v;
    } else {
        if (i0 < nt) y[i0] = v.x;
        if (i0 + 1 < nt) y[i0 + 1] = v.y;
        if (i0 + 2 < nt) y[i0 + 2] = v.z;
        if (i0 + 3 < nt) y[i0 + 3] = v.w;
    }
}

// ------------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------------
template <int M, int V>
__device__ __forceinline__ void rfft_body(const FftArgs &a, int bid) {
    extern __shared__ __align__(16) float2 sm[];
    constexpr int T = Team<M>::T;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    const TileCoord c = coord_of<M>(a.g, tr, bid);
    float2 *buf = sm + tr * Team<M>::STRIDE;
    float4 h[NPAIR];
    float2 v[FFT_P];
    const float *x = a.tin + (c.valid ? (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj : 0);
    load_pairs<M, V>(x, a.nt, c.valid, a.vec, t, h);
    pairs_to_regs<M, V>(h, v);
    rfft_regs_to_smem<M, V>(v, buf, t, a.tw, a.twN);
    __syncthreads();
    tile_store_spec<M>(sm, a.spec, a.g, bid);
}

template <int M, int V>
__global__ void __launch_bounds__(Team<M>::THREADS, Team<M>::MINB) k_rfft(FftArgs a) {
    rfft_body<M, V>(a, blockIdx.x);
}

// spectra -> s * irfft, causal window [0, nt)
template <int M, int V>
__global__ void __launch_bounds__(Team<M>::THREADS, Team<M>::MINB) k_irfft_out(FftArgs a) {
    const int bid = blockIdx.x;
    extern __shared__ __align__(16) float2 sm[];
    constexpr int T = Team<M>::T, R = fft_radix(M, 0, V), QQ = FFT_P / R / 2, S = M / R;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    tile_load_spec<M>(sm, a.spec, a.g, bid);
    __syncthreads();
    const TileCoord c = coord_of<M>(a.g, tr, bid);
    float2 *buf = sm + tr * Team<M>::STRIDE;
    float2 v[FFT_P];
    irfft_smem_to_regs<M, V>(v, buf, t, a.tw, a.twN);
    if (!c.valid) return;   // no barrier follows
    float *y = a.tout + (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj;
#pragma unroll
    for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
        for (int r = 0; r < R / 2; ++r) {
            const float2 z0 = v[(2 * qq) * R + r], z1 = v[(2 * qq + 1) * R + r];
            store_quad(y, 2 * (2 * t + 2 * T * qq + r * S), a.nt, a.vec,
                       make_float4(z0.x * a.s, z0.y * a.s, z1.x * a.s, z1.y * a.s));
        }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
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

// four samples starting at i0: z = s * p - o inside the window [0, nt), zero outside
__device__ __forceinline__ float4 resid_quad(float2 p0, float2 p1, float4 o, float s, int i0, int nt) {
    float4 z;
    z.x = (i0 < nt) ? fmaf(p0.x, s, -o.x) : 0.f;
    z.y = (i0 + 1 < nt) ? fmaf(p0.y, s, -o.y) : 0.f;
    z.z = (i0 + 2 < nt) ? fmaf(p1.x, s, -o.z) : 0.f;
    z.w = (i0 + 3 < nt) ? fmaf(p1.y, s, -o.w) : 0.f;
    return z;
}

// Residual step: R = s * irfft(Uh)[0:nt] - U_obs[row], loss partial 1/2 sum R^2 (FP64), Rh = rfft(R)
// written in place over Uh.  Trace grid: i = batch entry b, j = virtual source v.
// tile bid of nblk tiles; the last tile to finish (atomic ticket) sums the partials of all nblk
template <int M, int V>
__device__ __forceinline__ void residual_body(const FftArgs &a, int bid, int nblk) {
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[32];
    __shared__ bool am_last;
    constexpr int T = Team<M>::T, R = fft_radix(M, 0, V), QQ = FFT_P / R / 2, S = M / R;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    const TileCoord c = coord_of<M>(a.g, tr, bid);

    // observed row for this trace, prefetched before the transforms
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
    tile_load_spec<M>(sm, a.spec, a.g, bid);
    __syncthreads();
    float2 *buf = sm + tr * Team<M>::STRIDE;
    float2 v[FFT_P];
    float4 o[NPAIR];   // observed row, loaded after the first inverse pass (its latency overlaps the rest)
    irfft_smem_to_regs_mid<M, V>(v, buf, t, a.tw, a.twN,
                                 [&] { load_pairs<M, V>(uo ? uo : a.uobs, a.nt, uo != nullptr, a.vec, t, o); });

    double l2 = 0.0;
    float4 z[NPAIR];
#pragma unroll
    for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
        for (int r = 0; r < R / 2; ++r) {
            const int hs = qq * (R / 2) + r;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c.valid) {
                q = resid_quad(v[(2 * qq) * R + r], v[(2 * qq + 1) * R + r], o[hs], a.s,
                               2 * (2 * t + 2 * T * qq + r * S), a.nt);
                l2 += (double)q.x * q.x + (double)q.y * q.y + (double)q.z * q.z + (double)q.w * q.w;
            }
            z[hs] = q;
        }
    pairs_to_regs<M, V>(z, v);
    team_sync<T>();          // every thread of the team has finished reading buf
    rfft_regs_to_smem<M, V>(v, buf, t, a.tw, a.twN);
    __syncthreads();
    tile_store_spec<M>(sm, a.spec, a.g, bid);

    // deterministic loss: per-block partials, summed in block order by the last block to finish
    const double bs = block_sum(l2, red);
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
        s = block_sum(s, red);   // fixed assignment and order: deterministic
        if (threadIdx.x == 0) {
            if (a.loss) *a.loss = 0.5 * s;
            *a.counter = 0u;
        }
    }
}

template <int M, int V>
__global__ void __launch_bounds__(Team<M>::THREADS, Team<M>::MINB) k_residual(FftArgs a) {
    residual_body<M, V>(a, blockIdx.x, gridDim.x);
}

// Update: g = s * irfft(Gh)[0:nt];  X <- X - alpha g (SGD), or with the causality mute and/or Nesterov
// momentum (see the else branch);  optionally Gh <- rfft(X_new) (in place).
// Trace grid: i = receiver r, j = virtual source v (model layout [nv][nr][nt]).
//
// Symmetric model (a.g.sym, reciprocity on a square grid with X[v][r] = X[r][v], and so the velocity or the
// moments of a symmetric start): only the tiles on or above the TR-block diagonal run; a trace (v, r) of a
// tile above it (r >= TR (v / TR + 1)) also writes its mirror (r, v) of each array, which it equals, and the
// spectra below the block diagonal are left to launch_mirror_lower or to the transposed read of the
// forward product.  Traces of the diagonal blocks run in both orders (their mirrors are in the same
// block row and column), so every element of X is written once.
template <int M, int V, bool KEEP, bool EXT>
__device__ __forceinline__ void update_body(const FftArgs &a, int bid_in) {
    extern __shared__ __align__(16) float2 sm[];
    constexpr int T = Team<M>::T, R = fft_radix(M, 0, V), QQ = FFT_P / R / 2, S = M / R;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    const int bid = a.g.sym ? sym_tile_to_full(a.g, Team<M>::TR, bid_in) : bid_in;
    const TileCoord c = coord_of<M>(a.g, tr, bid);
    float *x = a.tout + (c.valid ? (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj : 0);
    // the mirror trace (r, v) of a trace above the block diagonal
    float *xm = (a.g.sym && c.valid && c.i / Team<M>::TR > c.j / Team<M>::TR)
                    ? a.tout + (long long)c.j * a.g.tsi + (long long)c.i * a.g.tsj
                    : nullptr;

    tile_load_spec<M>(sm, a.spec, a.g, bid);
    __syncthreads();
    float2 *buf = sm + tr * Team<M>::STRIDE;
    float2 v[FFT_P];
    float4 xo[NPAIR];   // model samples, loaded after the first inverse pass (latency overlaps the rest)
    irfft_smem_to_regs_mid<M, V>(v, buf, t, a.tw, a.twN, [&] { load_pairs<M, V>(x, a.nt, c.valid, a.vec, t, xo); });
    const float nas = -a.alpha * a.s;
    if constexpr (!EXT) {
        // SGD: X <- X - alpha g
#pragma unroll
        for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
            for (int r = 0; r < R / 2; ++r) {
                const int hs = qq * (R / 2) + r;
                const int i0 = 2 * (2 * t + 2 * T * qq + r * S);
                const float2 g0 = v[(2 * qq) * R + r], g1 = v[(2 * qq + 1) * R + r];
                const float4 xv = xo[hs];
                float4 z;
                z.x = (i0 < a.nt) ? fmaf(nas, g0.x, xv.x) : 0.f;
                z.y = (i0 + 1 < a.nt) ? fmaf(nas, g0.y, xv.y) : 0.f;
                z.z = (i0 + 2 < a.nt) ? fmaf(nas, g1.x, xv.z) : 0.f;
                z.w = (i0 + 3 < a.nt) ? fmaf(nas, g1.y, xv.w) : 0.f;
                if (c.valid) store_quad(x, i0, a.nt, a.vec, z);
                if (xm) store_quad(xm, i0, a.nt, a.vec, z);
                xo[hs] = z;
            }
    } else {
        // causality mute (the step is zero before the first kept sample) and, with a velocity,
        // Nesterov momentum on the look-ahead point: V <- mu V + step, X <- X + mu V + step;
        // or, with Adam moments m and v (Kingma & Ba, Algorithm 1) of the preconditioned gradient g:
        // m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, X <- X - alpha (c1 m) / (sqrt(c2 v) + eps)
        const int first = (a.mute && c.valid) ? __ldg(a.mute + (long long)c.j * a.g.ni + c.i) : 0;
        const long long toff = c.valid ? (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj : 0;
        float *vp = (a.vel && c.valid) ? a.vel + toff : nullptr;
        float *mp = (a.adam_m && c.valid) ? a.adam_m + toff : nullptr;
        float *sp = (a.adam_v && c.valid) ? a.adam_v + toff : nullptr;
#pragma unroll
        for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
            for (int r = 0; r < R / 2; ++r) {
                const int hs = qq * (R / 2) + r;
                const int i0 = 2 * (2 * t + 2 * T * qq + r * S);
                const float2 g0 = v[(2 * qq) * R + r], g1 = v[(2 * qq + 1) * R + r];
                const float4 xv = xo[hs];
                const float gk[4] = {g0.x, g0.y, g1.x, g1.y}, xk[4] = {xv.x, xv.y, xv.z, xv.w};
                float4 vv = vp ? load_quad(vp, i0, a.nt, a.vec) : make_float4(0.f, 0.f, 0.f, 0.f);
                float4 mv = mp ? load_quad(mp, i0, a.nt, a.vec) : make_float4(0.f, 0.f, 0.f, 0.f);
                float4 sv = sp ? load_quad(sp, i0, a.nt, a.vec) : make_float4(0.f, 0.f, 0.f, 0.f);
                float vk[4] = {vv.x, vv.y, vv.z, vv.w}, mk[4] = {mv.x, mv.y, mv.z, mv.w};
                float sk[4] = {sv.x, sv.y, sv.z, sv.w}, zk[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (mp) {
                        const float g = (i0 + k >= first) ? a.s * gk[k] : 0.f;
                        mk[k] = fmaf(a.beta1, mk[k], (1.f - a.beta1) * g);
                        sk[k] = fmaf(a.beta2, sk[k], (1.f - a.beta2) * (g * g));
                        zk[k] = xk[k] - a.alpha * (mk[k] * a.c1) / (sqrtf(sk[k] * a.c2) + a.eps);
                    } else {
                        const float st = (i0 + k >= first) ? nas * gk[k] : 0.f;
                        if (vp) {
                            vk[k] = fmaf(a.mu, vk[k], st);
                            zk[k] = fmaf(a.mu, vk[k], xk[k] + st);
                        } else {
                            zk[k] = xk[k] + st;
                        }
                    }
                    if (i0 + k >= a.nt) zk[k] = 0.f;
                }
                const float4 z = make_float4(zk[0], zk[1], zk[2], zk[3]);
                if (c.valid) store_quad(x, i0, a.nt, a.vec, z);
                if (vp) store_quad(vp, i0, a.nt, a.vec, make_float4(vk[0], vk[1], vk[2], vk[3]));
                if (mp) {
                    store_quad(mp, i0, a.nt, a.vec, make_float4(mk[0], mk[1], mk[2], mk[3]));
                    store_quad(sp, i0, a.nt, a.vec, make_float4(sk[0], sk[1], sk[2], sk[3]));
                }
                if (xm) {   // the mirror trace of a symmetric model, and of its velocity or moments
                    const long long moff = xm - a.tout;
                    store_quad(xm, i0, a.nt, a.vec, z);
                    if (vp) store_quad(a.vel + moff, i0, a.nt, a.vec, make_float4(vk[0], vk[1], vk[2], vk[3]));
                    if (mp) {
                        store_quad(a.adam_m + moff, i0, a.nt, a.vec, make_float4(mk[0], mk[1], mk[2], mk[3]));
                        store_quad(a.adam_v + moff, i0, a.nt, a.vec, make_float4(sk[0], sk[1], sk[2], sk[3]));
                    }
                }
                xo[hs] = z;
            }
    }
    if constexpr (KEEP) {
        pairs_to_regs<M, V>(xo, v);
        team_sync<T>();
        rfft_regs_to_smem<M, V>(v, buf, t, a.tw, a.twN);
        __syncthreads();
        tile_store_spec<M>(sm, a.spec, a.g, bid);
    }
}

template <int M, int V, bool KEEP, bool EXT>
__global__ void __launch_bounds__(Team<M>::THREADS, Team<M>::MINB) k_update(FftArgs a) {
    update_body<M, V, KEEP, EXT>(a, blockIdx.x);
}

// work-queue forms: persistent CTAs taking (problem, tile) items until the queue is empty
template <int M, int V>
__global__ void __launch_bounds__(Team<M>::THREADS, Team<M>::MINB) k_rfft_q(WorkQueue q) {
    const FftArgs *args = static_cast<const FftArgs *>(q.args);
    int m = 0, tile = 0;
    __shared__ FftArgs sa;
    while (queue_next(q, m, tile) >= 0) {
        queue_args(args + m, sa);
        __syncthreads();
        rfft_body<M, V>(sa, tile);
    }
}

template <int M, int V>
__global__ void __launch_bounds__(Team<M>::THREADS, Team<M>::MINB) k_residual_q(WorkQueue q) {
    const FftArgs *args = static_cast<const FftArgs *>(q.args);
    int m = 0, tile = 0;
    __shared__ FftArgs sa;
    while (queue_next(q, m, tile) >= 0) {
        queue_args(args + m, sa);
        __syncthreads();
        residual_body<M, V>(sa, tile, __ldg(q.start + m + 1) - __ldg(q.start + m));
    }
}

template <int M, int V>
__global__ void __launch_bounds__(Team<M>::THREADS, Team<M>::MINB) k_update_q(WorkQueue q) {
    const FftArgs *args = static_cast<const FftArgs *>(q.args);
    int m = 0, tile = 0;
    __shared__ FftArgs sa;
    while (queue_next(q, m, tile) >= 0) {
        queue_args(args + m, sa);
        __syncthreads();
        update_body<M, V, true, false>(sa, tile);
    }
}

// ------------------------------------------------------------------------------------------------
// persistent update with a prefetched next tile (two tile buffers within 227 KB of shared memory:
// M <= 1536): each CTA walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; while it transforms one tile, cp.async copies the next tile's gradient
// spectra into its second buffer, so the CTA keeps HBM reads in flight through its compute phase.
// ------------------------------------------------------------------------------------------------
// two tile buffers of the persistent update fit in a CTA's shared memory (227 KB)
template <int M>
__host__ __device__ constexpr bool pf_fits() {
    return 2 * Team<M>::SMEM <= 232448;
}

template <int M>
__device__ __forceinline__ TileCoord coord_at(const TraceGrid &g, int tile, int tr) {
    constexpr int TR = Team<M>::TR;
    const int ti = 1 << g.ti_log2;
    const int tj = TR >> g.ti_log2;
    const int ntile_i = (g.ni + ti - 1) / ti;
    const int bi = tile % ntile_i, bj = tile / ntile_i;
    TileCoord c;
    c.i = bi * ti + (tr & (ti - 1));
    c.j = bj * tj + (tr >> g.ti_log2);
    c.valid = c.i < g.ni && c.j < g.nj;
    return c;
}

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}

// the spectra of `tile` -> buf by cp.async (bin M into the spare slot padi(M); invalid traces
// zero-filled); one commit group
template <int M>
__device__ __forceinline__ void tile_prefetch_spec(float2 *buf, const float2 *__restrict__ spec, const TraceGrid &g, int tile) {
    constexpr int TR = Team<M>::TR, STR = Team<M>::STRIDE, P = Team<M>::P, T = Team<M>::T;
    const int tr = threadIdx.x % TR, f0 = threadIdx.x / TR;
    const TileCoord c = coord_at<M>(g, tile, tr);
    const float2 *s = spec + (c.valid ? (long long)c.i * g.ssi + (long long)c.j * g.ssj : 0);
    const int nbytes = c.valid ? 8 : 0;
    float2 *b = buf + tr * STR;
#pragma unroll
    for (int it = 0; it < P; ++it) {
        const int f = f0 + it * T;
        cp_async8(b + padi(f), c.valid ? s + (long long)f * g.ssf : spec, nbytes);
    }
    if (f0 == 0) cp_async8(b + padi(M), c.valid ? s + (long long)M * g.ssf : spec, nbytes);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int M, int V, bool KEEP>
__global__ void __launch_bounds__(Team<M>::THREADS, Team<M>::MINB) k_update_pf(FftArgs a, int ntiles) {
    extern __shared__ __align__(16) float2 sm[];
    constexpr int T = Team<M>::T, TR = Team<M>::TR, R = fft_radix(M, 0, V), QQ = FFT_P / R / 2, S = M / R;
    constexpr int BUF = TR * Team<M>::STRIDE;
    const int tr = threadIdx.x / T, t = threadIdx.x % T;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;   // CTA-uniform
    tile_prefetch_spec<M>(sm, a.spec, a.g, tile);
    const float nas = -a.alpha * a.s;
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        float2 *cur = sm + (it & 1) * BUF;
        const TileCoord c = coord_at<M>(a.g, tile, tr);
        float *x = a.tout + (c.valid ? (long long)c.i * a.g.tsi + (long long)c.j * a.g.tsj : 0);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();   // this tile's spectra have landed; every thread is done with the previous tile
        if (threadIdx.x < TR) {   // slot 0 packs (Re X[0], Re X[M])
            float2 *b = cur + threadIdx.x * Team<M>::STRIDE;
            b[0] = make_float2(b[0].x, b[padi(M)].x);
        }
        __syncthreads();
        const int nxt = tile + gridDim.x;
        if (nxt < ntiles) tile_prefetch_spec<M>(sm + ((it + 1) & 1) * BUF, a.spec, a.g, nxt);
        float2 *buf = cur + tr * Team<M>::STRIDE;
        float2 v[FFT_P];
        float4 xo[NPAIR];
        irfft_smem_to_regs_mid<M, V>(v, buf, t, a.tw, a.twN, [&] { load_pairs<M, V>(x, a.nt, c.valid, a.vec, t, xo); });
#pragma unroll
        for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
            for (int r = 0; r < R / 2; ++r) {
                const int hs = qq * (R / 2) + r;
                const int i0 = 2 * (2 * t + 2 * T * qq + r * S);
                const float2 g0 = v[(2 * qq) * R + r], g1 = v[(2 * qq + 1) * R + r];
                const float4 xv = xo[hs];
                float4 z;
                z.x = (i0 < a.nt) ? fmaf(nas, g0.x, xv.x) : 0.f;
                z.y = (i0 + 1 < a.nt) ? fmaf(nas, g0.y, xv.y) : 0.f;
                z.z = (i0 + 2 < a.nt) ? fmaf(nas, g1.x, xv.z) : 0.f;
                z.w = (i0 + 3 < a.nt) ? fmaf(nas, g1.y, xv.w) : 0.f;
                if (c.valid) store_quad(x, i0, a.nt, a.vec, z);
                xo[hs] = z;
            }
        if constexpr (KEEP) {
            pairs_to_regs<M, V>(xo, v);
            team_sync<T>();
            rfft_regs_to_smem<M, V>(v, buf, t, a.tw, a.twN);
            __syncthreads();
            tile_store_spec<M>(cur, a.spec, a.g, tile);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// launchers of one complex length M (instantiated in fft_m*.cu)
// ------------------------------------------------------------------------------------------------
template <int M>
int blocks_for(const TraceGrid &g) {
    // -1: the grid was laid out for CTAs of another trace count (more traces along i than a CTA holds), or
    // an upper enumeration of a grid that is not square with whole CTAs along i
    const int ti = 1 << g.ti_log2, tj = Team<M>::TR >> g.ti_log2;
    if (tj < 1) return -1;
    if (g.sym) return (tj == 1 && g.ni == g.nj) ? (int)sym_tiles(g.ni, Team<M>::TR) : -1;
    return ((g.ni + ti - 1) / ti) * ((g.nj + tj - 1) / tj);
}

template <int M>
struct FftLaunch {
    static cudaError_t prepare();
    static cudaError_t rfft(const FftArgs &a, cudaStream_t st);
    static cudaError_t irfft_out(const FftArgs &a, cudaStream_t st);
    static cudaError_t residual(const FftArgs &a, int nblocks_expected, cudaStream_t st);
    static cudaError_t update(bool keep, const FftArgs &a, cudaStream_t st);
    static cudaError_t queue_rfft(int variant, const WorkQueue &q, cudaStream_t st);
    static cudaError_t queue_residual(int variant, const WorkQueue &q, cudaStream_t st);
    static cudaError_t queue_update(int variant, const WorkQueue &q, cudaStream_t st);
};

#ifdef SMDD_FFT_INSTANTIATE
// call f(std::integral_constant<int, V>) with V the radix-order variant (variant 1 only where it differs)
template <int M, class F>
static void with_variant(int v, F &&f) {
    if constexpr (fft_variant_distinct(M)) {
        if (v == 1) f(std::integral_constant<int, 1>{});
        else f(std::integral_constant<int, 0>{});
    } else {
        f(std::integral_constant<int, 0>{});
    }
}

template <int M>
cudaError_t FftLaunch<M>::prepare() {
    const int sm = (int)Team<M>::SMEM;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 2; ++v)
        with_variant<M>(v, [&](auto vc) {
            constexpr int V = decltype(vc)::value;
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rfft<M, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_irfft_out<M, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residual<M, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_update<M, V, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_update<M, V, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rfft_q<M, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_residual_q<M, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_update_q<M, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        });
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_update<M, 0, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_update<M, 0, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if constexpr (pf_fits<M>()) {
        for (int v = 0; v < 2; ++v)
            with_variant<M>(v, [&](auto vc) {
                constexpr int V = decltype(vc)::value;
                if (e == cudaSuccess) e = cudaFuncSetAttribute(k_update_pf<M, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * sm);
                if (e == cudaSuccess) e = cudaFuncSetAttribute(k_update_pf<M, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * sm);
            });
    }
    return e;
}

template <int M>
cudaError_t FftLaunch<M>::rfft(const FftArgs &a, cudaStream_t st) {
    const int nb = blocks_for<M>(a.g);
    if (nb < 0) return cudaErrorInvalidValue;
    if (nb == 0) return cudaSuccess;
    with_variant<M>(a.variant, [&](auto vc) {
        k_rfft<M, decltype(vc)::value><<<nb, Team<M>::THREADS, Team<M>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

template <int M>
cudaError_t FftLaunch<M>::irfft_out(const FftArgs &a, cudaStream_t st) {
    const int nb = blocks_for<M>(a.g);
    if (nb < 0) return cudaErrorInvalidValue;
    if (nb == 0) return cudaSuccess;
    with_variant<M>(a.variant, [&](auto vc) {
        k_irfft_out<M, decltype(vc)::value><<<nb, Team<M>::THREADS, Team<M>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

template <int M>
cudaError_t FftLaunch<M>::residual(const FftArgs &a, int nblocks_expected, cudaStream_t st) {
    const int nb = blocks_for<M>(a.g);
    if (nb <= 0 || nb > nblocks_expected) return cudaErrorInvalidValue;
    with_variant<M>(a.variant, [&](auto vc) {
        k_residual<M, decltype(vc)::value><<<nb, Team<M>::THREADS, Team<M>::SMEM, st>>>(a);
    });
    return cudaGetLastError();
}

// the persistent prefetching update: as many CTAs as fit on the GPU at once, each walking the tiles;
// returns false (nothing launched) where two tile buffers do not fit
template <int M>
static bool launch_update_pf(bool keep, const FftArgs &a, int ntiles, cudaStream_t st) {
    if constexpr (pf_fits<M>()) {
        with_variant<M>(a.variant, [&](auto vc) {
            constexpr int V = decltype(vc)::value;
            auto kern = keep ? k_update_pf<M, V, true> : k_update_pf<M, V, false>;
            int per_sm = 0, dev = 0, nsm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Team<M>::THREADS, 2 * Team<M>::SMEM);
            const int grid = std::max(1, std::min(ntiles, std::max(1, per_sm) * std::max(1, nsm)));
            kern<<<grid, Team<M>::THREADS, 2 * Team<M>::SMEM, st>>>(a, ntiles);
        });
        return true;
    } else {
        return false;
    }
}

template <int M>
cudaError_t FftLaunch<M>::update(bool keep, const FftArgs &a, cudaStream_t st) {
    const bool ext = a.vel || a.mute || a.adam_m;
    const int nb = blocks_for<M>(a.g);
    if (nb < 0) return cudaErrorInvalidValue;
    if (nb == 0) return cudaSuccess;
    if (a.prefetch && !ext && !a.g.sym && launch_update_pf<M>(keep, a, nb, st)) {
        // persistent, prefetching form launched
    } else if (ext) {
        // momentum / Adam / causality mute: radix order 0 only (the caller passes its twiddle table)
        if (a.variant != 0) return cudaErrorInvalidValue;
        if (keep) k_update<M, 0, true, true><<<nb, Team<M>::THREADS, Team<M>::SMEM, st>>>(a);
        else k_update<M, 0, false, true><<<nb, Team<M>::THREADS, Team<M>::SMEM, st>>>(a);
    } else {
        with_variant<M>(a.variant, [&](auto vc) {
            constexpr int V = decltype(vc)::value;
            if (keep) k_update<M, V, true, false><<<nb, Team<M>::THREADS, Team<M>::SMEM, st>>>(a);
            else k_update<M, V, false, false><<<nb, Team<M>::THREADS, Team<M>::SMEM, st>>>(a);
        });
    }
    return cudaGetLastError();
}

// work-queue launches: resident CTAs on every SM take (problem, tile) items until the queue is empty
template <class KF>
static cudaError_t launch_queue_kernel(KF kern, int threads, size_t smem, const WorkQueue &q, cudaStream_t st) {
    if (q.total <= 0) return cudaSuccess;
    const int grid = queue_grid(kern, threads, smem, q.total);
    kern<<<grid, threads, smem, st>>>(q);
    return cudaGetLastError();
}

template <int M>
cudaError_t FftLaunch<M>::queue_rfft(int variant, const WorkQueue &q, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    with_variant<M>(variant, [&](auto vc) {
        e = launch_queue_kernel(k_rfft_q<M, decltype(vc)::value>, Team<M>::THREADS, Team<M>::SMEM, q, st);
    });
    return e;
}

template <int M>
cudaError_t FftLaunch<M>::queue_residual(int variant, const WorkQueue &q, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    with_variant<M>(variant, [&](auto vc) {
        e = launch_queue_kernel(k_residual_q<M, decltype(vc)::value>, Team<M>::THREADS, Team<M>::SMEM, q, st);
    });
    return e;
}

template <int M>
cudaError_t FftLaunch<M>::queue_update(int variant, const WorkQueue &q, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    with_variant<M>(variant, [&](auto vc) {
        e = launch_queue_kernel(k_update_q<M, decltype(vc)::value>, Team<M>::THREADS, Team<M>::SMEM, q, st);
    });
    return e;
}
#endif  // SMDD_FFT_INSTANTIATE

}  // namespace smdd
