// Team FFT building blocks for the MDC hot path (sm_103a).
//
// Appendix A evaluates the multi-dimensional convolution as FFT along time -> one complex matrix
// product per frequency -> inverse FFT.  Here every time trace of length nt is zero padded to
// N = nfft = 2M >= 2nt-1 samples (linear, not circular, convolution on [0, nt)) and transformed as a
// real sequence through a complex FFT of length M on z[n] = x[2n] + i x[2n+1]:
//   X[k] = 1/2 (Z[k] + conj Z[M-k]) - i/2 w_N^k (Z[k] - conj Z[M-k]),   k = 0..M,
// and back through the matching pre-processing and an inverse complex FFT of length M.
//
// A "team" of T = M/P threads owns one trace; each thread holds P complex values in registers.
// The complex FFT is a self-sorting Stockham factorisation M = R_1 R_2 ... R_m (radices 3, 4 or 8,
// fixed at compile time): pass p with radix R and span Ns = R_1...R_{p-1} maps butterfly j (inputs
// j + r M/R) to outputs (j - j%Ns) R + j%Ns + r Ns after the twiddles w_{Ns R}^{r (j%Ns)}.  Lengths
// M = 2^k use radices 4 and 8; M = 1536 (FFT length 3072, the shortest 3-smooth length >= 2 nt - 1 for
// nt in 1025 .. 1536) adds one radix-3 pass in the middle of the plan, which moves its values through
// shared memory on its own (512 butterflies over 64 of the 96 threads of a team).  Between
// passes the values go through shared memory; the float2 index is XOR-swizzled within 16-element
// groups so that both the contiguous reads and the strided writes of a half-warp hit distinct banks.
// The first forward pass reads its inputs straight from registers (global loads or the output of a
// previous inverse FFT), and the last inverse pass leaves its outputs in registers in exactly that
// order, so an inverse FFT, an element-wise epilogue and a forward FFT chain without a shared-memory
// round trip.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace smdd {

// ------------------------------------------------------------------------------------------------
// complex helpers (float2 = re, im)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 4) & 15); }

// ------------------------------------------------------------------------------------------------
// small DFTs in registers (unnormalised; INV uses the conjugate roots)
// ------------------------------------------------------------------------------------------------
template <bool INV>
__device__ __forceinline__ void dft2(float2 &a0, float2 &a1) {
    float2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    float2 t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// multiply by w_8^K (forward root exp(-2 pi i K / 8); conjugate for INV), K = 1, 2, 3
template <bool INV, int K>
__device__ __forceinline__ float2 rot8(float2 a) {
    constexpr float h = 0.70710678118654752440f;
    if (K == 1) return INV ? make_float2((a.x - a.y) * h, (a.x + a.y) * h) : make_float2((a.x + a.y) * h, (a.y - a.x) * h);
    if (K == 2) return mul_mi<INV>(a);
    return INV ? make_float2(-(a.x + a.y) * h, (a.x - a.y) * h) : make_float2((a.y - a.x) * h, -(a.x + a.y) * h);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2 *a) {
    // even / odd halves: y_k = E_k + w8^k O_k, y_{k+4} = E_k - w8^k O_k
    dft4<INV>(a[0], a[2], a[4], a[6]);
    dft4<INV>(a[1], a[3], a[5], a[7]);
    float2 o1 = rot8<INV, 1>(a[3]), o2 = rot8<INV, 2>(a[5]), o3 = rot8<INV, 3>(a[7]);
    float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    a[0] = cadd(e0, a[1]);
    a[4] = csub(e0, a[1]);
    a[1] = cadd(e1, o1);
    a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2);
    a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3);
    a[7] = csub(e3, o3);
}

// radix-3 DFT: y0 = a0 + a1 + a2, y1/2 = a0 - (a1 + a2)/2 -/+ i (sqrt(3)/2) (a1 - a2) (forward roots
// w_3 = exp(-2 pi i / 3); the signs of the imaginary term swap for INV)
template <bool INV>
__device__ __forceinline__ void dft3(float2 &a0, float2 &a1, float2 &a2) {
    constexpr float h = 0.86602540378443864676f;   // sqrt(3) / 2
    const float2 s = cadd(a1, a2), d = csub(a1, a2);
    const float2 m = make_float2(fmaf(-0.5f, s.x, a0.x), fmaf(-0.5f, s.y, a0.y));
    const float2 q = mul_mi<INV>(make_float2(h * d.x, h * d.y));   // -i h d (forward), +i h d (inverse)
    a0 = cadd(a0, s);
    a1 = cadd(m, q);
    a2 = csub(m, q);
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2 *a) {
    if constexpr (R == 2) dft2<INV>(a[0], a[1]);
    else if constexpr (R == 4) dft4<INV>(a[0], a[1], a[2], a[3]);
    else dft8<INV>(a);
}


// ------------------------------------------------------------------------------------------------
// FFT plans: forward radix of pass p for complex length M (the inverse uses the radices in reverse
// order).  Radices 4 and 8 take a thread's 16 values as two or more butterflies; a radix-3 pass runs
// through pass3_smem instead.
// ------------------------------------------------------------------------------------------------
constexpr int FFT_P = 16;   // complex values per thread

__host__ __device__ constexpr int fft_npass(int M) { return M <= 64 ? 2 : M <= 512 ? 3 : 4; }
__host__ __device__ constexpr bool is_pow2c(int x) { return x > 0 && (x & (x - 1)) == 0; }
// variant 0: the default radix order; variant 1: the same radices in reverse order (identical to
// variant 0 where every radix is 8).  Both are valid Stockham plans; which one is faster for a given
// shape is left to measurement (the plan autotuner).
__host__ __device__ constexpr int fft_radix0(int M, int p) {
    return M == 32 ? (p == 0 ? 8 : 4)
         : M == 64 ? 8
         : M == 128 ? (p == 0 ? 8 : 4)
         : M == 256 ? (p == 2 ? 4 : 8)
         : M == 512 ? 8
         : M == 1024 ? (p < 2 ? 8 : 4)
         : M == 2048 ? (p == 3 ? 4 : 8)
         : M == 1536 ? (p == 2 ? 3 : 8)    // 8 * 8 * 3 * 8: the radix-3 pass is never the first or last
         : 8;  // 4096
}
__host__ __device__ constexpr int fft_radix(int M, int p, int v = 0) {
    return v == 0 ? fft_radix0(M, p) : fft_radix0(M, fft_npass(M) - 1 - p);
}
__host__ __device__ constexpr bool fft_variant_distinct(int M) {
    for (int p = 0; p < fft_npass(M); ++p)
        if (fft_radix(M, p, 0) != fft_radix(M, p, 1)) return true;
    return false;
}
__host__ __device__ constexpr int fft_span(int M, int p, int v = 0) {
    return p == 0 ? 1 : fft_span(M, p - 1, v) * fft_radix(M, p - 1, v);
}
__host__ __device__ constexpr int ifft_radix(int M, int p, int v = 0) { return fft_radix(M, fft_npass(M) - 1 - p, v); }
__host__ __device__ constexpr int ifft_span(int M, int p, int v = 0) {
    return p == 0 ? 1 : ifft_span(M, p - 1, v) * ifft_radix(M, p - 1, v);
}
__host__ __device__ constexpr int dir_radix(int M, bool inv, int p, int v = 0) { return inv ? ifft_radix(M, p, v) : fft_radix(M, p, v); }
__host__ __device__ constexpr int dir_span(int M, bool inv, int p, int v = 0) { return inv ? ifft_span(M, p, v) : fft_span(M, p, v); }

// Twiddle tables, one per pass p >= 1 of each direction: entry [r][k] (r < R, k < Ns) holds
// w_{Ns R}^{r k} (forward roots; the inverse multiplies by their conjugates).  k is the fast index, so
// the adjacent butterflies of a thread and of neighbouring lanes read adjacent entries.  Offsets in float2.
__host__ __device__ constexpr int tw_off(int M, bool inv, int p, int v = 0) {
    int off = 0;
    if (inv)
        for (int q = 1; q < fft_npass(M); ++q) off += fft_span(M, q, v) * fft_radix(M, q, v);
    for (int q = 1; q < p; ++q) off += dir_span(M, inv, q, v) * dir_radix(M, inv, q, v);
    return off;
}
__host__ __device__ constexpr int tw_size(int M, int v = 0) { return tw_off(M, true, fft_npass(M), v); }

// Shared-memory layout of one trace: element i at float2 index i + 2 (i / 16).  The padding keeps
// every pair (2m, 2m+1) 16-byte aligned and makes the 128-bit accesses of the passes bank-conflict
// free; for the index patterns below the padded address splits into a per-thread base plus a
// compile-time offset.
__host__ __device__ constexpr int padi(int i) { return i + 2 * (i >> 4); }

// Launch geometry of the trace kernels for complex length M: a team of T = M/16 threads per trace,
// TR traces per CTA.  The defaults can be overridden at compile time for tuning sweeps.
#ifndef SMDD_FFT_TRACES
#define SMDD_FFT_TRACES 8
#endif
#ifndef SMDD_FFT_MINB
#define SMDD_FFT_MINB 3
#endif
#ifndef SMDD_FFT_MINB_LARGE          // the same for M >= 1024 (teams of 64 threads or more)
#define SMDD_FFT_MINB_LARGE SMDD_FFT_MINB
#endif
#ifndef SMDD_FFT_MIN_TR              // fewest traces per CTA for M <= 1024
#define SMDD_FFT_MIN_TR 2
#endif
#ifndef SMDD_FFT_TR_2048             // traces per CTA at M = 2048 (teams of 128 threads)
#define SMDD_FFT_TR_2048 8
#endif
#ifndef SMDD_FFT_TR_1536             // traces per CTA at M = 1536 (teams of 96 threads; 8 measured 1.2x
#define SMDD_FFT_TR_1536 8           // faster than 4 on the update at nt 1500, 1200 x 200)
#endif
#ifndef SMDD_FFT_NAMED_BAR           // 1: teams of more than one warp sync on their own named barrier
#define SMDD_FFT_NAMED_BAR 1
#endif

template <int M>
struct Team {
    static constexpr int P = FFT_P;
    static constexpr int T = M / P;                           // threads per trace
    static constexpr int TR_RAW = SMDD_FFT_TRACES * 512 / M;  // SMDD_FFT_TRACES traces per CTA at M = 512
    // traces per CTA: a CTA moves TR consecutive traces x 8 bytes of each frequency row of the
    // spectra, so small TR wastes sectors; at M = 2048 the CTA takes as many traces as 1024 threads
    // hold (8: 64-byte rows; measured 1.5x faster than 2 traces despite 64 registers per thread), else
    // at least SMDD_FFT_MIN_TR; at most 1024 threads
    static constexpr int TR_MIN = M == 2048 ? SMDD_FFT_TR_2048 : M == 1536 ? SMDD_FFT_TR_1536 : SMDD_FFT_MIN_TR;
    static constexpr int TR_LO = TR_RAW < TR_MIN ? TR_MIN : TR_RAW;
    static constexpr int TR = T * TR_LO > 1024 ? 1024 / T : TR_LO;
    static constexpr int THREADS = T * TR;                    // CTA size
    // float2 per trace buffer: padi(M) is a multiple of 16; the extra 16/TR float2 make the TR traces x
    // 16/TR bins that a half-warp touches in the tile loads / stores fall on 16 distinct bank pairs
    static constexpr int STRIDE = padi(M) + (TR >= 8 ? 2 : 16 / TR);
    static constexpr size_t SMEM = (size_t)TR * STRIDE * sizeof(float2);
    static_assert(T <= 32 || TR <= 15, "at most 15 named team barriers");
    // resident CTAs per SM asked of the compiler: never below ~80 registers per thread
    static constexpr int MINB_ASK = M >= 1024 ? SMDD_FFT_MINB_LARGE : SMDD_FFT_MINB;
    static constexpr int MINB = (768 / THREADS) < 1 ? 1 : ((768 / THREADS) < MINB_ASK ? 768 / THREADS : MINB_ASK);
};

// Synchronise the T threads of one trace's team (team k = threads [kT, (k+1)T) of the CTA).  Every
// thread of a team reaches the same sequence of team syncs.
template <int T>
__device__ __forceinline__ void team_sync() {
    if constexpr (T <= 32) {
        __syncwarp();
    } else if constexpr (SMDD_FFT_NAMED_BAR) {
        static_assert(T % 32 == 0, "named barriers count whole warps");
        // barrier 0 is __syncthreads; teams use 1..TR (TR <= 15 for every team size here)
        asm volatile("bar.sync %0, %1;\n" ::"r"(1 + (int)(threadIdx.x / T)), "n"(T) : "memory");
    } else {
        __syncthreads();
    }
}

__device__ __forceinline__ float4 lds4(const float2 *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sts4(float2 *p, float2 lo, float2 hi) {
    *reinterpret_cast<float4 *>(p) = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Register convention for a pass of radix R: thread t owns the butterflies j = 2t + e + 2T qq
// (e in {0,1}, qq < 8/R); a[(2 qq + e) R + r] holds element j + r M/R of the pass input.

template <int M, int R>
__device__ __forceinline__ void pass_load(const float2 *buf, int t, float2 (&a)[FFT_P]) {
    constexpr int T = M / FFT_P, QQ = FFT_P / R / 2, S = M / R;
    const float2 *b = buf + padi(2 * t);
#pragma unroll
    for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 v = lds4(b + padi(2 * T * qq + r * S));
            a[(2 * qq) * R + r] = make_float2(v.x, v.y);
            a[(2 * qq + 1) * R + r] = make_float2(v.z, v.w);
        }
}

// Twiddle powers w^r, r < R, from the loaded w^1 (and w^4 when R = 8): at most three dependent
// complex products per power (a few ulp), instead of one table load per power.
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 w1, float2 w4, float2 (&w)[R]) {
    w[0] = make_float2(1.f, 0.f);
    w[1] = w1;
    if constexpr (R >= 4) {
        w[2] = cmul(w1, w1);
        w[3] = cmul(w[2], w1);
    }
    if constexpr (R == 8) {
        w[4] = w4;
        w[5] = cmul(w4, w1);
        w[6] = cmul(w4, w[2]);
        w[7] = cmul(w4, w[3]);
    }
}

template <int M, int R, int NS, bool INV, int TWOFF>
__device__ __forceinline__ void pass_compute(float2 (&a)[FFT_P], int t, const float2 *__restrict__ tw) {
    constexpr int T = M / FFT_P, QQ = FFT_P / R / 2;
#pragma unroll
    for (int qq = 0; qq < QQ; ++qq) {
        if constexpr (NS > 1) {
            // butterflies j and j+1 use twiddle columns k0 and k0+1, adjacent in each row of the table
            // (NS is even, so j and j+1 share the block of NS)
            const int k0 = is_pow2c(NS) ? ((2 * t + 2 * T * qq) & (NS - 1)) : ((2 * t + 2 * T * qq) % NS);
            const float4 v1 = __ldg(reinterpret_cast<const float4 *>(tw + TWOFF + 1 * NS + k0));
            float4 v4 = v1;
            if constexpr (R == 8) v4 = __ldg(reinterpret_cast<const float4 *>(tw + TWOFF + 4 * NS + k0));
            // one butterfly's powers at a time: half the twiddle registers live at once
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                float2 w[R];
                twiddle_powers<R>(e ? make_float2(v1.z, v1.w) : make_float2(v1.x, v1.y),
                                  e ? make_float2(v4.z, v4.w) : make_float2(v4.x, v4.y), w);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 &x = a[(2 * qq + e) * R + r];
                    x = INV ? cmulc(x, w[r]) : cmul(x, w[r]);
                }
            }
        }
        dftR<R, INV>(&a[(2 * qq) * R]);
        dftR<R, INV>(&a[(2 * qq + 1) * R]);
    }
}

template <int M, int R, int NS>
__device__ __forceinline__ void pass_store(float2 *buf, int t, const float2 (&a)[FFT_P]) {
    constexpr int T = M / FFT_P, QQ = FFT_P / R / 2;
    if constexpr (!is_pow2c(NS)) {
        static_assert((2 * T) % NS == 0, "the butterflies j0 + 2T qq share the residue of j0");
        // spans with a factor 3: the padded index of every store is formed in full (the per-thread base
        // plus immediate split needs power-of-two blocks); pairs stay 16-byte aligned (j even, NS even)
        const int j0 = 2 * t, k = j0 % NS;
#pragma unroll
        for (int qq = 0; qq < QQ; ++qq) {
            const int o = (j0 + 2 * T * qq - k) * R + k;   // j0 + 2T qq has the same residue k (2T % NS == 0)
#pragma unroll
            for (int r = 0; r < R; ++r) sts4(buf + padi(o + r * NS), a[(2 * qq) * R + r], a[(2 * qq + 1) * R + r]);
        }
    } else if constexpr (NS == 1) {
        float2 *b = buf + padi(2 * t * R);
#pragma unroll
        for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
            for (int e = 0; e < 2; ++e)
#pragma unroll
                for (int r = 0; r < R; r += 2)
                    sts4(b + padi(e * R + 2 * T * R * qq + r), a[(2 * qq + e) * R + r], a[(2 * qq + e) * R + r + 1]);
    } else if constexpr (NS <= 2 * T) {
        float2 *b = buf + padi((2 * t - ((2 * t) & (NS - 1))) * R + ((2 * t) & (NS - 1)));
#pragma unroll
        for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
            for (int r = 0; r < R; ++r)
                sts4(b + padi(2 * T * R * qq + r * NS), a[(2 * qq) * R + r], a[(2 * qq + 1) * R + r]);
    } else {
        float2 *b = buf + padi(2 * t);
#pragma unroll
        for (int qq = 0; qq < QQ; ++qq)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int c = (2 * T * qq - ((2 * T * qq) % NS)) * R + ((2 * T * qq) % NS) + r * NS;
                sts4(b + padi(c), a[(2 * qq) * R + r], a[(2 * qq + 1) * R + r]);
            }
    }
}

// A radix-3 pass of span NS, shared memory to shared memory (never the first or last pass of a plan, so
// no register hand-over): butterfly j reads j + r M/3, applies w_{3 NS}^{r (j % NS)} (table rows 1 and 2),
// transforms and stores at (j - j % NS) 3 + j % NS + r NS.  Team syncs between the loads and the stores
// and at the end.
//
// The M/3 butterflies go to the TA = pass3_threads(M) first threads of the team, j = t + TA q (q < M/(3 TA)),
// TA a multiple of 16 that divides M/3 and NS | TA: every thread then has the same count, j % NS = t % NS
// for all its butterflies (one pair of twiddles per pass), and its shared-memory offsets are per-thread
// bases plus compile-time constants.  (At M = 1536: 64 of the 96 threads, 8 butterflies each.)
__host__ __device__ constexpr int pass3_threads(int M, int NS) {
    int best = 0;
    for (int ta = 16; ta <= M / FFT_P; ta += 16)
        if ((M / 3) % ta == 0 && ta % NS == 0) best = ta;
    return best;
}

template <int M, bool INV, int NS, int TWOFF>
__device__ __forceinline__ void pass3_smem(float2 *buf, int t, const float2 *__restrict__ tw) {
    constexpr int T = M / FFT_P, NBF = M / 3;
    constexpr int TA = pass3_threads(M, NS);
    if constexpr (TA > 0 && NS % 16 == 0) {
        // spans that are multiples of 16: every offset below splits as padi(base) + padi(constant)
        constexpr int NQ = NBF / TA;
        if (t < TA) {
            const int k = t % NS;
            float2 w1 = make_float2(1.f, 0.f), w2 = w1;
            if constexpr (NS > 1) {
                w1 = __ldg(tw + TWOFF + NS + k);
                w2 = __ldg(tw + TWOFF + 2 * NS + k);
            }
            const float2 *src = buf + padi(t);
            float2 x[NQ][3];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int r = 0; r < 3; ++r) x[q][r] = src[padi(TA * q + r * NBF)];
            team_sync<T>();
            float2 *dst = buf + padi((t - k) * 3 + k);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if constexpr (NS > 1) {
                    x[q][1] = INV ? cmulc(x[q][1], w1) : cmul(x[q][1], w1);
                    x[q][2] = INV ? cmulc(x[q][2], w2) : cmul(x[q][2], w2);
                }
                dft3<INV>(x[q][0], x[q][1], x[q][2]);
#pragma unroll
                for (int r = 0; r < 3; ++r) dst[padi(3 * TA * q + r * NS)] = x[q][r];
            }
        } else {
            team_sync<T>();
        }
        team_sync<T>();
    } else if constexpr (TA > 0) {
        // spans below 16 (NS | 16): the store offset (j - k) 3 + k + r NS has three per-thread bases
        constexpr int NQ = NBF / TA;
        if (t < TA) {
            const int k = t % NS;
            float2 w1 = make_float2(1.f, 0.f), w2 = w1;
            if constexpr (NS > 1) {
                w1 = __ldg(tw + TWOFF + NS + k);
                w2 = __ldg(tw + TWOFF + 2 * NS + k);
            }
            const float2 *src = buf + padi(t);
            float2 x[NQ][3];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int r = 0; r < 3; ++r) x[q][r] = src[padi(TA * q + r * NBF)];
            team_sync<T>();
            const int o = (t - k) * 3 + k;   // 3 TA q is a multiple of 16: padi(o + r NS + 3 TA q) = padi(o + r NS) + padi(3 TA q)
            float2 *d0 = buf + padi(o), *d1 = buf + padi(o + NS), *d2 = buf + padi(o + 2 * NS);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if constexpr (NS > 1) {
                    x[q][1] = INV ? cmulc(x[q][1], w1) : cmul(x[q][1], w1);
                    x[q][2] = INV ? cmulc(x[q][2], w2) : cmul(x[q][2], w2);
                }
                dft3<INV>(x[q][0], x[q][1], x[q][2]);
                d0[padi(3 * TA * q)] = x[q][0];
                d1[padi(3 * TA * q)] = x[q][1];
                d2[padi(3 * TA * q)] = x[q][2];
            }
        } else {
            team_sync<T>();
        }
        team_sync<T>();
    } else {
        // general case: butterfly j = t + T q, the last round partial
        constexpr int NQ = (NBF + T - 1) / T;
        float2 x[NQ][3];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int j = t + T * q;
            if (j < NBF) {
#pragma unroll
                for (int r = 0; r < 3; ++r) x[q][r] = buf[padi(j + r * NBF)];
            }
        }
        team_sync<T>();
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int j = t + T * q;
            if (j < NBF) {
                const int k = j % NS;
                if constexpr (NS > 1) {
                    const float2 w1 = __ldg(tw + TWOFF + NS + k), w2 = __ldg(tw + TWOFF + 2 * NS + k);
                    x[q][1] = INV ? cmulc(x[q][1], w1) : cmul(x[q][1], w1);
                    x[q][2] = INV ? cmulc(x[q][2], w2) : cmul(x[q][2], w2);
                }
                dft3<INV>(x[q][0], x[q][1], x[q][2]);
                const int o = (j - k) * 3 + k;
#pragma unroll
                for (int r = 0; r < 3; ++r) buf[padi(o + r * NS)] = x[q][r];
            }
        }
        team_sync<T>();
    }
}

template <int M, bool INV, int p, int PEND, int V>
__device__ __forceinline__ void passes_from(float2 (&a)[FFT_P], float2 *buf, int t, const float2 *__restrict__ tw) {
    // passes p .. PEND-1 of a direction: load, compute, and (except for the last inverse pass) store
    if constexpr (p < PEND) {
        constexpr int R = dir_radix(M, INV, p, V), NS = dir_span(M, INV, p, V);
        if constexpr (R == 3) {
            static_assert(p > 0 && p + 1 < fft_npass(M), "the radix-3 pass sits inside the plan");
            pass3_smem<M, INV, NS, tw_off(M, INV, p, V)>(buf, t, tw);
        } else {
            pass_load<M, R>(buf, t, a);
            if constexpr (!INV) team_sync<M / FFT_P>();
            pass_compute<M, R, NS, INV, tw_off(M, INV, p, V)>(a, t, tw);
            if constexpr (!INV || p + 1 < fft_npass(M)) {
                if constexpr (INV) team_sync<M / FFT_P>();
                pass_store<M, R, NS>(buf, t, a);
                team_sync<M / FFT_P>();
            }
        }
        passes_from<M, INV, p + 1, PEND, V>(a, buf, t, tw);
    }
}

// w_32^m = exp(-2 pi i m / 32), m in [0, 32): the roots used by the real-spectrum passes
__device__ __forceinline__ float2 root32(int m) {
    constexpr float c[9] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                            0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                            0.19509032201612826785f, 0.0f};   // cos(pi m / 16), m = 0..8
    m &= 31;
    const int q = m >> 3, rr = m & 7;
    float x = c[rr], y = c[8 - rr];        // cos, sin of the angle inside the quadrant
    float cs, sn;
    switch (q) {
        case 0: cs = x; sn = y; break;
        case 1: cs = -y; sn = x; break;
        case 2: cs = -x; sn = -y; break;
        default: cs = y; sn = -x; break;
    }
    return make_float2(cs, -sn);
}

// The butterflies of the last forward pass and of the first inverse pass (radix R, span M/R): thread t
// owns the pairs u = t + T q (q < 8/R) and, for each, the butterflies ja = u and jb = M/R - u
// (jb = M/(2R) for u = 0).  The bins k = ja + r M/R and M - k = jb + (R-1-r) M/R then lie in the same
// thread, so the real-signal post- and pre-processing run in registers.
template <int M, int V>
struct EdgePass {
    static constexpr int R = fft_radix(M, fft_npass(M) - 1, V);
    static constexpr int S = M / R;     // span of the last forward pass = stride of its inputs
    static constexpr int NP = 8 / R;    // pairs per thread
};

// Last forward pass + real post-processing.  Input: buf after the other forward passes.  Output: buf
// holds X[1..M-1] in their slots and (X[0], X[M]) in slot 0.  Ends with a team sync.
template <int M, int V>
__device__ __forceinline__ void fwd_last_real(float2 (&a)[FFT_P], float2 *buf, int t, const float2 *__restrict__ tw,
                                              const float2 *__restrict__ twN) {
    constexpr int T = M / FFT_P, R = EdgePass<M, V>::R, S = EdgePass<M, V>::S, NP = EdgePass<M, V>::NP;
    constexpr int TWOFF = tw_off(M, false, fft_npass(M) - 1, V);
    int ja[NP], jb[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int u = t + T * q;
        ja[q] = u;
        jb[q] = u ? S - u : S / 2;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            a[(2 * q) * R + r] = buf[padi(ja[q] + r * S)];
            a[(2 * q + 1) * R + r] = buf[padi(jb[q] + r * S)];
        }
    }
    team_sync<T>();
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int u = ja[q];
        float2 *A = &a[(2 * q) * R], *B = &a[(2 * q + 1) * R];
        // twiddles w_M^{r j}: ja from the table, jb = S - u from w_M^{r S} conj(w_M^{r u}) = w_R^r conj(.)
        const float2 t1 = __ldg(tw + TWOFF + 1 * S + u);
        const float2 t4 = (R == 8) ? __ldg(tw + TWOFF + 4 * S + u) : t1;
        float2 wa[R];
        twiddle_powers<R>(t1, t4, wa);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            A[r] = cmul(A[r], wa[r]);
            const float2 wb = u ? cmul(root32(32 * r / R), cconj(wa[r])) : root32(16 * r / R);
            B[r] = cmul(B[r], wb);
        }
        dftR<R, false>(A);
        dftR<R, false>(B);
        // X[k] = e - i w_N^k d, e = (Z[k] + conj Z[M-k]) / 2, d = (Z[k] - conj Z[M-k]) / 2; each bin goes to
        // its slot as soon as it is formed (every load of this pass precedes the team sync above), so A
        // and B are read-only here and no output array is held in registers
        const float2 wn = __ldg(twN + u);   // w_N^u
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 za = A[r], zma = u ? B[R - 1 - r] : A[(R - r) % R];
            const float2 zb = B[r], zmb = u ? A[R - 1 - r] : B[R - 1 - r];
            const float2 wka = cmul(wn, root32(16 * r / R));                                   // w_N^{u + r S}
            const float2 wkb = u ? cmul(root32(16 * (r + 1) / R), cconj(wn)) : root32(8 / R + 16 * r / R);
            const float2 pa = cmul(wka, cscale(csub(za, cconj(zma)), 0.5f));
            const float2 pb = cmul(wkb, cscale(csub(zb, cconj(zmb)), 0.5f));
            float2 xa = cadd(cscale(cadd(za, cconj(zma)), 0.5f), mul_mi<false>(pa));
            const float2 xb = cadd(cscale(cadd(zb, cconj(zmb)), 0.5f), mul_mi<false>(pb));
            if (r == 0 && u == 0) xa = make_float2(xa.x, A[0].x - A[0].y);   // slot 0: X[0], X[M] = Re Z[0] - Im Z[0]
            buf[padi(ja[q] + r * S)] = xa;
            buf[padi(jb[q] + r * S)] = xb;
        }
    }
    team_sync<T>();
}

// First inverse pass with the real pre-processing: buf holds a real-signal spectrum (slot 0 = (X[0],
// X[M])).  Forms Z[k] = E + i O, E = X[k] + conj X[M-k], O = (X[k] - conj X[M-k]) w_N^{-k}, applies the
// radix-R inverse butterflies and stores the pass output.  Ends with a team sync.
template <int M, int V>
__device__ __forceinline__ void inv_first_real(float2 (&a)[FFT_P], float2 *buf, int t, const float2 *__restrict__ twN) {
    constexpr int T = M / FFT_P, R = EdgePass<M, V>::R, S = EdgePass<M, V>::S, NP = EdgePass<M, V>::NP;
    int ja[NP], jb[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int u = t + T * q;
        ja[q] = u;
        jb[q] = u ? S - u : S / 2;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            a[(2 * q) * R + r] = buf[padi(ja[q] + r * S)];
            a[(2 * q + 1) * R + r] = buf[padi(jb[q] + r * S)];
        }
    }
    team_sync<T>();
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int u = ja[q];
        float2 *A = &a[(2 * q) * R], *B = &a[(2 * q + 1) * R];
        const float2 s0 = A[0];
        const float2 xm0 = make_float2(s0.y, 0.f);   // X[M] when u == 0
        if (u == 0) A[0] = make_float2(s0.x, 0.f);
        const float2 wn = __ldg(twN + u);
        float2 za[R], zb[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 xa = A[r], xma = u ? B[R - 1 - r] : (r == 0 ? xm0 : A[(R - r) % R]);
            const float2 xb = B[r], xmb = u ? A[R - 1 - r] : B[R - 1 - r];
            const float2 wka = cmul(wn, root32(16 * r / R));
            const float2 wkb = u ? cmul(root32(16 * (r + 1) / R), cconj(wn)) : root32(8 / R + 16 * r / R);
            const float2 oa = cmulc(csub(xa, cconj(xma)), wka);   // times w_N^{-k}
            const float2 ob = cmulc(csub(xb, cconj(xmb)), wkb);
            za[r] = cadd(cadd(xa, cconj(xma)), mul_mi<true>(oa));   // E + i O
            zb[r] = cadd(cadd(xb, cconj(xmb)), mul_mi<true>(ob));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            A[r] = za[r];
            B[r] = zb[r];
        }
        dftR<R, true>(A);
        dftR<R, true>(B);
#pragma unroll
        for (int r = 0; r < R; r += 2) {
            sts4(buf + padi(ja[q] * R + r), A[r], A[r + 1]);
            sts4(buf + padi(jb[q] * R + r), B[r], B[r + 1]);
        }
    }
    team_sync<T>();
}

// Forward real FFT of length 2M.  Input: registers in first-pass order (time samples).  Output: the
// real-signal spectrum in buf (slot 0 = (X[0], X[M]), bins 1..M-1 in their slots, padded layout).  Ends
// with a team sync.  No thread of the team may still read buf on entry.
template <int M, int V>
__device__ __forceinline__ void rfft_regs_to_smem(float2 (&a)[FFT_P], float2 *buf, int t, const float2 *__restrict__ tw,
                                                  const float2 *__restrict__ twN) {
    constexpr int R0 = fft_radix(M, 0, V);
    pass_compute<M, R0, 1, false, 0>(a, t, tw);
    pass_store<M, R0, 1>(buf, t, a);
    team_sync<M / FFT_P>();
    passes_from<M, false, 1, fft_npass(M) - 1, V>(a, buf, t, tw);
    fwd_last_real<M, V>(a, buf, t, tw, twN);
}

// Inverse real FFT of length 2M (unnormalised: yields 2M x).  Input: real-signal spectrum in buf.
// Output: registers in first-forward-pass order (time samples).  The last pass reads buf, so the caller
// must sync the team before writing buf again.
template <int M, int V>
__device__ __forceinline__ void irfft_smem_to_regs(float2 (&a)[FFT_P], float2 *buf, int t, const float2 *__restrict__ tw,
                                                   const float2 *__restrict__ twN) {
    inv_first_real<M, V>(a, buf, t, twN);
    passes_from<M, true, 1, fft_npass(M), V>(a, buf, t, tw);
}

// The same with `mid()` run after the first pass: a caller that needs time-domain inputs after the
// transform issues their loads there, so they are not held in registers through the real
// pre-processing (the pass with the most live values) but still overlap the remaining passes.
//
// Where the second inverse pass is the radix-3 pass (the one that holds the most values at once), mid()
// runs after it instead.
template <int M, int V>
__host__ __device__ constexpr int irfft_mid_pass() {
    return (fft_npass(M) > 2 && ifft_radix(M, 1, V) == 3) ? 2 : 1;
}

template <int M, int V, class F>
__device__ __forceinline__ void irfft_smem_to_regs_mid(float2 (&a)[FFT_P], float2 *buf, int t, const float2 *__restrict__ tw,
                                                       const float2 *__restrict__ twN, F &&mid) {
    constexpr int MP = irfft_mid_pass<M, V>();
    inv_first_real<M, V>(a, buf, t, twN);
    passes_from<M, true, 1, MP, V>(a, buf, t, tw);
    mid();
    passes_from<M, true, MP, fft_npass(M), V>(a, buf, t, tw);
}

}  // namespace smdd
