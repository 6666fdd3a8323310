// Two-pass team FFT (radix-order variant 2) for complex lengths M = 128 .. 1024.
//
// M = 32 * R2.  A team of T = M / 32 threads owns one trace (at most a warp, so the team syncs are warp
// syncs); thread t holds the P = 32 complex values n = t + T m (m < 32) in register m.  The complex
// FFT is the self-sorting Stockham factorisation M = R1 * R2, R1 = 32:
//   pass 1 (span 1):   thread t transforms its own 32 values (a radix-32 butterfly, j = t) and writes
//                      the outputs y[32 t + k] to shared memory;
//   pass 2 (span 32):  butterflies j' = t + T q (q < 32 / R2) read y[j' + 32 r] (r < R2), multiply by
//                      w_M^{r j'} and transform; output r' of butterfly q is element j' + 32 r' =
//                      t + T (q + (32 / R2) r'), i.e. register q + (32 / R2) r' again.
// So both directions take and leave the values in the same per-thread order, one shared-memory
// exchange per transform.  The real-signal post-processing of the forward transform pairs bin k with
// bin M - k, which lies in lane (T - t) of the team: it is fetched with warp shuffles; the
// pre-processing of the inverse transform reads both bins from the spectrum tile in shared memory.
// Shared-memory layout of a trace: element i at float2 index i + (i / 32); every access is 8 bytes, and
// both the pass-1 stores (32 consecutive elements per thread) and the pass-2 loads (consecutive
// elements across threads) fall on distinct banks.
#pragma once

#include "smdd_fft.cuh"

namespace smdd {

__host__ __device__ constexpr int pad2(int i) { return i + (i >> 5); }

template <int M>
struct Fft2 {
    static_assert(M >= 128 && M <= 1024, "two-pass FFT for 128 <= M <= 1024");
    static constexpr int P = 32;
    static constexpr int R2 = M / 32;
    static constexpr int T = M / 32;                     // threads per trace
    static constexpr int Q = 32 / R2;                    // pass-2 butterflies per thread
    static constexpr int TR = 256 / T;                   // traces per CTA (256 threads)
    static constexpr int THREADS = T * TR;
    // float2 per trace buffer: pad2(M) plus an offset that puts the traces a half-warp of the tile
    // loader touches (16 / min(TR,16) bins of each of min(TR,16) traces) on distinct banks
    static constexpr int STRIDE = pad2(M) + (TR >= 16 ? 1 : 16 / TR);
    static constexpr size_t SMEM = (size_t)TR * STRIDE * sizeof(float2);
};

// w_64^m = exp(-2 pi i m / 64) for a compile-time m: the root that steps bin k = t + T m of a team
// (T / 2M = 1/64), so w_N^k = w_N^t w_64^m with one table load per thread
__host__ __device__ constexpr float2 root64(int m) {
    constexpr float c[17] = {1.0f, 0.99518472667219688624f, 0.98078528040323044913f, 0.95694033573220886494f,
                             0.92387953251128675613f, 0.88192126434835502971f, 0.83146961230254523708f,
                             0.77301045336273696081f, 0.70710678118654752440f, 0.63439328416364549822f,
                             0.55557023301960222474f, 0.47139673682599764856f, 0.38268343236508977173f,
                             0.29028467725446236764f, 0.19509032201612826785f, 0.09801714032956060199f,
                             0.0f};   // cos(pi j / 32), j = 0..16
    m &= 63;
    const int q = m >> 4, rr = m & 15;
    const float x = c[rr], y = c[16 - rr];   // cos, sin of the angle inside the quadrant
    return q == 0 ? make_float2(x, -y) : q == 1 ? make_float2(-y, -x) : q == 2 ? make_float2(-x, y) : make_float2(y, x);
}

// multiply by w_32^m (forward root exp(-2 pi i m / 32); conjugate for INV), m a compile-time constant
template <bool INV, int MM>
__device__ __forceinline__ float2 rot32(float2 a) {
    constexpr int m = ((MM % 32) + 32) % 32;
    if constexpr (m == 0) return a;
    else if constexpr (m == 8) return mul_mi<INV>(a);
    else if constexpr (m == 16) return make_float2(-a.x, -a.y);
    else if constexpr (m == 24) return mul_mi<!INV>(a);
    else if constexpr (m == 4) return rot8<INV, 1>(a);
    else if constexpr (m == 12) return rot8<INV, 3>(a);
    else if constexpr (m == 20) return make_float2(-rot8<INV, 1>(a).x, -rot8<INV, 1>(a).y);
    else if constexpr (m == 28) return make_float2(-rot8<INV, 3>(a).x, -rot8<INV, 3>(a).y);
    else {
        const float2 w = root32(m);
        return INV ? cmulc(a, w) : cmul(a, w);
    }
}

// radix-8 DFT of a[s], a[s + d], ..., a[s + 7d] (in place); HALF: the last four inputs are zero
template <bool INV, bool HALF, int S, int D, int N>
__device__ __forceinline__ void dft8_strided(float2 (&a)[N]) {
    float2 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (HALF && i >= 4) ? make_float2(0.f, 0.f) : a[S + i * D];
    if constexpr (HALF) {
        // even / odd halves with two zero inputs each: dft4(p, q, 0, 0) = (p + q, p - i q, p - q, p + i q)
        const float2 e0 = cadd(x[0], x[2]), e2 = csub(x[0], x[2]);
        const float2 iq = mul_mi<INV>(x[2]);
        const float2 e1 = cadd(x[0], iq), e3 = csub(x[0], iq);
        const float2 o0 = cadd(x[1], x[3]), o2 = csub(x[1], x[3]);
        const float2 iq1 = mul_mi<INV>(x[3]);
        const float2 o1 = cadd(x[1], iq1), o3 = csub(x[1], iq1);
        const float2 t1 = rot8<INV, 1>(o1), t2 = rot8<INV, 2>(o2), t3 = rot8<INV, 3>(o3);
        x[0] = cadd(e0, o0);
        x[4] = csub(e0, o0);
        x[1] = cadd(e1, t1);
        x[5] = csub(e1, t1);
        x[2] = cadd(e2, t2);
        x[6] = csub(e2, t2);
        x[3] = cadd(e3, t3);
        x[7] = csub(e3, t3);
    } else {
        dft8<INV>(x);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) a[S + i * D] = x[i];
}

template <bool INV, int S, int D, int N>
__device__ __forceinline__ void dft4_strided(float2 (&a)[N]) {
    dft4<INV>(a[S], a[S + D], a[S + 2 * D], a[S + 3 * D]);
}

// DFT-32 of the 32 registers a[B .. B+32) in place, natural order in and out.  Decimation in time by
// 4: four DFT-8s over a[B + 4 n + s] (n < 8), twiddles w_32^{s k'}, then a DFT-4 over s for every
// k'.  HALF: inputs 16..31 are zero (zero padding of the forward transform).
template <bool INV, bool HALF, int B, int N>
__device__ __forceinline__ void dft32_regs(float2 (&a)[N]) {
    float2 y[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) y[i] = a[B + i];
    // DFT-8 of each residue class s (elements 4n + s) in place
    dft8_strided<INV, HALF, 0, 4>(y);
    dft8_strided<INV, HALF, 1, 4>(y);
    dft8_strided<INV, HALF, 2, 4>(y);
    dft8_strided<INV, HALF, 3, 4>(y);
    // y[4 k' + s] now holds Y_s[k']; twiddle and DFT-4 over s: X[k' + 8 q]
#pragma unroll
    for (int kp = 0; kp < 8; ++kp) {
        float2 z0 = y[4 * kp + 0];
        float2 z1, z2, z3;
        switch (kp) {   // compile-time after unrolling
#define SMDD_TW(K)                                   \
    case K:                                          \
        z1 = rot32<INV, 1 * K>(y[4 * K + 1]);        \
        z2 = rot32<INV, 2 * K>(y[4 * K + 2]);        \
        z3 = rot32<INV, 3 * K>(y[4 * K + 3]);        \
        break;
            SMDD_TW(0) SMDD_TW(1) SMDD_TW(2) SMDD_TW(3) SMDD_TW(4) SMDD_TW(5) SMDD_TW(6) SMDD_TW(7)
#undef SMDD_TW
        }
        dft4<INV>(z0, z1, z2, z3);
        a[B + kp] = z0;
        a[B + kp + 8] = z1;
        a[B + kp + 16] = z2;
        a[B + kp + 24] = z3;
    }
}

// DFT-16 of the 16 registers a[B + D i] (i < 16), natural order, in place.  Decimation in time by 4:
// four DFT-4s over i = 4 n + s, twiddles w_16^{s k'} = w_32^{2 s k'}, DFT-4 over s.
template <bool INV, int B, int D, int N>
__device__ __forceinline__ void dft16_regs(float2 (&a)[N]) {
    float2 y[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) y[i] = a[B + D * i];
    dft4_strided<INV, 0, 4>(y);
    dft4_strided<INV, 1, 4>(y);
    dft4_strided<INV, 2, 4>(y);
    dft4_strided<INV, 3, 4>(y);
#pragma unroll
    for (int kp = 0; kp < 4; ++kp) {
        float2 z0 = y[4 * kp + 0];
        float2 z1, z2, z3;
        switch (kp) {
#define SMDD_TW(K)                                   \
    case K:                                          \
        z1 = rot32<INV, 2 * 1 * K>(y[4 * K + 1]);    \
        z2 = rot32<INV, 2 * 2 * K>(y[4 * K + 2]);    \
        z3 = rot32<INV, 2 * 3 * K>(y[4 * K + 3]);    \
        break;
            SMDD_TW(0) SMDD_TW(1) SMDD_TW(2) SMDD_TW(3)
#undef SMDD_TW
        }
        dft4<INV>(z0, z1, z2, z3);
        a[B + D * kp] = z0;
        a[B + D * (kp + 4)] = z1;
        a[B + D * (kp + 8)] = z2;
        a[B + D * (kp + 12)] = z3;
    }
}

// radix-R2 DFT of the registers a[B + D r] (r < R2), natural order, in place
template <int R2, bool INV, int B, int D, int N>
__device__ __forceinline__ void dftR2_regs(float2 (&a)[N]) {
    if constexpr (R2 == 32) {
        static_assert(D == 1, "the radix-32 pass-2 butterfly is one per thread");
        dft32_regs<INV, false, B>(a);
    } else if constexpr (R2 == 16) {
        dft16_regs<INV, B, D>(a);
    } else if constexpr (R2 == 8) {
        dft8_strided<INV, false, B, D>(a);
    } else {
        dft4_strided<INV, B, D>(a);
    }
}

// Pass 1 + exchange + pass 2 of one direction.  a: the 32 values n = t + T m in register m (pass-1
// order); on return the transform's outputs in the same order.  HALF_IN: the inputs with m >= 16 are
// zero (forward transform of zero-padded data).  buf: this trace's shared-memory buffer; tw2: the
// pass-2 table [r][j'] = w_M^{r j'} (r < R2, j' < 32).  Ends with a team sync after the last read.
template <int M, bool INV, bool HALF_IN>
__device__ __forceinline__ void fft2_core(float2 (&a)[32], float2 *buf, int t, const float2 *__restrict__ tw2) {
    using F = Fft2<M>;
    constexpr int T = F::T, R2 = F::R2, Q = F::Q;
    dft32_regs<INV, HALF_IN, 0>(a);
    // y[32 t + k] = a[k]
#pragma unroll
    for (int k = 0; k < 32; ++k) buf[pad2(32 * t + k)] = a[k];
    __syncwarp();
    // pass 2: butterfly j' = t + T q reads y[j' + 32 r] into register q + Q r
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int jp = t + T * q;
#pragma unroll
        for (int r = 0; r < R2; ++r) a[q + Q * r] = buf[pad2(jp + 32 * r)];
    }
    __syncwarp();   // every lane of the team has read buf: the caller may write it again
    // twiddles w_M^{r j'}: r = r_lo + 8 r_hi, from the table rows r_lo (< 8) and 8 r_hi (each row r holds
    // w_M^{r j'} for j' < 32): R2/8 + 6 loads and R2 - 8 products instead of R2 - 1 loads
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int jp = t + T * q;
        constexpr int RL = R2 < 8 ? R2 : 8, RH = R2 / RL;
        float2 wl[RL], wh[RH];
#pragma unroll
        for (int r = 1; r < RL; ++r) wl[r] = __ldg(tw2 + r * 32 + jp);
#pragma unroll
        for (int h = 1; h < RH; ++h) wh[h] = __ldg(tw2 + h * RL * 32 + jp);
#pragma unroll
        for (int r = 1; r < R2; ++r) {
            const int lo = r % RL, hi = r / RL;
            const float2 w = hi == 0 ? wl[lo] : lo == 0 ? wh[hi] : cmul(wl[lo], wh[hi]);
            a[q + Q * r] = INV ? cmulc(a[q + Q * r], w) : cmul(a[q + Q * r], w);
        }
    }
    // the DFTs of the pass-2 butterflies: butterfly q owns registers q + Q r
    if constexpr (Q == 1) dftR2_regs<R2, INV, 0, 1>(a);
    else if constexpr (Q == 2) { dftR2_regs<R2, INV, 0, 2>(a); dftR2_regs<R2, INV, 1, 2>(a); }
    else if constexpr (Q == 4) {
        dftR2_regs<R2, INV, 0, 4>(a); dftR2_regs<R2, INV, 1, 4>(a);
        dftR2_regs<R2, INV, 2, 4>(a); dftR2_regs<R2, INV, 3, 4>(a);
    } else {
        dftR2_regs<R2, INV, 0, 8>(a); dftR2_regs<R2, INV, 1, 8>(a); dftR2_regs<R2, INV, 2, 8>(a);
        dftR2_regs<R2, INV, 3, 8>(a); dftR2_regs<R2, INV, 4, 8>(a); dftR2_regs<R2, INV, 5, 8>(a);
        dftR2_regs<R2, INV, 6, 8>(a); dftR2_regs<R2, INV, 7, 8>(a);
    }
}

// Forward real FFT of length 2M: a holds z[n] = (x[2n], x[2n+1]) for n = t + T m (m < 16; registers
// 16..31 are ignored: zero padding).  Writes the real-signal spectrum into buf (slot 0 = (X[0], X[M]),
// bin k at pad2(k)).  Ends with a team sync.
template <int M>
__device__ __forceinline__ void rfft2_regs_to_smem(float2 (&a)[32], float2 *buf, int t, const float2 *__restrict__ tw2,
                                                   const float2 *__restrict__ twN) {
    using F = Fft2<M>;
    constexpr int T = F::T;
    fft2_core<M, false, true>(a, buf, t, tw2);
    // thread t holds Z[k], k = t + T m.  Z[M - k] = Z[(T - t) + T (31 - m)] is register 31 - m of lane
    // T - t (t > 0), and register (32 - m) % 32 of this lane for t = 0.
    // (pass 2 left buf free: its last reads precede the sync at the end of fft2_core)
    const unsigned lane = threadIdx.x & 31;
    const int src = (int)(lane & ~(unsigned)(T - 1)) + ((T - t) & (T - 1));
    const float2 wt = __ldg(twN + t);              // w_N^t; w_N^k = w_N^t w_64^m
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const float sx = __shfl_sync(0xffffffffu, a[31 - m].x, src);
        const float sy = __shfl_sync(0xffffffffu, a[31 - m].y, src);
        const float2 zm = (t == 0) ? a[(32 - m) & 31] : make_float2(sx, sy);
        const float2 z = a[m];
        const int k = t + T * m;
        const float2 wn = cmul(wt, root64(m));     // w_N^k, N = 2M
        const float2 e = cscale(cadd(z, cconj(zm)), 0.5f);
        const float2 d = cmul(wn, cscale(csub(z, cconj(zm)), 0.5f));
        float2 x = cadd(e, mul_mi<false>(d));
        if (m == 0 && t == 0) x.y = a[0].x - a[0].y;   // slot 0 packs X[0] and X[M]
        buf[pad2(k)] = x;
    }
    __syncwarp();
}

// Inverse real FFT of length 2M (unnormalised: 2M x).  buf holds a real-signal spectrum (slot 0 =
// (X[0], X[M])).  On return a holds z[n] = (x[2n], x[2n+1]) for n = t + T m (only m < 16 are ever
// needed by the callers).  Ends with a team sync after the last read of buf.
template <int M>
__device__ __forceinline__ void irfft2_smem_to_regs(float2 (&a)[32], float2 *buf, int t, const float2 *__restrict__ tw2,
                                                    const float2 *__restrict__ twN) {
    using F = Fft2<M>;
    constexpr int T = F::T;
    // pre-processing: Z[k] = E + i O, E = X[k] + conj X[M-k], O = (X[k] - conj X[M-k]) w_N^{-k}
    const float2 wt = __ldg(twN + t);
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const int k = t + T * m;
        float2 xk = buf[pad2(k)];
        float2 xm = buf[pad2(M - k)];              // k = 0: pad2(M) is slot M, read but replaced below
        if (k == 0) {
            const float2 s0 = xk;
            xk = make_float2(s0.x, 0.f);
            xm = make_float2(s0.y, 0.f);
        }
        const float2 wn = cmul(wt, root64(m));
        const float2 e = cadd(xk, cconj(xm));
        const float2 o = cmulc(csub(xk, cconj(xm)), wn);
        a[m] = cadd(e, mul_mi<true>(o));
    }
    __syncwarp();
    fft2_core<M, true, false>(a, buf, t, tw2);
}

}  // namespace smdd
