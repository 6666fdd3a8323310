// Team FFT building blocks for the MDC hot path (sm_103a).
//
// Appendix A evaluates the multi-dimensional convolution as FFT along time -> one complex matrix
// product per frequency -> inverse FFT.  Here every time trace of length nt is zero padded to
// N = nfft = 2M >= 2nt-1 samples (linear, not circular, convolution on [0, nt)) and transformed as a
// real sequence through a complex FFT of length M on z[n] = x[2n] + i x[2n+1]:
//   X[k] = 1/2 (Z[k] + conj Z[M-k]) - i/2 w_N^k (Z[k] - conj Z[M-k]),   k = 0..M,
// and back through the matching pre-processing and an inverse complex FFT of length M.
//
// A "team" of T = M/16 threads owns one trace; each thread holds P = 16 complex values in registers.
// The complex FFT is a self-sorting Stockham factorisation M = R_1 R_2 ... R_m (radix 8 or 16 per
// pass, decided at compile time): pass p with radix R and span Ns = R_1...R_{p-1} maps butterfly j
// (inputs j + r M/R) to outputs (j - j%Ns) R + j%Ns + r Ns after the twiddles w_{Ns R}^{r (j%Ns)}.
// Between passes the values go through shared memory; the float2 index is XOR-swizzled within
// 16-element groups so that both the contiguous reads and the strided writes of a half-warp hit
// distinct banks.  The first forward pass reads its inputs straight from registers (global loads or
// the output of a previous inverse FFT), and the last inverse pass leaves its outputs in registers in
// exactly that order, so an inverse FFT, an element-wise epilogue and a forward FFT chain without a
// shared-memory round trip.
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

// multiply by w_8^k (forward root exp(-2 pi i k / 8); conjugate for INV), k = 1, 2, 3
template <bool INV, int K>
__device__ __forceinline__ float2 rot8(float2 a) {
    constexpr float h = 0.70710678118654752440f;
    if (K == 1) return INV ? make_float2((a.x - a.y) * h, (a.x + a.y) * h) : make_float2((a.x + a.y) * h, (a.y - a.x) * h);
    if (K == 2) return mul_mi<INV>(a);
    // K == 3
    return INV ? make_float2(-(a.x + a.y) * h, (a.x - a.y) * h) : make_float2((a.y - a.x) * h, -(a.x + a.y) * h);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2 *a) {
    // split into even / odd halves: y_k = E_k + w8^k O_k, y_{k+4} = E_k - w8^k O_k
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

// multiply by w_16^e, e in [0, 9] (forward root exp(-2 pi i e / 16))
template <bool INV>
__device__ __forceinline__ float2 rot16(float2 a, int e) {
    constexpr float c1 = 0.92387953251128675613f;  // cos(pi/8)
    constexpr float s1 = 0.38268343236508977173f;  // sin(pi/8)
    constexpr float h = 0.70710678118654752440f;   // cos(pi/4)
    float c, s;
    switch (e) {
        case 0: return a;
        case 1: c = c1; s = s1; break;
        case 2: c = h; s = h; break;
        case 3: c = s1; s = c1; break;
        case 4: return mul_mi<INV>(a);
        case 6: c = -h; s = h; break;
        case 9: c = -c1; s = -s1; break;
        default: c = 0.f; s = 0.f; break;  // e in {5,7,8} never occurs (n1, k1 < 4)
    }
    // forward: (c - i s) ; inverse: (c + i s)
    return INV ? make_float2(a.x * c - a.y * s, a.x * s + a.y * c) : make_float2(a.x * c + a.y * s, a.y * c - a.x * s);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2 *a) {
    // 16 = 4 x 4: n = n1 + 4 n2, k = k1 + 4 k2
    // inner DFT4 over n2 for each n1, twiddle w16^{n1 k1}, outer DFT4 over n1 for each k1.
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) dft4<INV>(a[n1], a[n1 + 4], a[n1 + 8], a[n1 + 12]);
    // now a[n1 + 4 k1] = B[n1][k1]
#pragma unroll
    for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) a[n1 + 4 * k1] = rot16<INV>(a[n1 + 4 * k1], n1 * k1);
    float2 y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 b0 = a[0 + 4 * k1], b1 = a[1 + 4 * k1], b2 = a[2 + 4 * k1], b3 = a[3 + 4 * k1];
        dft4<INV>(b0, b1, b2, b3);
        y[k1 + 0] = b0;
        y[k1 + 4] = b1;
        y[k1 + 8] = b2;
        y[k1 + 12] = b3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = y[i];
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2 *a) {
    if constexpr (R == 2) dft2<INV>(a[0], a[1]);
    else if constexpr (R == 4) dft4<INV>(a[0], a[1], a[2], a[3]);
    else if constexpr (R == 8) dft8<INV>(a);
    else dft16<INV>(a);
}

// ------------------------------------------------------------------------------------------------
// FFT plans: forward radices per pass for the complex length M (the inverse uses them reversed).
// ------------------------------------------------------------------------------------------------
__host__ __device__ constexpr int fft_npass(int M) {
    return M <= 16 ? 1 : M <= 256 ? 2 : 3;
}
__host__ __device__ constexpr int fft_radix(int M, int p) {
    // M = 32: 8*4 ... the product of the radices of a plan is M; each radix divides 16.
    return M == 16 ? 16
         : M == 32 ? (p == 0 ? 8 : 4)
         : M == 64 ? 8
         : M == 128 ? (p == 0 ? 8 : 16)
         : M == 256 ? 16
         : M == 512 ? 8
         : M == 1024 ? (p == 0 ? 16 : 8)
         : M == 2048 ? (p == 2 ? 8 : 16)
         : 16;  // 4096
}
// span before pass p of the forward plan
__host__ __device__ constexpr int fft_span(int M, int p) {
    return p == 0 ? 1 : fft_span(M, p - 1) * fft_radix(M, p - 1);
}
// inverse plan: pass p uses forward radix npass-1-p; its span is the product of the previous inverse radices
__host__ __device__ constexpr int ifft_radix(int M, int p) { return fft_radix(M, fft_npass(M) - 1 - p); }
__host__ __device__ constexpr int ifft_span(int M, int p) {
    return p == 0 ? 1 : ifft_span(M, p - 1) * ifft_radix(M, p - 1);
}

template <int M>
struct Team {
    static constexpr int T = M / 16;          // threads per trace
    static constexpr int TR = M <= 512 ? 16 : 8192 / M;   // traces per CTA
    static constexpr int THREADS = T * TR;    // CTA size
    static constexpr int STRIDE = M + 1;      // float2 per trace buffer in shared memory
    static constexpr size_t SMEM = (size_t)TR * STRIDE * sizeof(float2);
};

template <int T>
__device__ __forceinline__ void team_sync() {
    if constexpr (T <= 32) __syncwarp();
    else __syncthreads();
}

// registers: a[q*R + r] holds element j + r*(M/R) of the pass input, j = t + T*q
template <int M, int R>
__device__ __forceinline__ void pass_load(const float2 *buf, int t, float2 (&a)[16]) {
    constexpr int T = M / 16, Q = 16 / R, S = M / R;
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) a[q * R + r] = buf[swz(t + T * q + r * S)];
}

template <int M, int R, int NS, bool INV>
__device__ __forceinline__ void pass_compute(float2 (&a)[16], int t, const float2 *__restrict__ twM) {
    constexpr int T = M / 16, Q = 16 / R;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if constexpr (NS > 1) {
            const int k = (t + T * q) & (NS - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 w = __ldg(&twM[r * k * (M / (NS * R))]);
                a[q * R + r] = INV ? cmulc(a[q * R + r], w) : cmul(a[q * R + r], w);
            }
        }
        dftR<R, INV>(&a[q * R]);
    }
}

template <int M, int R, int NS>
__device__ __forceinline__ void pass_store(float2 *buf, int t, const float2 (&a)[16]) {
    constexpr int T = M / 16, Q = 16 / R;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int j = t + T * q, k = j & (NS - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) buf[swz((j - k) * R + k + r * NS)] = a[q * R + r];
    }
}

// Forward complex FFT of length M.  Input: registers in first-pass order (element t + T q + r M/R_1 in
// a[q R_1 + r]).  Output: natural order in buf (swizzled).  Ends with a team sync.
// The caller must make sure no thread of the team still reads buf before this is called.
template <int M>
__device__ __forceinline__ void fft_forward_regs_to_smem(float2 (&a)[16], float2 *buf, int t,
                                                         const float2 *__restrict__ twM) {
    constexpr int T = M / 16;
    constexpr int NP = fft_npass(M);
    pass_compute<M, fft_radix(M, 0), 1, false>(a, t, twM);
    pass_store<M, fft_radix(M, 0), 1>(buf, t, a);
    team_sync<T>();
    if constexpr (NP > 1) {
        pass_load<M, fft_radix(M, 1)>(buf, t, a);
        team_sync<T>();
        pass_compute<M, fft_radix(M, 1), fft_span(M, 1), false>(a, t, twM);
        pass_store<M, fft_radix(M, 1), fft_span(M, 1)>(buf, t, a);
        team_sync<T>();
    }
    if constexpr (NP > 2) {
        pass_load<M, fft_radix(M, 2)>(buf, t, a);
        team_sync<T>();
        pass_compute<M, fft_radix(M, 2), fft_span(M, 2), false>(a, t, twM);
        pass_store<M, fft_radix(M, 2), fft_span(M, 2)>(buf, t, a);
        team_sync<T>();
    }
}

// Inverse complex FFT of length M (unnormalised).  Input: natural order in buf.  Output: registers in
// first-forward-pass order (element t + T q + r M/R_1 in a[q R_1 + r]).  buf is free afterwards only
// after a team sync (the last pass reads it).
template <int M>
__device__ __forceinline__ void fft_inverse_smem_to_regs(float2 (&a)[16], float2 *buf, int t,
                                                         const float2 *__restrict__ twM) {
    constexpr int T = M / 16;
    constexpr int NP = fft_npass(M);
    pass_load<M, ifft_radix(M, 0)>(buf, t, a);
    pass_compute<M, ifft_radix(M, 0), 1, true>(a, t, twM);
    if constexpr (NP > 1) {
        team_sync<T>();
        pass_store<M, ifft_radix(M, 0), 1>(buf, t, a);
        team_sync<T>();
        pass_load<M, ifft_radix(M, 1)>(buf, t, a);
        pass_compute<M, ifft_radix(M, 1), ifft_span(M, 1), true>(a, t, twM);
    }
    if constexpr (NP > 2) {
        team_sync<T>();
        pass_store<M, ifft_radix(M, 1), ifft_span(M, 1)>(buf, t, a);
        team_sync<T>();
        pass_load<M, ifft_radix(M, 2)>(buf, t, a);
        pass_compute<M, ifft_radix(M, 2), ifft_span(M, 2), true>(a, t, twM);
    }
}

// After the forward complex FFT (Z in buf, natural order): form the real-input spectrum in place.
// Bins 1..M-1 in their slots; slot 0 holds (X[0], X[M]) (both real).  Ends with a team sync.
template <int M>
__device__ __forceinline__ void real_post(float2 *buf, int t, const float2 *__restrict__ twN) {
    constexpr int T = M / 16;
    for (int k = t; k <= M / 2; k += T) {
        if (k == 0) {
            const float2 z = buf[swz(0)];
            buf[swz(0)] = make_float2(z.x + z.y, z.x - z.y);
            continue;
        }
        const float2 zk = buf[swz(k)], zm = buf[swz(M - k)];
        const float2 e = cscale(cadd(zk, cconj(zm)), 0.5f);
        const float2 d = cscale(csub(zk, cconj(zm)), 0.5f);
        const float2 p = cmul(__ldg(&twN[k]), d);
        buf[swz(k)] = cadd(e, mul_mi<false>(p));                  // e - i p
        if (k != M - k) buf[swz(M - k)] = cadd(cconj(e), mul_mi<false>(cconj(p)));  // conj(e) - i conj(p)
    }
    team_sync<T>();
}

// Before the inverse complex FFT: buf holds a real-signal spectrum (slot 0 = (X[0], X[M]), bins
// 1..M-1 in their slots).  Forms Z[k] = E + i O with E = X[k] + conj X[M-k],
// O = (X[k] - conj X[M-k]) w_N^{-k}; the inverse complex FFT of Z then yields N x[2n] + i N x[2n+1].
// Ends with a team sync.
template <int M>
__device__ __forceinline__ void real_pre(float2 *buf, int t, const float2 *__restrict__ twN) {
    constexpr int T = M / 16;
    for (int k = t; k <= M / 2; k += T) {
        if (k == 0) {
            const float2 s = buf[swz(0)];
            buf[swz(0)] = make_float2(s.x + s.y, s.x - s.y);
            continue;
        }
        const float2 xk = buf[swz(k)], xm = buf[swz(M - k)];
        const float2 e = cadd(xk, cconj(xm));
        const float2 o = cmulc(csub(xk, cconj(xm)), __ldg(&twN[k]));   // times w_N^{-k}
        buf[swz(k)] = cadd(e, mul_mi<true>(o));                        // e + i o
        if (k != M - k) buf[swz(M - k)] = cadd(cconj(e), mul_mi<true>(cconj(o)));
    }
    team_sync<T>();
}

}  // namespace smdd
