// Three-pass team FFT for complex length M = 1536 (FFT length 3072; radix-order variant 2 of that
// length, the counterpart of the two-pass FFT of smdd_fft2.cuh for M = 128 .. 1024).
//
// One warp owns one trace (T = 32 threads); thread t holds the P = 48 complex values n = t + 32 m
// (m < 48) in register m.  The complex FFT is the self-sorting Stockham factorisation 1536 = 48 * 4 * 8:
//   pass 1 (radix 48, span 1):   thread t transforms its own 48 values in registers (decimation in time
//                                by 3: three DFT-16s over m = 3 n + s, twiddles w_48^{s k}, sixteen
//                                DFT-3s) and writes the outputs y[48 t + k] to shared memory;
//   pass 2 (radix 4, span 48):   butterflies j = t + 32 q (q < 12) read y[j + 384 r] (r < 4), multiply
//                                by w_192^{r (j % 48)}, transform, and write (j - j%48) 4 + j%48 + 48 r;
//   pass 3 (radix 8, span 192):  butterflies j = t + 32 q (q < 6) read j + 192 r (r < 8) into register
//                                q + 6 r, multiply by w_1536^{r j} and transform; output r' of butterfly
//                                q is element j + 192 r' = t + 32 (q + 6 r'), i.e. register q + 6 r'.
// So both directions take and leave the values in the same per-thread order, with two shared-memory
// exchanges per transform and warp syncs only.  The real-signal post-processing pairs bin k = t + 32 m
// with M - k, held by lane (32 - t) % 32 in register 47 - m (register (48 - m) % 48 of lane 0 for t = 0),
// through warp shuffles; w_N^k = w_N^t w_96^m (N = 3072).  Shared-memory layout of a trace: element i at
// float2 index i + i / 32 (every access 8 bytes; the stride-48 stores of pass 1 hit each bank pair twice
// per warp, the minimum for 32 lanes of 8 bytes).
#pragma once

#include "smdd_fft2.cuh"

namespace smdd {

struct Fft3 {
    static constexpr int M = 1536;
    static constexpr int P = 48;
    static constexpr int T = 32;                           // threads per trace (one warp)
    static constexpr int TR = 8;                           // traces per CTA (256 threads)
    static constexpr int THREADS = T * TR;
    static constexpr int STRIDE = pad2(M) + 2;             // float2 per trace buffer (+2: traces of a
                                                           // tile-loader half-warp on distinct banks)
    static constexpr size_t SMEM = (size_t)TR * STRIDE * sizeof(float2);
    static constexpr int TW2 = 4 * 48;                     // pass-2 table [r][k] = w_192^{r k}
    static constexpr int TW_SIZE = TW2 + 8 * 192;          // + pass-3 table [r][j] = w_1536^{r j}
};

// w_96^m = exp(-2 pi i m / 96) for a compile-time m (m taken mod 96)
__host__ __device__ constexpr float2 root96(int m) {
    constexpr float c[25] = {1.0f,
                             0.99785892323860347819f, 0.99144486137381041114f, 0.98078528040323044913f,
                             0.96592582628906828675f, 0.94693012949510569490f, 0.92387953251128675613f,
                             0.89687274153268836784f, 0.86602540378443864676f, 0.83146961230254523708f,
                             0.79335334029123516458f, 0.75183980747897738046f, 0.70710678118654752440f,
                             0.65934581510006884849f, 0.60876142900872063942f, 0.55557023301960222474f,
                             0.50000000000000000000f, 0.44228869021900124935f, 0.38268343236508977173f,
                             0.32143946530316158978f, 0.25881904510252076235f, 0.19509032201612826785f,
                             0.13052619222005159155f, 0.06540312923014306684f, 0.0f};   // cos(pi j / 48)
    m = ((m % 96) + 96) % 96;
    const int q = m / 24, rr = m % 24;
    const float x = c[rr], y = c[24 - rr];   // cos, sin of the angle inside the quadrant
    return q == 0 ? make_float2(x, -y) : q == 1 ? make_float2(-y, -x) : q == 2 ? make_float2(-x, y) : make_float2(y, x);
}

// multiply by w_48^J (forward root; conjugate for INV), J a compile-time constant
template <bool INV, int J>
__device__ __forceinline__ float2 rot48(float2 a) {
    constexpr int j = ((J % 48) + 48) % 48;
    if constexpr (j == 0) return a;
    else if constexpr (j == 12) return mul_mi<INV>(a);
    else if constexpr (j == 24) return make_float2(-a.x, -a.y);
    else if constexpr (j == 36) return mul_mi<!INV>(a);
    else {
        const float2 w = root96(2 * j);
        return INV ? cmulc(a, w) : cmul(a, w);
    }
}

// DFT-48 of the 48 registers, natural order in and out (register m = element m of this thread's
// stride-32 subsequence).  Decimation in time by 3: DFT-16 over m = 3 n + s for s = 0, 1, 2, then for
// every k < 16: Y_s[k] w_48^{s k} and a DFT-3 over s giving outputs k, k + 16, k + 32.
template <bool INV>
__device__ __forceinline__ void dft48_regs(float2 (&a)[48]) {
    dft16_regs<INV, 0, 3>(a);
    dft16_regs<INV, 1, 3>(a);
    dft16_regs<INV, 2, 3>(a);
    float2 y[48];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        float2 y0 = a[3 * k], y1, y2;
        switch (k) {   // compile-time after unrolling
#define SMDD_TW48(K)                                     \
    case K:                                              \
        y1 = rot48<INV, K>(a[3 * K + 1]);                \
        y2 = rot48<INV, 2 * K>(a[3 * K + 2]);            \
        break;
            SMDD_TW48(0) SMDD_TW48(1) SMDD_TW48(2) SMDD_TW48(3) SMDD_TW48(4) SMDD_TW48(5) SMDD_TW48(6)
            SMDD_TW48(7) SMDD_TW48(8) SMDD_TW48(9) SMDD_TW48(10) SMDD_TW48(11) SMDD_TW48(12) SMDD_TW48(13)
            SMDD_TW48(14) SMDD_TW48(15)
#undef SMDD_TW48
        }
        dft3<INV>(y0, y1, y2);
        y[k] = y0;
        y[k + 16] = y1;
        y[k + 32] = y2;
    }
#pragma unroll
    for (int m = 0; m < 48; ++m) a[m] = y[m];
}

// One direction of the complex FFT of length 1536.  a: the 48 values n = t + 32 m in register m; on
// return the transform's outputs in the same order.  buf: this trace's shared-memory buffer; tw: the
// tables of Fft3 (pass 2 at 0, pass 3 at TW2).  Ends with a warp sync after the last read of buf.
template <bool INV>
__device__ __forceinline__ void fft3_core(float2 (&a)[48], float2 *buf, int t, const float2 *__restrict__ tw) {
    // pass 1: radix 48 in registers; y[48 t + k] = a[k]
    dft48_regs<INV>(a);
#pragma unroll
    for (int k = 0; k < 48; ++k) buf[pad2(48 * t + k)] = a[k];
    __syncwarp();
    // pass 2: radix 4, span 48; butterfly q of this thread (j = t + 32 q) holds input r in register q + 12 r
#pragma unroll
    for (int q = 0; q < 12; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) a[q + 12 * r] = buf[pad2(t + 32 * q + 384 * r)];
    __syncwarp();   // every lane has read buf: the outputs may overwrite it
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const int j = t + 32 * q, k = j % 48;
#pragma unroll
        for (int r = 1; r < 4; ++r) {
            const float2 w = __ldg(tw + r * 48 + k);
            a[q + 12 * r] = INV ? cmulc(a[q + 12 * r], w) : cmul(a[q + 12 * r], w);
        }
        dft4<INV>(a[q], a[q + 12], a[q + 24], a[q + 36]);
        const int o = (j - k) * 4 + k;
#pragma unroll
        for (int r = 0; r < 4; ++r) buf[pad2(o + 48 * r)] = a[q + 12 * r];
    }
    __syncwarp();
    // pass 3: radix 8, span 192; butterfly q (j = t + 32 q) holds input r in register q + 6 r
#pragma unroll
    for (int q = 0; q < 6; ++q)
#pragma unroll
        for (int r = 0; r < 8; ++r) a[q + 6 * r] = buf[pad2(t + 32 * q + 192 * r)];
    __syncwarp();   // every lane has read buf: the caller may write it again
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int j = t + 32 * q;
        // twiddles w_1536^{r j}: w^1 and w^4 from the table, the other powers by products (a few ulp)
        const float2 w1 = __ldg(tw + Fft3::TW2 + 192 + j), w4 = __ldg(tw + Fft3::TW2 + 4 * 192 + j);
        float2 w[8];
        twiddle_powers<8>(w1, w4, w);
        float2 x[8];
        x[0] = a[q];
#pragma unroll
        for (int r = 1; r < 8; ++r) x[r] = INV ? cmulc(a[q + 6 * r], w[r]) : cmul(a[q + 6 * r], w[r]);
        dft8<INV>(x);
#pragma unroll
        for (int r = 0; r < 8; ++r) a[q + 6 * r] = x[r];
    }
}

// Forward real FFT of length 3072: a holds z[n] = (x[2n], x[2n+1]) for n = t + 32 m (m < 24; registers
// 24..47 are ignored: zero padding).  Writes the real-signal spectrum into buf (slot 0 = (X[0], X[M]),
// bin k at pad2(k)).  Ends with a warp sync.
__device__ __forceinline__ void rfft3_regs_to_smem(float2 (&a)[48], float2 *buf, int t, const float2 *__restrict__ tw,
                                                   const float2 *__restrict__ twN) {
#pragma unroll
    for (int m = 24; m < 48; ++m) a[m] = make_float2(0.f, 0.f);
    fft3_core<false>(a, buf, t, tw);
    // Z[M - k] for k = t + 32 m: register 47 - m of lane 32 - t (t > 0), register (48 - m) % 48 of lane 0
    const int src = (32 - t) & 31;
    const float2 wt = __ldg(twN + t);              // w_N^t; w_N^k = w_N^t w_96^m
#pragma unroll
    for (int m = 0; m < 48; ++m) {
        const float sx = __shfl_sync(0xffffffffu, a[47 - m].x, src);
        const float sy = __shfl_sync(0xffffffffu, a[47 - m].y, src);
        const float2 zm = (t == 0) ? a[(48 - m) % 48] : make_float2(sx, sy);
        const float2 z = a[m];
        const float2 wn = cmul(wt, root96(m));
        const float2 e = cscale(cadd(z, cconj(zm)), 0.5f);
        const float2 d = cmul(wn, cscale(csub(z, cconj(zm)), 0.5f));
        float2 x = cadd(e, mul_mi<false>(d));
        if (m == 0 && t == 0) x.y = a[0].x - a[0].y;   // slot 0 packs X[0] and X[M]
        buf[pad2(t + 32 * m)] = x;
    }
    __syncwarp();
}

// Inverse real FFT of length 3072 (unnormalised: 3072 x).  buf holds a real-signal spectrum (slot 0 =
// (X[0], X[M])).  On return a holds z[n] = (x[2n], x[2n+1]) for n = t + 32 m (the callers use m < 24).
// Ends with a warp sync after the last read of buf.
__device__ __forceinline__ void irfft3_smem_to_regs(float2 (&a)[48], float2 *buf, int t, const float2 *__restrict__ tw,
                                                    const float2 *__restrict__ twN) {
    constexpr int M = Fft3::M;
    const float2 wt = __ldg(twN + t);
#pragma unroll
    for (int m = 0; m < 48; ++m) {
        const int k = t + 32 * m;
        float2 xk = buf[pad2(k)];
        float2 xm = buf[pad2(M - k)];              // k = 0: slot M, read but replaced below
        if (k == 0) {
            const float2 s0 = xk;
            xk = make_float2(s0.x, 0.f);
            xm = make_float2(s0.y, 0.f);
        }
        const float2 wn = cmul(wt, root96(m));
        const float2 e = cadd(xk, cconj(xm));
        const float2 o = cmulc(csub(xk, cconj(xm)), wn);
        a[m] = cadd(e, mul_mi<true>(o));
    }
    __syncwarp();
    fft3_core<true>(a, buf, t, tw);
}

}  // namespace smdd
