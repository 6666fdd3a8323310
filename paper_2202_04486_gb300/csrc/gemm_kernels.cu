// Per-frequency complex matrix products of the MDC hot path (FP32 SIMT path).
//
// Eq. 2 states the MDC as one matrix product per frequency; Appendix A calls it the batched MMM.  With
// the model spectra Xh_f [nv x nr] (rows v) and the kernel spectra Dh_f [ns x nr] (rows s):
//   forward (Eq. 2, batch of Eq. 5):  Uh_f[v][b] = sum_r Xh_f[v][r] Dh_f[idx_b][r]
//   adjoint (Eq. 6):                  Gh_f[v][r] = sum_b Rh_f[v][b] conj(Dh_f[idx_b][r])
// The batch gather of kernel rows (the random subset of sources of Eq. 6) happens in the operand
// load: row idx_b of Dh_f is read in place, no gathered copy is made.
//
// With reciprocity (C_r of Eq. 4) the adjoint writes 1/2 (Gh_f + Gh_f^T) directly: since
// Gh_f^T[v][r] = sum_b conj(Dh_f[idx_b][v]) Rh_f[r][b], the symmetric part is one product with
// inner dimension 2 nb, A' = [Rh | conj(Dh_B)^T], B' = [conj(Dh_B) ; Rh^T], evaluated on the upper
// triangle of tiles only and mirrored into the lower triangle through shared memory.
#include "smdd_fft.cuh"
#include "smdd_internal.h"

namespace smdd {

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// acc += a * b (complex)
__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// ------------------------------------------------------------------------------------------------
// forward: C[f][v][b] = sum_r A[f][v][r] * Dh[f][idx_b][r]
// CTA: 4 warps, 128 rows v x 16 batch columns, one frequency.  Lane (vg = lane & 7, bg = lane >> 3)
// of warp w owns rows v0 + 32w + vg + 8i and columns b0 + bg + 4j (i, j < 4): a 4 x 4 complex register
// tile.  K (= nr) streams in chunks of 16 through a two-stage cp.async pipeline; every operand load is
// 128-bit (two consecutive k) and the 144-byte row pitch puts the 8 distinct rows of a load in 8
// distinct bank groups.
// ------------------------------------------------------------------------------------------------
constexpr int FW_THREADS = 128, FW_ROWS = 128, FW_NB = 16, FW_KC = 16, FW_LD = FW_KC + 2;
constexpr int FW_STAGE = (FW_ROWS + FW_NB) * FW_LD;   // float2 per stage
constexpr size_t FW_SMEM = 2 * FW_STAGE * sizeof(float2);

__global__ void __launch_bounds__(FW_THREADS, 4) k_cgemm_fwd(GemmArgs a) {
    extern __shared__ __align__(16) float2 gsm[];
    const int f = blockIdx.z;
    const int v0 = blockIdx.x * FW_ROWS, b0 = blockIdx.y * FW_NB;
    if (a.nf_active > 0 && f >= a.nf_active) {
        zero_tile(a.C + (long long)f * a.sCf, a.ldb, v0, FW_ROWS, b0, FW_NB, a.nv, a.nb);
        return;
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int vg = lane & 7, bg = lane >> 3;
    const float2 *Af = a.A + (long long)f * a.sAf;
    const float2 *Df = a.Dh + (long long)f * a.sDf;

    // kernel row of the batch column this thread stages (one 16-byte chunk per thread per stage)
    const int db = tid >> 3, dpart = tid & 7;
    int drow = -1;
    if (b0 + db < a.nb) {
        drow = a.idx[b0 + db];
        if (drow < 0 || drow >= a.ns) {
            atomicOr(a.status, 1);
            drow = -1;
        }
    }

    auto load_stage = [&](int stage, int k0) {
        float2 *sX = gsm + stage * FW_STAGE;
        float2 *sD = sX + FW_ROWS * FW_LD;
#pragma unroll
        for (int u = 0; u < (FW_ROWS * FW_KC / 2) / FW_THREADS; ++u) {
            const int c = tid + u * FW_THREADS;
            const int row = c >> 3, part = c & 7;
            const int k = k0 + 2 * part, v = v0 + row;
            int bytes = 0;
            const float2 *src = Af;
            if (v < a.nv && k < a.nr) {
                bytes = (k + 1 < a.nr) ? 16 : 8;
                src = Af + (long long)v * a.ldr + k;
            }
            cp_async16(sX + row * FW_LD + 2 * part, src, bytes);
        }
        {
            const int k = k0 + 2 * dpart;
            int bytes = 0;
            const float2 *src = Df;
            if (drow >= 0 && k < a.nr) {
                bytes = (k + 1 < a.nr) ? 16 : 8;
                src = Df + (long long)drow * a.ldr + k;
            }
            cp_async16(sD + db * FW_LD + 2 * dpart, src, bytes);
        }
        cp_async_commit();
    };

    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    const bool active = v0 + 32 * warp < a.nv;   // warps whose rows all lie past nv skip the products

    const int nk = (a.nr + FW_KC - 1) / FW_KC;
    load_stage(0, 0);
    for (int kc = 0; kc < nk; ++kc) {
        if (kc + 1 < nk) {
            load_stage((kc + 1) & 1, (kc + 1) * FW_KC);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (active) {
            const float2 *sX = gsm + (kc & 1) * FW_STAGE + (32 * warp + vg) * FW_LD;
            const float2 *sD = gsm + (kc & 1) * FW_STAGE + FW_ROWS * FW_LD + bg * FW_LD;
#pragma unroll
            for (int kk = 0; kk < FW_KC; kk += 2) {
                float4 x[4], d[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = *reinterpret_cast<const float4 *>(sX + 8 * i * FW_LD + kk);
#pragma unroll
                for (int j = 0; j < 4; ++j) d[j] = *reinterpret_cast<const float4 *>(sD + 4 * j * FW_LD + kk);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        cmac(acc[i][j], make_float2(x[i].x, x[i].y), make_float2(d[j].x, d[j].y));
                        cmac(acc[i][j], make_float2(x[i].z, x[i].w), make_float2(d[j].z, d[j].w));
                    }
            }
        }
        __syncthreads();
    }

    float2 *Cf = a.C + (long long)f * a.sCf;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int v = v0 + 32 * warp + vg + 8 * i;
        if (v >= a.nv) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + bg + 4 * j;
            if (b < a.nb) Cf[(long long)v * a.ldb + b] = acc[i][j];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// adjoint: C[f][v][r] = outscale * sum_k A'[v][k] B'[k][r]
//   k < nb :  A' = Rh[f][v][k],            B' = conj(Dh[f][idx_k][r])
//   k >= nb (reciprocity only, k' = k - nb):  A' = conj(Dh[f][idx_k'][v]),  B' = Rh[f][r][k']
// CTA tile TT x TT (TT = 64 or 32).  A warp covers 4*VPN rows x TT columns: lane (vp = lane / RG,
// rg = lane % RG) owns rows v0 + 4*VPN*w + 4vp + {0,1,2,3} and columns r0 + {2rg, 2rg+1, 2rg+TT/2,
// 2rg+TT/2+1}.  Operands are staged by cp.async in their global layouts -- residual-spectrum rows [v][k]
// and kernel-spectrum rows [k][r] -- and conjugated when used; chunks of 16 k per half.  Warps whose
// rows all lie past nv skip the products.
// ------------------------------------------------------------------------------------------------
constexpr int AD_KC = 16, AD_LDR = AD_KC + 2, AD_MAXNB = 1024;

template <int TT>
struct AdjGeom {
    static constexpr int RG = TT / 4;             // lanes along r
    static constexpr int VPN = 32 / RG;           // lane groups along v
    static constexpr int WROWS = 4 * VPN;         // rows per warp
    static constexpr int WARPS = TT / WROWS;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int RROWS = TT * AD_LDR;     // float2: residual rows of one block
    static constexpr int DROWS = AD_KC * TT;      // float2: kernel rows at one block's columns
    static constexpr size_t SMEM_OPER = 2 * (RROWS + DROWS) * sizeof(float2);
    static constexpr size_t SMEM_MIRROR = TT * (TT + 1) * sizeof(float2);
    static constexpr size_t SMEM = SMEM_OPER > SMEM_MIRROR ? SMEM_OPER : SMEM_MIRROR;
};

// stage rows [c0, c0 + TT) x k [k0, k0 + 16) of Rh (row pitch ldb) into s[TT][AD_LDR]
template <int TT>
__device__ __forceinline__ void stage_rrows(float2 *s, const float2 *Rf, int ldb, int c0, int nc, int k0, int nb, int tid) {
    constexpr int NT = AdjGeom<TT>::THREADS;
#pragma unroll
    for (int u = 0; u < TT * AD_KC / 2 / NT; ++u) {
        const int c = tid + u * NT, row = c >> 3, part = c & 7;
        const int k = k0 + 2 * part;
        int bytes = 0;
        const float2 *src = Rf;
        if (c0 + row < nc && k < nb) {
            bytes = (k + 1 < nb) ? 16 : 8;
            src = Rf + (long long)(c0 + row) * ldb + k;
        }
        cp_async16(s + row * AD_LDR + 2 * part, src, bytes);
    }
}

// stage kernel rows idx[k0 .. k0 + 16) at columns [c0, c0 + TT) into s[16][TT]
template <int TT>
__device__ __forceinline__ void stage_drows(float2 *s, const float2 *Df, int ldr, const int *sidx, int c0, int nc, int k0,
                                            int nb, int tid) {
    constexpr int NT = AdjGeom<TT>::THREADS, PARTS = TT / 2;
#pragma unroll
    for (int u = 0; u < AD_KC * TT / 2 / NT; ++u) {
        const int c = tid + u * NT, kk = c / PARTS, part = c % PARTS;
        const int col = c0 + 2 * part;
        int bytes = 0;
        const float2 *src = Df;
        if (k0 + kk < nb && col < nc) {
            const int srow = sidx[k0 + kk];
            if (srow >= 0) {
                bytes = (col + 1 < nc) ? 16 : 8;
                src = Df + (long long)srow * ldr + col;
            }
        }
        cp_async16(s + kk * TT + 2 * part, src, bytes);
    }
}

// acc += a * conj(b)
__device__ __forceinline__ void cmac_c(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.y, b.x, acc.y);
    acc.y = fmaf(-a.x, b.y, acc.y);
}

template <int TT, bool RECIP>
__global__ void __launch_bounds__(AdjGeom<TT>::THREADS, TT == 64 ? 3 : 8) k_cgemm_adj(GemmArgs a) {
    using G = AdjGeom<TT>;
    extern __shared__ __align__(16) float2 gsm[];
    float2 *sRv = gsm;                  // [TT][AD_LDR]  Rh rows of the v block
    float2 *sDr = sRv + G::RROWS;       // [16][TT]      kernel rows at the r block
    float2 *sRr = sDr + G::DROWS;       // [TT][AD_LDR]  Rh rows of the r block (reciprocity)
    float2 *sDv = sRr + G::RROWS;       // [16][TT]      kernel rows at the v block (reciprocity)
    __shared__ int sidx[AD_MAXNB];
    const int f = blockIdx.y;
    int vb, rb;
    if (RECIP) {   // upper-triangular tile enumeration: vb <= rb
        int t = blockIdx.x, row = 0, len = a.tiles_v;
        while (t >= len) { t -= len; ++row; --len; }
        vb = row;
        rb = row + t;
    } else {
        vb = blockIdx.x / a.tiles_r;
        rb = blockIdx.x % a.tiles_r;
    }
    const int v0 = vb * TT, r0 = rb * TT;
    if (a.nf_active > 0 && f >= a.nf_active) {
        zero_tile(a.C + (long long)f * a.sCf, a.ldr, v0, TT, r0, TT, a.nv, a.nr);
        if (RECIP) zero_tile(a.C + (long long)f * a.sCf, a.ldr, r0, TT, v0, TT, a.nr, a.nv);
        return;
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int vp = lane / G::RG, rg = lane % G::RG;
    const int vl = G::WROWS * warp + 4 * vp;     // first local row of the thread
    const bool active = v0 + G::WROWS * warp < a.nv;
    const float2 *Rf = a.A + (long long)f * a.sAf;
    const float2 *Df = a.Dh + (long long)f * a.sDf;

    for (int b = tid; b < a.nb; b += G::THREADS) {
        int s = a.idx[b];
        if (s < 0 || s >= a.ns) {
            atomicOr(a.status, 1);
            s = -1;
        }
        sidx[b] = s;
    }
    __syncthreads();

    float2 acc[4][4];   // [row][column: 2rg, 2rg+1, 2rg+TT/2, 2rg+TT/2+1]
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < a.nb; k0 += AD_KC) {
        stage_rrows<TT>(sRv, Rf, a.ldb, v0, a.nv, k0, a.nb, tid);
        stage_drows<TT>(sDr, Df, a.ldr, sidx, r0, a.nr, k0, a.nb, tid);
        if (RECIP) {
            stage_rrows<TT>(sRr, Rf, a.ldb, r0, a.nr, k0, a.nb, tid);
            stage_drows<TT>(sDv, Df, a.ldr, sidx, v0, a.nv, k0, a.nb, tid);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        const int kn = min(AD_KC, a.nb - k0);
        if (active) {
            // first half: Rh[v][k] * conj(Dh[idx_k][r])
            for (int kk = 0; kk < kn; kk += 2) {   // kn odd: column kn is zero filled
                float4 av[4], b0[2], b1[2];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4 *>(sRv + (vl + i) * AD_LDR + kk);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    b0[h] = *reinterpret_cast<const float4 *>(sDr + kk * TT + 2 * rg + (TT / 2) * h);
                    b1[h] = *reinterpret_cast<const float4 *>(sDr + (kk + 1) * TT + 2 * rg + (TT / 2) * h);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 a0 = make_float2(av[i].x, av[i].y), a1 = make_float2(av[i].z, av[i].w);
                        cmac_c(acc[i][2 * h], a0, make_float2(b0[h].x, b0[h].y));
                        cmac_c(acc[i][2 * h + 1], a0, make_float2(b0[h].z, b0[h].w));
                        cmac_c(acc[i][2 * h], a1, make_float2(b1[h].x, b1[h].y));
                        cmac_c(acc[i][2 * h + 1], a1, make_float2(b1[h].z, b1[h].w));
                    }
            }
            if (RECIP) {
                // second half: conj(Dh[idx_k][v]) * Rh[r][k]  (= the transpose of the first half)
                for (int kk = 0; kk < kn; kk += 2) {
                    float4 d0[2], d1[2], rv[4];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {   // rows vl + 2h, vl + 2h + 1 at k and k+1
                        d0[h] = *reinterpret_cast<const float4 *>(sDv + kk * TT + vl + 2 * h);
                        d1[h] = *reinterpret_cast<const float4 *>(sDv + (kk + 1) * TT + vl + 2 * h);
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int rl = 2 * rg + (j & 1) + (TT / 2) * (j >> 1);
                        rv[j] = *reinterpret_cast<const float4 *>(sRr + rl * AD_LDR + kk);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 dk0 = d0[i >> 1], dk1 = d1[i >> 1];
                        const float2 c0 = (i & 1) ? make_float2(dk0.z, dk0.w) : make_float2(dk0.x, dk0.y);
                        const float2 c1 = (i & 1) ? make_float2(dk1.z, dk1.w) : make_float2(dk1.x, dk1.y);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            cmac_c(acc[i][j], make_float2(rv[j].x, rv[j].y), c0);   // Rh[r][k] conj(Dh[k][v])
                            cmac_c(acc[i][j], make_float2(rv[j].z, rv[j].w), c1);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }

    float2 *Cf = a.C + (long long)f * a.sCf;
    const bool diag = RECIP && (vb == rb);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int vv = vl + i, v = v0 + vv;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int rr = 2 * rg + (TT / 2) * h, r = r0 + rr;
            const float2 x0 = cscale(acc[i][2 * h], a.outscale), x1 = cscale(acc[i][2 * h + 1], a.outscale);
            if (v < a.nv) {
                const bool w0 = r < a.nr && (!diag || v <= r), w1 = r + 1 < a.nr && (!diag || v <= r + 1);
                float2 *dst = Cf + (long long)v * a.ldr + r;
                if (w0 && w1) *reinterpret_cast<float4 *>(dst) = make_float4(x0.x, x0.y, x1.x, x1.y);
                else {
                    if (w0) dst[0] = x0;
                    if (w1) dst[1] = x1;
                }
            }
            if (RECIP) {   // mirror buffer (r, v); operands are dead after the final barrier
                gsm[rr * (TT + 1) + vv] = x0;
                gsm[(rr + 1) * (TT + 1) + vv] = x1;
            }
        }
    }
    if (RECIP && (diag || !a.no_mirror)) {   // diagonal tiles always mirror (see GemmArgs::no_mirror)
        __syncthreads();
        for (int e = tid; e < TT * TT; e += G::THREADS) {
            const int rr = e / TT, vv = e % TT;
            const int r = r0 + rr, v = v0 + vv;
            if (v < a.nv && r < a.nr && (!diag || v < r)) Cf[(long long)r * a.ldr + v] = gsm[rr * (TT + 1) + vv];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Few virtual sources (nv <= 8, the matrix-vector regime of a single-virtual-source inversion): the
// products are bound by reading the batch rows of Dh once, so a warp streams one kernel row against
// the nv model rows (forward) or a thread owns one receiver and walks the batch (adjoint).
// ------------------------------------------------------------------------------------------------
constexpr int GV_THREADS = 256, GV_MAXV = 8;

// forward: C[f][v][b] = sum_r A[f][v][r] Dh[f][idx_b][r]; one warp per batch entry b
template <int NV>
__global__ void __launch_bounds__(GV_THREADS) k_gemv_fwd(GemmArgs a) {
    const int f = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.y * (GV_THREADS / 32) + warp;
    if (b >= a.nb) return;   // warp-uniform; no barrier in this kernel
    int s = a.idx[b];
    if (s < 0 || s >= a.ns) {
        if (lane == 0) atomicOr(a.status, 1);
        s = -1;
    }
    const float2 *Af = a.A + (long long)f * a.sAf;
    float2 acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = make_float2(0.f, 0.f);
    if (s >= 0) {
        const float2 *d = a.Dh + (long long)f * a.sDf + (long long)s * a.ldr;
        for (int r = lane; r < a.nr; r += 32) {
            const float2 dv = __ldg(d + r);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (v < a.nv) {
                    const float2 x = __ldg(Af + (long long)v * a.ldr + r);
                    acc[v].x = fmaf(x.x, dv.x, fmaf(-x.y, dv.y, acc[v].x));
                    acc[v].y = fmaf(x.x, dv.y, fmaf(x.y, dv.x, acc[v].y));
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc[v].x += __shfl_down_sync(0xffffffffu, acc[v].x, o);
            acc[v].y += __shfl_down_sync(0xffffffffu, acc[v].y, o);
        }
    if (lane == 0) {
        float2 *Cf = a.C + (long long)f * a.sCf;
#pragma unroll
        for (int v = 0; v < NV; ++v)
            if (v < a.nv) Cf[(long long)v * a.ldb + b] = make_float2(acc[v].x * a.outscale, acc[v].y * a.outscale);
    }
}

// adjoint (no reciprocity): C[f][v][r] = outscale * sum_b A[f][v][b] conj(Dh[f][idx_b][r]); one thread
// per receiver r, the batch walked in order (the coefficients are warp-uniform broadcasts)
template <int NV>
__global__ void __launch_bounds__(GV_THREADS) k_gemv_adj(GemmArgs a) {
    __shared__ int sidx[AD_MAXNB];
    const int f = blockIdx.x, r = blockIdx.y * GV_THREADS + threadIdx.x;
    for (int b = threadIdx.x; b < a.nb; b += GV_THREADS) {
        int s = a.idx[b];
        if (s < 0 || s >= a.ns) {
            atomicOr(a.status, 1);
            s = -1;
        }
        sidx[b] = s;
    }
    __syncthreads();
    if (r >= a.nr) return;   // after the only barrier
    const float2 *Af = a.A + (long long)f * a.sAf;
    const float2 *Df = a.Dh + (long long)f * a.sDf;
    float2 acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = make_float2(0.f, 0.f);
    for (int b = 0; b < a.nb; ++b) {
        const int s = sidx[b];
        if (s < 0) continue;
        const float2 d = __ldg(Df + (long long)s * a.ldr + r);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v < a.nv) {
                const float2 c = __ldg(Af + (long long)v * a.ldb + b);
                // c * conj(d)
                acc[v].x = fmaf(c.x, d.x, fmaf(c.y, d.y, acc[v].x));
                acc[v].y = fmaf(c.y, d.x, fmaf(-c.x, d.y, acc[v].y));
            }
        }
    }
    float2 *Cf = a.C + (long long)f * a.sCf;
#pragma unroll
    for (int v = 0; v < NV; ++v)
        if (v < a.nv) Cf[(long long)v * a.ldr + r] = make_float2(acc[v].x * a.outscale, acc[v].y * a.outscale);
}

bool gemv_supported(int nv) { return nv >= 1 && nv <= GV_MAXV; }

cudaError_t launch_gemv_fwd(const GemmArgs &a, int nf, cudaStream_t st) {
    if (!gemv_supported(a.nv) || nf < 1) return cudaErrorInvalidValue;
    if (a.nf_active > 0 && a.nf_active < nf) return cudaErrorInvalidValue;   // band limits use the tiled kernels
    const dim3 grid(nf, (a.nb + GV_THREADS / 32 - 1) / (GV_THREADS / 32));
    if (a.nv == 1) k_gemv_fwd<1><<<grid, GV_THREADS, 0, st>>>(a);
    else if (a.nv <= 2) k_gemv_fwd<2><<<grid, GV_THREADS, 0, st>>>(a);
    else if (a.nv <= 4) k_gemv_fwd<4><<<grid, GV_THREADS, 0, st>>>(a);
    else k_gemv_fwd<8><<<grid, GV_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gemv_adj(const GemmArgs &a, int nf, cudaStream_t st) {
    if (!gemv_supported(a.nv) || nf < 1 || a.nb > AD_MAXNB) return cudaErrorInvalidValue;
    if (a.nf_active > 0 && a.nf_active < nf) return cudaErrorInvalidValue;
    const dim3 grid(nf, (a.nr + GV_THREADS - 1) / GV_THREADS);
    if (a.nv == 1) k_gemv_adj<1><<<grid, GV_THREADS, 0, st>>>(a);
    else if (a.nv <= 2) k_gemv_adj<2><<<grid, GV_THREADS, 0, st>>>(a);
    else if (a.nv <= 4) k_gemv_adj<4><<<grid, GV_THREADS, 0, st>>>(a);
    else k_gemv_adj<8><<<grid, GV_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t gemm_prepare() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_cgemm_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FW_SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_cgemm_adj<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AdjGeom<64>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_cgemm_adj<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AdjGeom<64>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_cgemm_adj<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AdjGeom<32>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_cgemm_adj<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AdjGeom<32>::SMEM))) return e;
    return cudaSuccess;
}

cudaError_t launch_cgemm_fwd(const GemmArgs &a, int nf, cudaStream_t st) {
    dim3 grid((a.nv + FW_ROWS - 1) / FW_ROWS, (a.nb + FW_NB - 1) / FW_NB, nf);
    k_cgemm_fwd<<<grid, FW_THREADS, FW_SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int TT>
static void launch_adj_tt(const GemmArgs &a0, bool recip, int nf, cudaStream_t st) {
    GemmArgs a = a0;
    a.tiles_v = (a.nv + TT - 1) / TT;
    a.tiles_r = (a.nr + TT - 1) / TT;
    if (recip) {
        const int ntiles = a.tiles_v * (a.tiles_v + 1) / 2;
        k_cgemm_adj<TT, true><<<dim3(ntiles, nf), AdjGeom<TT>::THREADS, AdjGeom<TT>::SMEM, st>>>(a);
    } else {
        k_cgemm_adj<TT, false><<<dim3(a.tiles_v * a.tiles_r, nf), AdjGeom<TT>::THREADS, AdjGeom<TT>::SMEM, st>>>(a);
    }
}

cudaError_t launch_cgemm_adj(const GemmArgs &a, bool recip, int nf, cudaStream_t st, int tile) {
    // 32-wide tiles waste less of the (triangular, ragged) output at moderate sizes; 64-wide tiles
    // re-use each staged operand for twice the products when the matrices are large (tile = 0: choose
    // by that rule; 32 or 64: as given)
    if (tile == 0) tile = (a.nv <= 512 && a.nr <= 512) ? 32 : 64;
    if (tile == 32) launch_adj_tt<32>(a, recip, nf, st);
    else launch_adj_tt<64>(a, recip, nf, st);
    return cudaGetLastError();
}

}  // namespace smdd
