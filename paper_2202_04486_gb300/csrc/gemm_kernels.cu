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
// CTA: 128 threads, 256 rows v (thread t owns rows t and t+128), 16 batch columns, one frequency.
// K (= nr) streamed in chunks of 16 through a two-stage cp.async pipeline.
// ------------------------------------------------------------------------------------------------
constexpr int FW_THREADS = 128, FW_ROWS = 256, FW_NB = 16, FW_KC = 16, FW_LD = FW_KC + 2;
constexpr int FW_STAGE = (FW_ROWS + FW_NB) * FW_LD;   // float2 per stage
constexpr size_t FW_SMEM = 2 * FW_STAGE * sizeof(float2);

__global__ void __launch_bounds__(FW_THREADS) k_cgemm_fwd(GemmArgs a) {
    extern __shared__ __align__(16) float2 gsm[];
    const int f = blockIdx.z;
    const int v0 = blockIdx.x * FW_ROWS, b0 = blockIdx.y * FW_NB;
    const int tid = threadIdx.x;
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

    float2 acc[2][FW_NB];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int b = 0; b < FW_NB; ++b) acc[i][b] = make_float2(0.f, 0.f);

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
        const float2 *sX = gsm + (kc & 1) * FW_STAGE;
        const float2 *sD = sX + FW_ROWS * FW_LD;
#pragma unroll
        for (int kk = 0; kk < FW_KC; kk += 2) {
            const float4 xa = *reinterpret_cast<const float4 *>(sX + tid * FW_LD + kk);
            const float4 xb = *reinterpret_cast<const float4 *>(sX + (tid + 128) * FW_LD + kk);
#pragma unroll
            for (int b = 0; b < FW_NB; ++b) {
                const float4 d = *reinterpret_cast<const float4 *>(sD + b * FW_LD + kk);
                cmac(acc[0][b], make_float2(xa.x, xa.y), make_float2(d.x, d.y));
                cmac(acc[0][b], make_float2(xa.z, xa.w), make_float2(d.z, d.w));
                cmac(acc[1][b], make_float2(xb.x, xb.y), make_float2(d.x, d.y));
                cmac(acc[1][b], make_float2(xb.z, xb.w), make_float2(d.z, d.w));
            }
        }
        __syncthreads();
    }

    float2 *Cf = a.C + (long long)f * a.sCf;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int v = v0 + tid + 128 * i;
        if (v >= a.nv) continue;
        float2 *crow = Cf + (long long)v * a.ldb;
#pragma unroll
        for (int b = 0; b < FW_NB; b += 2) {
            if (b0 + b < a.nb)   // ldb is even, so column b0+b+1 exists (padding when == nb)
                *reinterpret_cast<float4 *>(crow + b0 + b) =
                    make_float4(acc[i][b].x, acc[i][b].y, acc[i][b + 1].x, acc[i][b + 1].y);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// adjoint: C[f][v][r] = outscale * sum_k A'[v][k] B'[k][r]
//   k < nb :  A' = Rh[f][v][k],            B' = conj(Dh[f][idx_k][r])
//   k >= nb (reciprocity only, k' = k - nb):  A' = conj(Dh[f][idx_k'][v]),  B' = Rh[f][r][k']
// CTA: 128 threads, tile 64 v x 64 r, warp w owns rows 16w..16w+15, lane owns columns lane, lane+32.
// ------------------------------------------------------------------------------------------------
constexpr int AD_THREADS = 128, AD_T = 64, AD_KC = 16;
constexpr size_t AD_SMEM_OPER = 2 * AD_KC * AD_T * sizeof(float2);
constexpr size_t AD_SMEM_MIRROR = AD_T * (AD_T + 1) * sizeof(float2);

template <bool RECIP>
__global__ void __launch_bounds__(AD_THREADS) k_cgemm_adj(GemmArgs a) {
    extern __shared__ __align__(16) float2 gsm[];
    float2 *sA = gsm;                  // [AD_KC][AD_T]  (k, v)
    float2 *sB = gsm + AD_KC * AD_T;   // [AD_KC][AD_T]  (k, r)
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
    const int v0 = vb * AD_T, r0 = rb * AD_T;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float2 *Rf = a.A + (long long)f * a.sAf;
    const float2 *Df = a.Dh + (long long)f * a.sDf;
    const int K = RECIP ? 2 * a.nb : a.nb;

    float2 acc[16][2];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < K; k0 += AD_KC) {
        // stage A' (k, v) and B' (k, r)
        for (int e = tid; e < AD_KC * AD_T; e += AD_THREADS) {
            // mapping 1: k fastest (rows of Rh are contiguous in k)
            {
                const int kk = e % AD_KC, col = e / AD_KC, k = k0 + kk;
                if (k < a.nb) {
                    const int v = v0 + col;
                    sA[kk * AD_T + col] = (v < a.nv) ? Rf[(long long)v * a.ldb + k] : make_float2(0.f, 0.f);
                } else if (RECIP && k < K) {
                    const int r = r0 + col;
                    sB[kk * AD_T + col] = (r < a.nr) ? Rf[(long long)r * a.ldb + (k - a.nb)] : make_float2(0.f, 0.f);
                }
            }
            // mapping 2: column fastest (rows of Dh are contiguous in r / v)
            {
                const int col = e % AD_T, kk = e / AD_T, k = k0 + kk;
                if (k < a.nb) {
                    const int s = a.idx[k], r = r0 + col;
                    float2 d = make_float2(0.f, 0.f);
                    if (s >= 0 && s < a.ns) {
                        if (r < a.nr) d = cconj(Df[(long long)s * a.ldr + r]);
                    } else if (col == 0) {
                        atomicOr(a.status, 1);
                    }
                    sB[kk * AD_T + col] = d;
                } else if (RECIP && k < K) {
                    const int s = a.idx[k - a.nb], v = v0 + col;
                    float2 d = make_float2(0.f, 0.f);
                    if (s >= 0 && s < a.ns && v < a.nv) d = cconj(Df[(long long)s * a.ldr + v]);
                    sA[kk * AD_T + col] = d;
                } else if (k >= K) {
                    sA[kk * AD_T + col] = make_float2(0.f, 0.f);
                    sB[kk * AD_T + col] = make_float2(0.f, 0.f);
                }
            }
        }
        __syncthreads();
        const int kmax = min(AD_KC, K - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            const float4 *ap = reinterpret_cast<const float4 *>(sA + kk * AD_T + warp * 16);
            float2 av[16];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 p = ap[i];
                av[2 * i] = make_float2(p.x, p.y);
                av[2 * i + 1] = make_float2(p.z, p.w);
            }
            const float2 b0 = sB[kk * AD_T + lane], b1 = sB[kk * AD_T + 32 + lane];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                cmac(acc[i][0], av[i], b0);
                cmac(acc[i][1], av[i], b1);
            }
        }
        __syncthreads();
    }

    float2 *Cf = a.C + (long long)f * a.sCf;
    const bool diag = RECIP && (vb == rb);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int v = v0 + warp * 16 + i;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = r0 + lane + 32 * h;
            const float2 val = cscale(acc[i][h], a.outscale);
            if (v < a.nv && r < a.nr && (!diag || v <= r)) Cf[(long long)v * a.ldr + r] = val;
            if (RECIP) gsm[(lane + 32 * h) * (AD_T + 1) + warp * 16 + i] = val;   // mirror buffer (r, v)
        }
    }
    if (RECIP) {
        // the operand buffers alias the mirror buffer: the K loop ended with a barrier, and the mirror
        // writes above only start after it
        __syncthreads();
        for (int e = tid; e < AD_T * AD_T; e += AD_THREADS) {
            const int rr = e / AD_T, vv = e % AD_T;
            const int r = r0 + rr, v = v0 + vv;
            if (v < a.nv && r < a.nr && (!diag || v < r)) Cf[(long long)r * a.ldr + v] = gsm[rr * (AD_T + 1) + vv];
        }
    }
}

cudaError_t gemm_prepare() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_cgemm_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FW_SMEM))) return e;
    const int adj = (int)(AD_SMEM_MIRROR > AD_SMEM_OPER ? AD_SMEM_MIRROR : AD_SMEM_OPER);
    if ((e = cudaFuncSetAttribute(k_cgemm_adj<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, adj))) return e;
    if ((e = cudaFuncSetAttribute(k_cgemm_adj<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, adj))) return e;
    return cudaSuccess;
}

cudaError_t launch_cgemm_fwd(const GemmArgs &a, int nf, cudaStream_t st) {
    dim3 grid((a.nv + FW_ROWS - 1) / FW_ROWS, (a.nb + FW_NB - 1) / FW_NB, nf);
    k_cgemm_fwd<<<grid, FW_THREADS, FW_SMEM, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cgemm_adj(const GemmArgs &a0, bool recip, int nf, cudaStream_t st) {
    GemmArgs a = a0;
    a.tiles_v = (a.nv + AD_T - 1) / AD_T;
    a.tiles_r = (a.nr + AD_T - 1) / AD_T;
    if (recip) {
        const int ntiles = a.tiles_v * (a.tiles_v + 1) / 2;
        k_cgemm_adj<true><<<dim3(ntiles, nf), AD_THREADS, AD_SMEM_MIRROR, st>>>(a);
    } else {
        k_cgemm_adj<false><<<dim3(a.tiles_v * a.tiles_r, nf), AD_THREADS, AD_SMEM_OPER, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace smdd
