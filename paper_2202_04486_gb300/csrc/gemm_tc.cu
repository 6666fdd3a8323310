// Per-frequency complex products on the tensor cores (tcgen05) with split-BF16 operands: the
// mixed-precision form of the batched MMM of Appendix A (Eq. 2 forward, Eq. 6 adjoint).
//
// Every FP32 operand value x is written to shared memory as two BF16 numbers, hi = bf16(x) and
// lo = bf16(x - hi); a real product is x*y ~ hi_x hi_y + hi_x lo_y + lo_x hi_y (the lo*lo term is
// dropped), accumulated in FP32 in tensor memory.  A complex product uses the four real products
// (re*re - im*im, re*im + im*re), the subtraction through the negate-B bit of the instruction
// descriptor.  So each K-step of 16 issues 12 MMAs of M = 128 rows into two accumulators (re, im).
//
// The CUDA threads of a CTA load the FP32 complex spectra (coalesced rows), split them and store the
// four BF16 planes (re hi, re lo, im hi, im lo) in the 128-byte swizzled layouts of tc_common.cuh -- or,
// for the adjoint of a plan that holds them, copy the planes from operand images split once per step
// (k_tc_adj_images); thread 0 issues the MMAs and commits them to an mbarrier; every wait is bounded.
// Status bits: 1 = a source index out of range, 2 = a bounded wait gave up.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "smdd_fft.cuh"
#include "smdd_internal.h"
#include "tc_common.cuh"
#include "work_queue.cuh"

namespace smdd {

constexpr int TC_THREADS = 256;
#ifndef SMDD_TC_FWD_STAGES
#define SMDD_TC_FWD_STAGES 1   // one stage: two CTAs share an SM and hide each other's load latency
#endif
constexpr int TC_FWD_STAGES = SMDD_TC_FWD_STAGES;

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// load 8 consecutive complex values row[k .. k+8), zero past n (row may be null: all zero)
__device__ __forceinline__ void load8(const float2 *row, int k, int n, float2 (&z)[8]) {
    if (row && k + 7 < n) {
        const float4 *p = reinterpret_cast<const float4 *>(row + k);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 v = __ldg(p + i);
            z[2 * i] = make_float2(v.x, v.y);
            z[2 * i + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) z[i] = (row && k + i < n) ? row[k + i] : make_float2(0.f, 0.f);
    }
}

// Row v of a symmetric model's spectra, elements k .. k+8 (zero past n), when only the part on and above
// the TR-block diagonal is stored: element r < lo = TR floor(v / TR) is read at (r, v) (column v of row r).
__device__ __forceinline__ void load8_sym(const float2 *Af, long long ld, int v, int k, int n, int lo, float2 (&z)[8]) {
    if (k >= lo) {
        load8(Af + (long long)v * ld, k, n, z);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = k + i;
            z[i] = r < n ? __ldg(r >= lo ? Af + (long long)v * ld + r : Af + (long long)r * ld + v) : make_float2(0.f, 0.f);
        }
    }
}

// store one 16-byte chunk of each plane; planes are `pstride` bytes apart
__device__ __forceinline__ void store_planes(uint8_t *base, int off, int pstride, const Chunk4 &c) {
    *reinterpret_cast<uint4 *>(base + off) = c.rh;
    *reinterpret_cast<uint4 *>(base + pstride + off) = c.rl;
    *reinterpret_cast<uint4 *>(base + 2 * pstride + off) = c.ih;
    *reinterpret_cast<uint4 *>(base + 3 * pstride + off) = c.il;
}

// 12 MMAs of one K-step: acc_re += Ar Br - Ai Bi, acc_im += Ar Bi + Ai Br, each real product split
// into hi*hi + hi*lo + lo*hi.  a[p], b[p]: descriptors of the planes (re hi, re lo, im hi, im lo).
__device__ __forceinline__ void mma_complex_split(uint32_t d_re, uint32_t d_im, const uint64_t (&a)[4],
                                                  const uint64_t (&b)[4], uint32_t idp, uint32_t idn, uint32_t acc) {
    umma_bf16(d_re, a[0], b[0], idp, acc);
    umma_bf16(d_re, a[0], b[1], idp, 1);
    umma_bf16(d_re, a[1], b[0], idp, 1);
    umma_bf16(d_re, a[2], b[2], idn, 1);
    umma_bf16(d_re, a[2], b[3], idn, 1);
    umma_bf16(d_re, a[3], b[2], idn, 1);
    umma_bf16(d_im, a[0], b[2], idp, acc);
    umma_bf16(d_im, a[0], b[3], idp, 1);
    umma_bf16(d_im, a[1], b[2], idp, 1);
    umma_bf16(d_im, a[2], b[0], idp, 1);
    umma_bf16(d_im, a[2], b[1], idp, 1);
    umma_bf16(d_im, a[3], b[0], idp, 1);
}

// ------------------------------------------------------------------------------------------------
// forward: C[f][v][b] = sum_r A[f][v][r] Dh[f][idx_b][r]   (M = 128 rows v, N = NB batch columns)
// K = nr streamed in chunks of 64 through two shared-memory stages.
// ------------------------------------------------------------------------------------------------
template <int NB, int NSTAGE>
struct TcFwd {
    static constexpr int A_PLANE = 128 * 128;           // bytes per plane per stage
    static constexpr int B_PLANE = NB * 128;
    static constexpr int STAGE = 4 * A_PLANE + 4 * B_PLANE;
    static constexpr size_t SMEM = NSTAGE * (size_t)STAGE + 1024;
    static constexpr uint32_t TMEM_COLS = 2 * NB <= 32 ? 32 : 2 * NB;   // power of two >= 32
};

// Tile (bx, by, bz) = (row block of 128 virtual sources, batch block of NB, bin f).  Q: a work-queue
// item of a persistent CTA, which owns its TMEM (tmem_q) for all its items; the barriers are
// invalidated at the end of the item so that the next one can initialise them again.
template <int NB, int NSTAGE, bool Q, bool SYM = false>
__device__ __forceinline__ void tc_fwd_body(const GemmArgs &a, int bx, int by, int bz, uint32_t tmem_q) {
    using G = TcFwd<NB, NSTAGE>;
    extern __shared__ uint8_t tc_raw[];
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int drows[NB];
    __shared__ int fail, issued;
    uint8_t *sm = align1024(tc_raw);
    const int f = bz, v0 = bx * 128, b0 = by * NB;
    if (a.nf_active > 0 && f >= a.nf_active) {   // above the band limit: zero products, no TMEM
        zero_tile(a.C + (long long)f * a.sCf, a.ldb, v0, 128, b0, NB, a.nv, a.nb);
        return;
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float2 *Af = a.A + (long long)f * a.sAf;
    const float2 *Df = a.Dh + (long long)f * a.sDf;

    for (int j = tid; j < NB; j += TC_THREADS) {
        int s = -1;
        if (b0 + j < a.nb) {
            s = a.idx[b0 + j];
            if (s < 0 || s >= a.ns) {
                atomicOr(a.status, 1);
                s = -1;
            }
        }
        drows[j] = s;
    }
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fail = 0;
        issued = 0;
        fence_mbar_init();
    }
    if (!Q && warp == 0) tmem_alloc(&tmem_holder, G::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = Q ? tmem_q : tmem_holder;
    constexpr uint32_t idp = umma_idesc(128, NB, 0, 0, 0), idn = umma_idesc(128, NB, 0, 0, 1);
    // failure-path check: before any copy or product, wait on a barrier that nothing arrives on (phase
    // 0 of bars[1] never completes here) for a short limit, then take the timeout path below
    if (a.wait_probe > 0) {
        if (tid == 0 && !mbar_wait_limit(&bars[1], 0, a.wait_probe)) fail = 1;
        __syncthreads();
    }

    const int nk = fail ? 0 : (a.nr + 63) / 64;
    for (int kc = 0; kc < nk; ++kc) {
        const int s = kc % NSTAGE;
        uint8_t *st = sm + s * G::STAGE;
        // model spectra rows: 128 rows x 8 chunks of 8 complex; every load of the chunk is issued
        // before the first split, so their latencies overlap, and before the wait for the stage, so
        // they also overlap the MMAs of the previous chunk
        {
            constexpr int UA = 128 * 8 / TC_THREADS;
            float2 z[UA][8];
#pragma unroll
            for (int i = 0; i < UA; ++i) {
                const int u = tid + i * TC_THREADS, row = u >> 3, c = u & 7, v = v0 + row;
                if (SYM && v < a.nv)
                    load8_sym(Af, a.ldr, v, kc * 64 + 8 * c, a.nr, a.sym_tr * (v / a.sym_tr), z[i]);
                else
                    load8(v < a.nv ? Af + (long long)v * a.ldr : nullptr, kc * 64 + 8 * c, a.nr, z[i]);
            }
            // stage s is free again once the MMAs of chunk kc - NSTAGE (the previous use of bars[s]) are done
            if (kc >= NSTAGE && !mbar_wait_bounded(&bars[s], ((kc - NSTAGE) / NSTAGE) & 1)) fail = 1;
#pragma unroll
            for (int i = 0; i < UA; ++i) {
                const int u = tid + i * TC_THREADS, row = u >> 3, c = u & 7;
                store_planes(st, row * 128 + ((c ^ (row & 7)) << 4), G::A_PLANE, split8(z[i], false));
            }
        }
        // gathered kernel rows of the batch
        for (int u = tid; u < NB * 8; u += TC_THREADS) {
            const int row = u >> 3, c = u & 7, srow = drows[row];
            float2 z[8];
            load8(srow >= 0 ? Df + (long long)srow * a.ldr : nullptr, kc * 64 + 8 * c, a.nr, z);
            store_planes(st + 4 * G::A_PLANE, row * 128 + ((c ^ (row & 7)) << 4), G::B_PLANE, split8(z, false));
        }
        fence_async_smem();
        __syncthreads();
        if (fail) break;
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint64_t ad[4], bd[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    ad[p] = umma_desc(smem_u32(st + p * G::A_PLANE + ks * 32), 16, 1024);
                    bd[p] = umma_desc(smem_u32(st + 4 * G::A_PLANE + p * G::B_PLANE + ks * 32), 16, 1024);
                }
                mma_complex_split(tmem, tmem + NB, ad, bd, idp, idn, (kc > 0 || ks > 0) ? 1u : 0u);
            }
            umma_commit(&bars[s]);
            issued = 1;
        }
    }
    const int last = nk - 1;
    if (!fail && !mbar_wait_bounded(&bars[last % NSTAGE], (last / NSTAGE) & 1)) fail = 1;
    __syncthreads();
    const bool ok = !fail;
    // after a timeout, give products still in flight one more bounded wait before TMEM is freed
    if (!ok && issued) mbar_wait_bounded(&bars[last % NSTAGE], (last / NSTAGE) & 1);
    tc_fence_after();
    __syncthreads();
    // epilogue: TMEM -> shared staging [128][NB] complex -> coalesced rows of C
    float2 *out = reinterpret_cast<float2 *>(sm);
    if (ok && warp < 4) {
        const int row = 32 * warp + lane;
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += 16) {
            float re[16], im[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, re);
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + NB + c0, im);
#pragma unroll
            for (int j = 0; j < 16; ++j) out[row * (NB + 1) + c0 + j] = make_float2(re[j], im[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (ok) {
        float2 *Cf = a.C + (long long)f * a.sCf;
        for (int e = tid; e < 128 * NB; e += TC_THREADS) {
            const int row = e / NB, j = e % NB, v = v0 + row, b = b0 + j;
            if (v < a.nv && b < a.nb) Cf[(long long)v * a.ldb + b] = out[row * (NB + 1) + j];
        }
    } else if (tid == 0) {
        atomicOr(a.status, 2);
    }
    if constexpr (Q) {
        __syncthreads();   // every wait on the barriers of this item is over
        if (tid == 0) {
            mbar_inval(&bars[0]);
            mbar_inval(&bars[1]);
        }
    } else {
        if (warp == 0) tmem_dealloc(tmem, G::TMEM_COLS);
    }
}

// SYM: the model spectra hold a symmetric model on and above the a.sym_tr-block diagonal only (load8_sym)
template <int NB, int NSTAGE, bool SYM = false>
__global__ void __launch_bounds__(TC_THREADS, NSTAGE == 1 ? 2 : 1) k_tc_fwd(GemmArgs a) {
    tc_fwd_body<NB, NSTAGE, false, SYM>(a, blockIdx.x, blockIdx.y, blockIdx.z, 0);
}

// work-queue form: persistent CTAs (TMEM allocated once) taking (problem, tile) items; tile t of a
// problem is (bx, by, bz) with t = (bz gy + by) gx + bx, gx = ceil(nv / 128), gy = ceil(nb / NB)
template <int NB>
__global__ void __launch_bounds__(TC_THREADS, 2) k_tc_fwd_q(WorkQueue q) {
    using G = TcFwd<NB, 1>;
    __shared__ uint32_t holder;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tmem_alloc(&holder, G::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = holder;
    const GemmArgs *args = static_cast<const GemmArgs *>(q.args);
    int m = 0, tile = 0;
    __shared__ GemmArgs sa;
    while (queue_next(q, m, tile) >= 0) {
        queue_args(args + m, sa);
        __syncthreads();
        const GemmArgs &a = sa;
        const int gx = (a.nv + 127) / 128, gy = (a.nb + NB - 1) / NB;
        const int bx = tile % gx, r = tile / gx;
        tc_fwd_body<NB, 1, true>(a, bx, r % gy, r / gy, tmem);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, G::TMEM_COLS);
}

// ------------------------------------------------------------------------------------------------
// adjoint: C[f][v][r] = outscale * sum_k A'[v][k] B'[k][r] on 128 x 128 tiles, K = nb in chunks of 32:
//   first half  A' = Rh[f][v][b],                 B' = conj(Dh[f][idx_b][r])
//   second half A' = conj(Dh[f][idx_b][v]),       B' = Rh[f][r][b]          (reciprocity)
// Both operands are stored MN-major (rows k, 128 contiguous m / n), so every plane is 32 x 256 bytes:
// the kernel rows of Dh are MN-major as loaded, and the residual rows (b contiguous in HBM) are copied
// by cp.async into a staging tile and transposed while they are split.  About 100 KB of shared memory:
// two CTAs share an SM, one CTA's epilogue overlapping the other's loads and products; the loads of
// the next chunk are issued before the wait for the previous chunk's products.
// With reciprocity only the upper-triangular tiles run and the transposed tile is mirrored.
// ------------------------------------------------------------------------------------------------
struct TcAdj {
    static constexpr int KC = 32;                       // K chunk
    static constexpr int PLANE = 2 * KC * 128;          // bytes: 2 atoms of 64 m/n x KC rows x 128 B
    static constexpr int OPER = 8 * PLANE;              // A' and B' planes (64 KB)
    static constexpr int SLD = KC + 2;                  // staging row pitch in float2 (16-byte multiple)
    static constexpr int STAGE = 128 * SLD * 8;         // residual staging tile (34 KB)
    static constexpr int OUT = 128 * 65 * 8;            // epilogue staging: 64 columns per pass
    static constexpr size_t BODY = (size_t)OPER + STAGE;
    static constexpr size_t SMEM = (BODY > OUT ? BODY : OUT) + 1024;
    static constexpr uint32_t TMEM_COLS = 256;
};

__device__ __forceinline__ void cp_async16_zfill(void *smem_dst, const void *gsrc, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Operand images: per bin f and K chunk kc, for every 128-wide block of the virtual sources (R, from the
// residual spectra) and of the receivers (D, from the conjugated kernel rows of the batch), the four
// split-BF16 planes exactly as the tile kernel's shared memory holds them (MN-major, 128-byte swizzle):
// R image of block b at [f][kc][b], D image of block b at [f][kc][tiles_v + b], TC_ADJ_IMG bytes each.
// The adjoint then copies two images per half instead of loading, transposing and splitting its operands
// (every operand block serves a whole row or column of output tiles).
constexpr int TC_ADJ_IMG = 4 * TcAdj::PLANE;

__global__ void __launch_bounds__(TC_THREADS) k_tc_adj_images(GemmArgs a, uint8_t *img) {
    using G = TcAdj;
    constexpr int KC = G::KC;
    extern __shared__ __align__(16) float2 stg[];   // residual staging [128][SLD]
    __shared__ int sidx[KC];
    const int blk = blockIdx.x, kc = blockIdx.y, f = blockIdx.z, tid = threadIdx.x;
    const int k0 = kc * KC, kn = min(KC, a.nb - k0);
    const int nbl = a.tiles_v + a.tiles_r;
    uint8_t *dst = img + (((long long)f * a.img_nkc + kc) * nbl + blk) * (long long)TC_ADJ_IMG;
    if (blk < a.tiles_v) {
        // R image: residual rows cr .. cr + 127 (b contiguous), staged, then transposed and split
        const int cr = blk * 128;
        const float2 *Rf = a.A + (long long)f * a.sAf;
        for (int u = tid; u < 128 * (KC / 2); u += TC_THREADS) {
            const int row = u / (KC / 2), pr = u % (KC / 2), k = k0 + 2 * pr, rr = cr + row;
            int bytes = 0;
            const float2 *src = Rf;
            if (rr < a.nv && k < a.nb) {
                bytes = (k + 1 < a.nb) ? 16 : 8;
                src = Rf + (long long)rr * a.ldb + k;
            }
            cp_async16_zfill(stg + row * G::SLD + 2 * pr, src, bytes);
        }
        cp_async_commit_wait_all();
        __syncthreads();
        for (int u = tid; u < KC * 16; u += TC_THREADS) {
            const int k = u % KC, ch = u / KC, at = ch >> 3, c = ch & 7;
            float2 z[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) z[j] = stg[(64 * at + 8 * c + j) * G::SLD + k];
            store_planes(dst, at * (KC * 128) + k * 128 + ((c ^ (k & 7)) << 4), G::PLANE, split8(z, false));
        }
    } else {
        // D image: conjugated kernel rows of the batch entries k0 .. k0 + 31, receivers cd .. cd + 127
        const int cd = (blk - a.tiles_v) * 128;
        if (tid < KC) {
            int sr = -1;
            if (tid < kn) {
                sr = a.idx[k0 + tid];
                if (sr < 0 || sr >= a.ns) {
                    atomicOr(a.status, 1);
                    sr = -1;
                }
            }
            sidx[tid] = sr;
        }
        __syncthreads();
        const float2 *Df = a.Dh + (long long)f * a.sDf;
        for (int u = tid; u < KC * 16; u += TC_THREADS) {
            const int k = u >> 4, ch = u & 15, at = ch >> 3, c = ch & 7;
            const int srow = sidx[k];
            float2 z[8];
            load8(srow >= 0 ? Df + (long long)srow * a.ldr : nullptr, cd + 64 * at + 8 * c, a.nr, z);
            store_planes(dst, at * (KC * 128) + k * 128 + ((c ^ (k & 7)) << 4), G::PLANE, split8(z, true));
        }
    }
}

// Tile bx of bin by (the upper-triangular enumeration with reciprocity); Q as for tc_fwd_body.  IMG: the
// operands come from the images of k_tc_adj_images (a.img).
template <bool RECIP, bool Q, bool TMA = false, bool IMG = false>
__device__ __forceinline__ void tc_adj_body(const GemmArgs &a, int bx, int by, uint32_t tmem_q,
                                            const CUtensorMap *tmap = nullptr) {
    using G = TcAdj;
    constexpr int KC = G::KC;
    extern __shared__ uint8_t tc_raw[];
    __shared__ uint64_t bar, probe_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ int sidx[1024];
    __shared__ int fail, issued;
    uint8_t *sm = align1024(tc_raw);
    uint8_t *sA = sm, *sB = sm + 4 * G::PLANE;
    float2 *stg = reinterpret_cast<float2 *>(sm + G::OPER);
    const int f = by;
    int vb, rb;
    if (RECIP) {
        int t = bx, row = 0, len = a.tiles_v;
        while (t >= len) { t -= len; ++row; --len; }
        vb = row;
        rb = row + t;
    } else {
        vb = bx / a.tiles_r;
        rb = bx % a.tiles_r;
    }
    const int v0 = vb * 128, r0 = rb * 128;
    if (a.nf_active > 0 && f >= a.nf_active) {   // above the band limit: zero products, no TMEM
        zero_tile(a.C + (long long)f * a.sCf, a.ldr, v0, 128, r0, 128, a.nv, a.nr);
        if (RECIP) zero_tile(a.C + (long long)f * a.sCf, a.ldr, r0, 128, v0, 128, a.nr, a.nv);
        return;
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float2 *Rf = a.A + (long long)f * a.sAf;
    const float2 *Df = a.Dh + (long long)f * a.sDf;

    if constexpr (!IMG) {
        for (int b = tid; b < a.nb; b += TC_THREADS) {
            int s = a.idx[b];
            if (s < 0 || s >= a.ns) {
                atomicOr(a.status, 1);
                s = -1;
            }
            sidx[b] = s;
        }
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init(&probe_bar, 1);
        fail = 0;
        issued = 0;
        fence_mbar_init();
    }
    if (!Q && warp == 0) tmem_alloc(&tmem_holder, G::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = Q ? tmem_q : tmem_holder;
    constexpr uint32_t idp = umma_idesc(128, 128, 1, 1, 0), idn = umma_idesc(128, 128, 1, 1, 1);
    // failure-path check: before any copy or product, wait on a barrier that nothing arrives on for a
    // short limit, then take the timeout path below
    if (a.wait_probe > 0) {
        if (tid == 0 && !mbar_wait_limit(&probe_bar, 0, a.wait_probe)) fail = 1;
        __syncthreads();
    }

    const int nkc = (a.nb + KC - 1) / KC;
    const int nhalf = RECIP ? 2 : 1;
    const int njobs = fail ? 0 : nkc * nhalf;
    constexpr int UD = KC * 16 / TC_THREADS;            // kernel-row units (8 complex) per thread
    int phase = 0;
    for (int job = 0; job < njobs; ++job) {
        const int kc = job / nhalf, half = job % nhalf;
        const int k0 = kc * KC;
        const int kn = min(KC, a.nb - k0), kpad = (kn + 15) & ~15;
        if constexpr (IMG) {
            // the previous products must be done reading the planes
            if (job > 0) {
                if (!mbar_wait_bounded(&bar, phase & 1)) fail = 1;
                ++phase;
            }
            tc_fence_after();
            // half 0: A' = R image of the row block, B' = D image of the column block; half 1 the other way
            const int nbl = a.tiles_v + a.tiles_r;
            const uint8_t *base = a.img + ((long long)f * a.img_nkc + kc) * nbl * (long long)TC_ADJ_IMG;
            const uint8_t *ia = base + (long long)(half ? a.tiles_v + vb : vb) * TC_ADJ_IMG;
            const uint8_t *ib = base + (long long)(half ? rb : a.tiles_v + rb) * TC_ADJ_IMG;
            for (int u = tid; u < TC_ADJ_IMG / 16; u += TC_THREADS) {
                cp_async16_zfill(sA + 16 * u, ia + 16 * u, 16);
                cp_async16_zfill(sB + 16 * u, ib + 16 * u, 16);
            }
            cp_async_commit_wait_all();
            fence_async_smem();
            __syncthreads();
        } else {
        const int cr = half ? r0 : v0, ncr = half ? a.nr : a.nv;   // residual rows of this half
        const int cd = half ? v0 : r0, ncd = half ? a.nv : a.nr;   // kernel-row columns of this half
        // residual rows -> staging (cp.async, zero-filled past the matrix); the staging tile was
        // released by the __syncthreads before the previous job's products
        for (int u = tid; u < 128 * (KC / 2); u += TC_THREADS) {
            const int row = u / (KC / 2), pr = u % (KC / 2), k = k0 + 2 * pr, rr = cr + row;
            int bytes = 0;
            const float2 *src = Rf;
            if (rr < ncr && k < a.nb) {
                bytes = (k + 1 < a.nb) ? 16 : 8;
                src = Rf + (long long)rr * a.ldb + k;
            }
            cp_async16_zfill(stg + row * G::SLD + 2 * pr, src, bytes);
        }
        // kernel rows (MN-major operand) -> registers
        float2 zd[UD][8];
#pragma unroll
        for (int i = 0; i < UD; ++i) {
            const int u = tid + i * TC_THREADS, k = u >> 4, ch = u & 15, at = ch >> 3, c = ch & 7;
            const int srow = (k < kn) ? sidx[k0 + k] : -1;
            load8(srow >= 0 ? Df + (long long)srow * a.ldr : nullptr, cd + 64 * at + 8 * c, ncd, zd[i]);
        }
        // the previous products must be done reading the planes
        if (job > 0) {
            if (!mbar_wait_bounded(&bar, phase & 1)) fail = 1;
            ++phase;
        }
        tc_fence_after();
        uint8_t *pD = half ? sA : sB, *pR = half ? sB : sA;
#pragma unroll
        for (int i = 0; i < UD; ++i) {
            const int u = tid + i * TC_THREADS, k = u >> 4, ch = u & 15, at = ch >> 3, c = ch & 7;
            store_planes(pD, at * (KC * 128) + k * 128 + ((c ^ (k & 7)) << 4), G::PLANE, split8(zd[i], true));
        }
        cp_async_commit_wait_all();
        __syncthreads();
        // staging -> transposed, split residual planes: thread (k, chunk) takes 8 consecutive rows
        for (int u = tid; u < KC * 16; u += TC_THREADS) {
            const int k = u % KC, ch = u / KC, at = ch >> 3, c = ch & 7;
            float2 z[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) z[j] = stg[(64 * at + 8 * c + j) * G::SLD + k];
            store_planes(pR, at * (KC * 128) + k * 128 + ((c ^ (k & 7)) << 4), G::PLANE, split8(z, false));
        }
        fence_async_smem();
        __syncthreads();
        }
        if (fail) break;
        if (tid == 0) {
            tc_fence_after();
            for (int ks = 0; ks < kpad / 16; ++ks) {
                uint64_t ad[4], bd[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    ad[p] = umma_desc(smem_u32(sA + p * G::PLANE + ks * 16 * 128), KC * 128, 1024);
                    bd[p] = umma_desc(smem_u32(sB + p * G::PLANE + ks * 16 * 128), KC * 128, 1024);
                }
                mma_complex_split(tmem, tmem + 128, ad, bd, idp, idn, (job > 0 || ks > 0) ? 1u : 0u);
            }
            umma_commit(&bar);
            issued = 1;
        }
    }
    if (!fail && !mbar_wait_bounded(&bar, phase & 1)) fail = 1;
    __syncthreads();
    const bool ok = !fail;
    // after a timeout, give products still in flight one more bounded wait before TMEM is freed
    if (!ok && issued) mbar_wait_bounded(&bar, phase & 1);
    tc_fence_after();
    // epilogue by the tensor memory accelerator for a tile written once (no reciprocity, or an off-diagonal
    // tile of a symmetric model's adjoint, whose mirror is not needed), in two passes of 64 columns: TMEM ->
    // four staged boxes of 16 complex x 128 rows (128-byte swizzle: granule g of row m at g ^ (m % 8)) ->
    // four tiled stores of the tensor map of C (clipped at nv and nr)
    if (TMA && (!RECIP || (a.no_mirror && vb != rb))) {
        for (int pass = 0; pass < 2; ++pass) {
            if (ok) {
                const int q = warp & 3, hc = warp >> 2;   // lanes 32q.., columns 32hc.. of this pass
                const int row = 32 * q + lane;
#pragma unroll
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    const int col = 64 * pass + 32 * hc + c0;
                    float re[16], im[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + col, re);
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 128 + col, im);
                    uint8_t *box = sm + ((32 * hc + c0) >> 4) * (128 * 128) + row * 128;
#pragma unroll
                    for (int g = 0; g < 8; ++g)
                        *reinterpret_cast<float4 *>(box + ((g ^ (row & 7)) << 4)) =
                            make_float4(re[2 * g] * a.outscale, im[2 * g] * a.outscale, re[2 * g + 1] * a.outscale,
                                        im[2 * g + 1] * a.outscale);
                }
            }
            fence_async_smem();   // the staged boxes are visible to the tensor memory accelerator
            tc_fence_before();
            __syncthreads();
            if (ok && tid == 0) {
#pragma unroll
                for (int b4 = 0; b4 < 4; ++b4) {
                    const int r = r0 + 64 * pass + 16 * b4;
                    if (r < a.nr) tma_store_3d(tmap, sm + b4 * (128 * 128), 2 * r, v0, f);
                }
                bulk_commit();
                bulk_wait_read();   // the staging may be written again
            }
            __syncthreads();
        }
        if (ok && tid == 0) bulk_wait_all();
        if (!ok && tid == 0) atomicOr(a.status, 2);
        if constexpr (Q) {
            if (tid == 0) {
                mbar_inval(&bar);
                mbar_inval(&probe_bar);
            }
        } else {
            if (warp == 0) tmem_dealloc(tmem, G::TMEM_COLS);
        }
        return;
    }
    // epilogue in two passes of 64 columns: TMEM -> shared staging [128][65] -> coalesced rows (and
    // the mirror)
    float2 *out = reinterpret_cast<float2 *>(sm);
    float2 *Cf = a.C + (long long)f * a.sCf;
    const bool diag = RECIP && vb == rb;
    for (int pass = 0; pass < 2; ++pass) {
        if (ok) {
            const int q = warp & 3, hc = warp >> 2;   // lanes 32q.., columns 32hc.. of this pass
            const int row = 32 * q + lane;
#pragma unroll
            for (int c0 = 0; c0 < 32; c0 += 16) {
                const int col = 64 * pass + 32 * hc + c0;
                float re[16], im[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + col, re);
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 128 + col, im);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    out[row * 65 + 32 * hc + c0 + j] = make_float2(re[j] * a.outscale, im[j] * a.outscale);
            }
        }
        tc_fence_before();
        __syncthreads();
        if (ok) {
            const int rp = r0 + 64 * pass;
            for (int e = tid; e < 128 * 64; e += TC_THREADS) {
                const int row = e >> 6, col = e & 63, v = v0 + row, r = rp + col;
                if (v < a.nv && r < a.nr && (!diag || v <= r)) Cf[(long long)v * a.ldr + r] = out[row * 65 + col];
            }
            // the mirror (diagonal tiles always: their lower half is read by the update of a symmetric model)
            if (RECIP && (diag || !a.no_mirror)) {
                for (int e = tid; e < 128 * 64; e += TC_THREADS) {
                    const int rr = e >> 7, vv = e & 127, v = v0 + vv, r = rp + rr;
                    if (v < a.nv && r < a.nr && (!diag || v < r)) Cf[(long long)r * a.ldr + v] = out[vv * 65 + rr];
                }
            }
        }
        __syncthreads();
    }
    if (!ok && tid == 0) atomicOr(a.status, 2);
    if constexpr (Q) {
        // the last loop iteration ended with a barrier after every wait: the barriers are free
        if (tid == 0) {
            mbar_inval(&bar);
            mbar_inval(&probe_bar);
        }
    } else {
        if (warp == 0) tmem_dealloc(tmem, G::TMEM_COLS);
    }
}

template <bool RECIP, bool IMG = false>
__global__ void __launch_bounds__(TC_THREADS, 2) k_tc_adj(GemmArgs a) {
    tc_adj_body<RECIP, false, false, IMG>(a, blockIdx.x, blockIdx.y, 0);
}

// the adjoint without reciprocity with its tile written by the tensor memory accelerator (tmap: the
// tensor map of the gradient spectra, i.e. of the model-spectra buffer, FP32 [nf][nv][2 nr])
template <bool IMG = false>
__global__ void __launch_bounds__(TC_THREADS, 2) k_tc_adj_tma(GemmArgs a, const __grid_constant__ CUtensorMap tmap) {
    tc_adj_body<false, false, true, IMG>(a, blockIdx.x, blockIdx.y, 0, &tmap);
}

// the adjoint of a symmetric model (reciprocity, a.no_mirror): off-diagonal tiles written by the tensor memory
// accelerator, diagonal tiles with their mirror by the threads
template <bool IMG = false>
__global__ void __launch_bounds__(TC_THREADS, 2) k_tc_adj_sym_tma(GemmArgs a, const __grid_constant__ CUtensorMap tmap) {
    tc_adj_body<true, false, true, IMG>(a, blockIdx.x, blockIdx.y, 0, &tmap);
}

// work-queue form: tile t of a problem is (bx, by) = (t % tiles, t / tiles) with tiles the output tiles
// of one bin (the upper triangle with reciprocity); tiles_v / tiles_r are set in the argument records
template <bool RECIP>
__global__ void __launch_bounds__(TC_THREADS, 2) k_tc_adj_q(WorkQueue q) {
    __shared__ uint32_t holder;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tmem_alloc(&holder, TcAdj::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = holder;
    const GemmArgs *args = static_cast<const GemmArgs *>(q.args);
    int m = 0, tile = 0;
    __shared__ GemmArgs sa;
    while (queue_next(q, m, tile) >= 0) {
        queue_args(args + m, sa);
        __syncthreads();
        const GemmArgs &a = sa;
        const int tiles = RECIP ? a.tiles_v * (a.tiles_v + 1) / 2 : a.tiles_v * a.tiles_r;
        tc_adj_body<RECIP, true>(a, tile % tiles, tile / tiles, tmem);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TcAdj::TMEM_COLS);
}

// ------------------------------------------------------------------------------------------------
// forward, streamed: the product of k_tc_fwd by a persistent, warp-specialised kernel, one CTA per SM.
// A CTA walks its tiles (f, 128 rows v, NB batch columns) chunk by chunk (64 of K = nr).
//  * control warp (warp 16, one lane): issues four tiled copies of the tensor memory accelerator per
//    chunk (boxes of 128 rows x 16 complex, 128-byte swizzled, zero-filled past nv and nr) into one of
//    two staging buffers, and the MMAs of each half chunk (K = 32) once the split warps report its
//    planes written;
//  * split warps (0-15): convert the staged FP32 spectra and the gathered kernel rows (loaded into
//    registers one chunk ahead) to the BF16 hi/lo planes, half by half, so the products of one half
//    run while the other half is split; at the end of a tile they read the accumulators from TMEM and
//    write the rows of C directly (16 consecutive complex per thread).
// The warps meet only on mbarriers (full: copies landed; ready: planes of a half written, one arrive
// per split warp; done: products of a half finished), every wait bounded.  Tiles are numbered
// t = (f * gy + batch tile) * gx + v tile; the CTA takes t = blockIdx.x, blockIdx.x + gridDim.x, ...;
// tiles of bins above the band limit are zero-filled first.
// ------------------------------------------------------------------------------------------------
constexpr int TCS_SPLIT = 512;                 // split warps 0-15
constexpr int TCS_THREADS = TCS_SPLIT + 32;    // + the control warp

template <int NB>
struct TcFwdS {
    static constexpr int A_PLANE = 128 * 128;
    static constexpr int B_PLANE = NB * 128;
    static constexpr int PLANES = 4 * A_PLANE + 4 * B_PLANE;
    static constexpr int BOX = 128 * 128;                  // one box: 128 rows x 16 complex FP32
    static constexpr int STG = 4 * BOX;                    // one chunk
    static constexpr size_t SMEM = PLANES + 2 * (size_t)STG + 1024;
    static constexpr uint32_t TMEM_COLS = 2 * NB <= 32 ? 32 : 2 * NB;
    static_assert(PLANES % 1024 == 0, "staging boxes must stay 1024-byte aligned");
    static_assert(NB * 4 <= TCS_SPLIT, "one kernel-row unit per split thread and half chunk");
};

struct FwdTile {
    int f, v0, b0;
};
template <int NB>
__device__ __forceinline__ FwdTile fwd_tile(int t, int gx, int gy) {
    const int vt = t % gx, r = t / gx;
    return FwdTile{r / gy, vt * 128, (r % gy) * NB};
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

template <int NB>
__global__ void __launch_bounds__(TCS_THREADS, 1)
    k_tc_fwd_stream(GemmArgs a, const __grid_constant__ CUtensorMap tmap, int gx, int gy, int n_active, int n_tiles) {
    using G = TcFwdS<NB>;
    extern __shared__ uint8_t tc_raw[];
    __shared__ uint64_t full[2];    // copies into staging buffer 0 / 1 landed
    __shared__ uint64_t ready[2];   // planes of half 0 / 1 written (one arrive per split warp)
    __shared__ uint64_t done[2];    // products of half 0 / 1 finished
    __shared__ uint32_t tmem_holder;
    __shared__ int fail, s_issued, s_last[2];
    uint8_t *planes = align1024(tc_raw);
    uint8_t *stg0 = planes + G::PLANES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int t = n_active + blockIdx.x; t < n_tiles; t += gridDim.x) {   // above the band limit
        const FwdTile T = fwd_tile<NB>(t, gx, gy);
        zero_tile(a.C + (long long)T.f * a.sCf, a.ldb, T.v0, 128, T.b0, NB, a.nv, a.nb);
    }
    const int my_tiles = (int)blockIdx.x < n_active ? (n_active - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (my_tiles == 0) return;
    const int nk = (a.nr + 63) / 64;
    const int nchunks = my_tiles * nk;

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&ready[i], TCS_SPLIT / 32);
            mbar_init(&done[i], 1);
        }
        fail = 0;
        s_issued = 0;
        s_last[0] = s_last[1] = -1;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_holder, G::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;

    if (warp == TCS_SPLIT / 32) {
        // ---------------- control warp ----------------
        if (lane == 0) {
            constexpr uint32_t idp = umma_idesc(128, NB, 0, 0, 0), idn = umma_idesc(128, NB, 0, 0, 1);
            auto issue = [&](int g) {   // four boxes of chunk g into staging buffer g & 1
                const FwdTile T = fwd_tile<NB>((int)blockIdx.x + (g / nk) * (int)gridDim.x, gx, gy);
                const int k0 = (g % nk) * 64;
                uint8_t *stg = stg0 + (g & 1) * G::STG;
                mbar_arrive_expect_tx(&full[g & 1], (uint32_t)G::STG);
#pragma unroll
                for (int j = 0; j < 4; ++j) tma_load_3d(stg + j * G::BOX, &tmap, 2 * k0 + 32 * j, T.v0, T.f, &full[g & 1]);
                s_issued = g + 1;
            };
            issue(0);
            if (nchunks > 1) issue(1);
            for (int g = 0; g < nchunks; ++g) {
                const int kc = g % nk;
                for (int h = 0; h < 2; ++h) {
                    if (!mbar_wait_bounded(&ready[h], g & 1)) {
                        fail = 1;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int k2 = 0; k2 < 2; ++k2) {
                        const int ks = 2 * h + k2;
                        uint64_t ad[4], bd[4];
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            ad[p] = umma_desc(smem_u32(planes + p * G::A_PLANE + ks * 32), 16, 1024);
                            bd[p] = umma_desc(smem_u32(planes + 4 * G::A_PLANE + p * G::B_PLANE + ks * 32), 16, 1024);
                        }
                        mma_complex_split(tmem, tmem + NB, ad, bd, idp, idn, (kc > 0 || ks > 0) ? 1u : 0u);
                    }
                    umma_commit(&done[h]);
                    s_last[h] = g;
                }
                if (*(volatile int *)&fail) break;
                if (g + 2 < nchunks) issue(g + 2);   // staging buffer g & 1: both halves split
            }
        }
    } else {
        // ---------------- split warps ----------------
        auto load_b = [&](int g, float2 (&zb)[2][8]) {
            // thread u < 4 NB: kernel row u / 4, 8 complex at columns 8 (4h + u % 4) of halves h = 0, 1
            // (an index out of range sets status bit 1 and gives a zero row)
            if (tid >= NB * 4) return;
            const FwdTile T = fwd_tile<NB>((int)blockIdx.x + (g / nk) * (int)gridDim.x, gx, gy);
            const int k0 = (g % nk) * 64, row = tid >> 2, c = tid & 3, b = T.b0 + row;
            const float2 *Df = a.Dh + (long long)T.f * a.sDf;
            int s = -1;
            if (b < a.nb) {
                s = a.idx[b];
                if (s < 0 || s >= a.ns) {
                    atomicOr(a.status, 1);
                    s = -1;
                }
            }
            const float2 *rowp = s >= 0 ? Df + (long long)s * a.ldr : nullptr;
            load8(rowp, k0 + 8 * c, a.nr, zb[0]);
            load8(rowp, k0 + 32 + 8 * c, a.nr, zb[1]);
        };
        float2 zb[2][8];
        load_b(0, zb);
        for (int g = 0; g < nchunks; ++g) {
            const int kc = g % nk;
            const uint8_t *stg = stg0 + (g & 1) * G::STG;
            if (!mbar_wait_bounded(&full[g & 1], (g >> 1) & 1)) fail = 1;   // chunk g staged
            for (int h = 0; h < 2 && !*(volatile int *)&fail; ++h) {
                if (g > 0 && !mbar_wait_bounded(&done[h], (g - 1) & 1)) {     // bytes of half h free
                    fail = 1;
                    break;
                }
                tc_fence_after();
                // units (row m, 8 complex c), c in 4h .. 4h+3: box c / 2, granules 4 (c % 2) .. +3 of
                // the row, each stored at granule ^ (m % 8)
                const int m = tid & 127, c = 4 * h + (tid >> 7);
                const uint8_t *row = stg + (c >> 1) * G::BOX + m * 128;
                float2 z[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 w = *reinterpret_cast<const float4 *>(row + (((4 * (c & 1) + j) ^ (m & 7)) << 4));
                    z[2 * j] = make_float2(w.x, w.y);
                    z[2 * j + 1] = make_float2(w.z, w.w);
                }
                store_planes(planes, m * 128 + ((c ^ (m & 7)) << 4), G::A_PLANE, split8(z, false));
                if (tid < NB * 4) {
                    const int brow = tid >> 2, bc = 4 * h + (tid & 3);
                    store_planes(planes + 4 * G::A_PLANE, brow * 128 + ((bc ^ (brow & 7)) << 4), G::B_PLANE,
                                 split8(zb[h], false));
                }
                fence_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ready[h]);
            }
            if (*(volatile int *)&fail) break;
            if (g + 1 < nchunks) load_b(g + 1, zb);
            if (kc == nk - 1) {
                // the tile's epilogue: done[1] of this chunk follows every earlier product
                if (!mbar_wait_bounded(&done[1], g & 1)) {
                    fail = 1;
                    break;
                }
                tc_fence_after();
                const FwdTile T = fwd_tile<NB>((int)blockIdx.x + (g / nk) * (int)gridDim.x, gx, gy);
                const int q = warp & 3, cc = warp >> 2;   // TMEM lanes 32q.., columns 16cc..
                if (16 * cc < NB) {
                    const int v = T.v0 + 32 * q + lane, c0 = 16 * cc;
                    float re[16], im[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + c0, re);
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + NB + c0, im);
                    if (v < a.nv) {
                        float2 *Crow = a.C + (long long)T.f * a.sCf + (long long)v * a.ldb + T.b0 + c0;
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (T.b0 + c0 + j < a.nb) Crow[j] = make_float2(re[j], im[j]);
                    }
                }
                tc_fence_before();   // the next tile's first products overwrite the accumulators
            }
        }
    }
    __syncthreads();
    if (fail) {
        // copies and products still in flight get one more bounded wait before the CTA frees TMEM
        // and exits
        if (tid == 0) {
            for (int i = max(0, s_issued - 2); i < s_issued; ++i) mbar_wait_bounded(&full[i & 1], (i >> 1) & 1);
            for (int h = 0; h < 2; ++h)
                if (s_last[h] >= 0) mbar_wait_bounded(&done[h], s_last[h] & 1);
            atomicOr(a.status, 2);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, G::TMEM_COLS);
}

// ------------------------------------------------------------------------------------------------
cudaError_t tc_prepare() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd<16, TC_FWD_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwd<16, TC_FWD_STAGES>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd<32, TC_FWD_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwd<32, TC_FWD_STAGES>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd<64, TC_FWD_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwd<64, TC_FWD_STAGES>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd<16, TC_FWD_STAGES, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwd<16, TC_FWD_STAGES>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd<32, TC_FWD_STAGES, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwd<32, TC_FWD_STAGES>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd<64, TC_FWD_STAGES, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwd<64, TC_FWD_STAGES>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd_stream<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwdS<16>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd_stream<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwdS<32>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd_stream<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwdS<64>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj_sym_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj_sym_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd_q<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwd<16, 1>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd_q<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwd<32, 1>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_fwd_q<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwd<64, 1>::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj_q<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    if ((e = cudaFuncSetAttribute(k_tc_adj_q<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdj::SMEM))) return e;
    return cudaSuccess;
}

cudaError_t launch_tc_fwd(const GemmArgs &a, int nf, cudaStream_t st) {
    const int gx = (a.nv + 127) / 128;
    constexpr int S = TC_FWD_STAGES;
    if (a.sym_tr > 0) {
        if (a.nb <= 16) k_tc_fwd<16, S, true><<<dim3(gx, 1, nf), TC_THREADS, TcFwd<16, S>::SMEM, st>>>(a);
        else if (a.nb <= 32) k_tc_fwd<32, S, true><<<dim3(gx, 1, nf), TC_THREADS, TcFwd<32, S>::SMEM, st>>>(a);
        else k_tc_fwd<64, S, true><<<dim3(gx, (a.nb + 63) / 64, nf), TC_THREADS, TcFwd<64, S>::SMEM, st>>>(a);
        return cudaGetLastError();
    }
    if (a.nb <= 16) k_tc_fwd<16, S><<<dim3(gx, 1, nf), TC_THREADS, TcFwd<16, S>::SMEM, st>>>(a);
    else if (a.nb <= 32) k_tc_fwd<32, S><<<dim3(gx, 1, nf), TC_THREADS, TcFwd<32, S>::SMEM, st>>>(a);
    else k_tc_fwd<64, S><<<dim3(gx, (a.nb + 63) / 64, nf), TC_THREADS, TcFwd<64, S>::SMEM, st>>>(a);
    return cudaGetLastError();
}

// Tensor map of the model spectra [nf][nv][ldr] complex, seen as FP32 [nf][nv][2 nr] (the padding
// column of an odd nr lies outside it): boxes of 32 floats x 128 rows x 1 bin, 128-byte swizzle,
// zero fill outside the tensor.  The encoder is taken from the driver at run time.
cudaError_t tc_encode_fwd_map(void *map_out, const float2 *Xh, int nr, int nv, int ldr, int nf) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)2 * nr, (cuuint64_t)nv, (cuuint64_t)nf};
    const cuuint64_t strides[2] = {(cuuint64_t)ldr * 8, (cuuint64_t)nv * ldr * 8};
    const cuuint32_t box[3] = {32, 128, 1}, estr[3] = {1, 1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap *>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                              const_cast<float2 *>(Xh), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_tc_fwd_stream(const GemmArgs &a, const void *map, int nf, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    CUtensorMap tmap;
    memcpy(&tmap, map, sizeof(tmap));
    const int gx = (a.nv + 127) / 128;
    const int nb_tile = a.nb <= 16 ? 16 : a.nb <= 32 ? 32 : 64;
    const int gy = (a.nb + nb_tile - 1) / nb_tile;
    const int nf_act = (a.nf_active > 0 && a.nf_active < nf) ? a.nf_active : nf;
    const int n_active = nf_act * gx * gy, n_tiles = nf * gx * gy;
    const int grid = std::max(1, std::min(n_tiles, sms));
    if (nb_tile == 16) k_tc_fwd_stream<16><<<grid, TCS_THREADS, TcFwdS<16>::SMEM, st>>>(a, tmap, gx, gy, n_active, n_tiles);
    else if (nb_tile == 32) k_tc_fwd_stream<32><<<grid, TCS_THREADS, TcFwdS<32>::SMEM, st>>>(a, tmap, gx, gy, n_active, n_tiles);
    else k_tc_fwd_stream<64><<<grid, TCS_THREADS, TcFwdS<64>::SMEM, st>>>(a, tmap, gx, gy, n_active, n_tiles);
    return cudaGetLastError();
}

int tc_fwd_queue_nb(int nb) { return nb <= 16 ? 16 : nb <= 32 ? 32 : 64; }

int tc_fwd_tiles(const GemmArgs &a, int nf) {
    const int NB = tc_fwd_queue_nb(a.nb);
    return ((a.nv + 127) / 128) * ((a.nb + NB - 1) / NB) * nf;
}

int tc_adj_tiles(GemmArgs &a, bool recip, int nf) {
    a.tiles_v = (a.nv + 127) / 128;
    a.tiles_r = (a.nr + 127) / 128;
    return (recip ? a.tiles_v * (a.tiles_v + 1) / 2 : a.tiles_v * a.tiles_r) * nf;
}

cudaError_t launch_tc_fwd_queue(int NB, const WorkQueue &q, cudaStream_t st) {
    if (q.total <= 0) return cudaSuccess;
    if (NB == 16) k_tc_fwd_q<16><<<queue_grid(k_tc_fwd_q<16>, TC_THREADS, TcFwd<16, 1>::SMEM, q.total), TC_THREADS, TcFwd<16, 1>::SMEM, st>>>(q);
    else if (NB == 32) k_tc_fwd_q<32><<<queue_grid(k_tc_fwd_q<32>, TC_THREADS, TcFwd<32, 1>::SMEM, q.total), TC_THREADS, TcFwd<32, 1>::SMEM, st>>>(q);
    else k_tc_fwd_q<64><<<queue_grid(k_tc_fwd_q<64>, TC_THREADS, TcFwd<64, 1>::SMEM, q.total), TC_THREADS, TcFwd<64, 1>::SMEM, st>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_tc_adj_queue(bool recip, const WorkQueue &q, cudaStream_t st) {
    if (q.total <= 0) return cudaSuccess;
    if (recip) k_tc_adj_q<true><<<queue_grid(k_tc_adj_q<true>, TC_THREADS, TcAdj::SMEM, q.total), TC_THREADS, TcAdj::SMEM, st>>>(q);
    else k_tc_adj_q<false><<<queue_grid(k_tc_adj_q<false>, TC_THREADS, TcAdj::SMEM, q.total), TC_THREADS, TcAdj::SMEM, st>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_tc_adj(const GemmArgs &a0, bool recip, int nf, cudaStream_t st, const void *map) {
    GemmArgs a = a0;
    a.tiles_v = (a.nv + 127) / 128;
    a.tiles_r = (a.nr + 127) / 128;
    const bool img = a.img != nullptr;
    if (recip && map && a.no_mirror) {
        CUtensorMap tmap;
        memcpy(&tmap, map, sizeof(tmap));
        const dim3 grid(a.tiles_v * (a.tiles_v + 1) / 2, nf);
        if (img) k_tc_adj_sym_tma<true><<<grid, TC_THREADS, TcAdj::SMEM, st>>>(a, tmap);
        else k_tc_adj_sym_tma<false><<<grid, TC_THREADS, TcAdj::SMEM, st>>>(a, tmap);
    } else if (recip) {
        if (img) k_tc_adj<true, true><<<dim3(a.tiles_v * (a.tiles_v + 1) / 2, nf), TC_THREADS, TcAdj::SMEM, st>>>(a);
        else k_tc_adj<true><<<dim3(a.tiles_v * (a.tiles_v + 1) / 2, nf), TC_THREADS, TcAdj::SMEM, st>>>(a);
    } else if (map) {
        CUtensorMap tmap;
        memcpy(&tmap, map, sizeof(tmap));
        if (img) k_tc_adj_tma<true><<<dim3(a.tiles_v * a.tiles_r, nf), TC_THREADS, TcAdj::SMEM, st>>>(a, tmap);
        else k_tc_adj_tma<false><<<dim3(a.tiles_v * a.tiles_r, nf), TC_THREADS, TcAdj::SMEM, st>>>(a, tmap);
    } else {
        if (img) k_tc_adj<false, true><<<dim3(a.tiles_v * a.tiles_r, nf), TC_THREADS, TcAdj::SMEM, st>>>(a);
        else k_tc_adj<false><<<dim3(a.tiles_v * a.tiles_r, nf), TC_THREADS, TcAdj::SMEM, st>>>(a);
    }
    return cudaGetLastError();
}

size_t tc_adj_image_bytes(int nv, int nr, int nb, int nf) {
    const int nkc = (nb + TcAdj::KC - 1) / TcAdj::KC;
    if (nkc < 1 || nkc > 2) return 0;
    return (size_t)nf * nkc * (size_t)((nv + 127) / 128 + (nr + 127) / 128) * TC_ADJ_IMG;
}

cudaError_t launch_tc_adj_images(const GemmArgs &a0, uint8_t *img, int nf, cudaStream_t st) {
    GemmArgs a = a0;
    a.tiles_v = (a.nv + 127) / 128;
    a.tiles_r = (a.nr + 127) / 128;
    a.img_nkc = (a.nb + TcAdj::KC - 1) / TcAdj::KC;
    const int nfa = (a.nf_active > 0 && a.nf_active < nf) ? a.nf_active : nf;   // bins above a band limit are zero
    k_tc_adj_images<<<dim3(a.tiles_v + a.tiles_r, a.img_nkc, nfa), TC_THREADS, TcAdj::STAGE, st>>>(a, img);
    return cudaGetLastError();
}

}  // namespace smdd
