// Blackwell (sm_103a) tensor-core building blocks: tcgen05.mma with BF16 operands in 128-byte
// swizzled shared memory and FP32 accumulators in tensor memory (TMEM).
//
// Shared-memory operand layouts (the canonical 128B-swizzle layouts of the UMMA matrix descriptor):
//   K-major tile  [rows][64 k]  : row = 128 B (64 bf16 along K); 16-byte chunk c of row r stored at
//                                 chunk c ^ (r & 7); 8-row groups 1024 B apart (SBO).  A K-step of 16
//                                 advances the descriptor start by 32 B inside the row.
//   MN-major tile [k][64 mn]    : the same with the roles swapped: row = one k, 64 elements along M/N;
//                                 atoms of 64 M/N elements LBO bytes apart, 8-k groups SBO = 1024 B apart.
// Every tile base is 1024-byte aligned.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace smdd {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// UMMA shared-memory matrix descriptor, 128-byte swizzle, descriptor version 1
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// instruction descriptor of tcgen05.mma kind::f16: BF16 x BF16 -> FP32, M x N, operand majors, negate B
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N, int amajor, int bmajor, int negb) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)negb << 14) | ((uint32_t)amajor << 15) |
           ((uint32_t)bmajor << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Wait for the given phase parity of an mbarrier, giving up after `limit` SM clock cycles.
// Returns false on timeout (the caller records the error and finishes without the result).
__device__ __forceinline__ bool mbar_wait_limit(uint64_t *bar, uint32_t parity, long long limit) {
    uint32_t done = 0;
    const long long t0 = clock64();
    while (!done) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (!done && clock64() - t0 > limit) return false;
    }
    return true;
}

// the same with the production limit: about a second of clock
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    return mbar_wait_limit(bar, parity, 2000000000LL);
}

// Announce `bytes` of asynchronous copies on the mbarrier and arrive on it (one thread).
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Tiled copy of one box of a 3D tensor by the tensor memory accelerator into this CTA's shared memory
// (coordinates innermost first; x times the element size a multiple of 16 bytes); completion counted
// on the mbarrier.  tmap: address of a tensor map in the kernel's parameter space.
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const void *tmap, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
            smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Tiled store of one box of a 3D tensor from this CTA's shared memory by the tensor memory accelerator
// (coordinates innermost first, never negative; x times the element size a multiple of 16 bytes; parts
// of the box outside the tensor are not written), as one bulk async-group operation of this thread.
__device__ __forceinline__ void tma_store_3d(const void *tmap, const void *smem_src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
                     reinterpret_cast<uint64_t>(tmap)),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(smem_src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// the shared-memory sources of this thread's committed bulk stores have been read (may be reused)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// this thread's committed bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// TMEM allocation by one full warp; the base address is written to *holder (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(holder)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols));
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + lo with hi = bf16(x), lo = bf16(x - hi): the compensated (split) BF16 representation
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo_elem, __nv_bfloat16 hi_elem) {
    return (uint32_t)__bfloat16_as_ushort(lo_elem) | ((uint32_t)__bfloat16_as_ushort(hi_elem) << 16);
}

// 8 complex values -> one 16-byte chunk in each of the four planes (re hi, re lo, im hi, im lo);
// conj negates the imaginary part first
struct Chunk4 {
    uint4 rh, rl, ih, il;
};
__device__ __forceinline__ Chunk4 split8(const float2 (&z)[8], bool conj) {
    __nv_bfloat16 rh[8], rl[8], ih[8], il[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        split_bf16(z[i].x, rh[i], rl[i]);
        split_bf16(conj ? -z[i].y : z[i].y, ih[i], il[i]);
    }
    Chunk4 c;
    c.rh = make_uint4(pack_bf16x2(rh[0], rh[1]), pack_bf16x2(rh[2], rh[3]), pack_bf16x2(rh[4], rh[5]), pack_bf16x2(rh[6], rh[7]));
    c.rl = make_uint4(pack_bf16x2(rl[0], rl[1]), pack_bf16x2(rl[2], rl[3]), pack_bf16x2(rl[4], rl[5]), pack_bf16x2(rl[6], rl[7]));
    c.ih = make_uint4(pack_bf16x2(ih[0], ih[1]), pack_bf16x2(ih[2], ih[3]), pack_bf16x2(ih[4], ih[5]), pack_bf16x2(ih[6], ih[7]));
    c.il = make_uint4(pack_bf16x2(il[0], il[1]), pack_bf16x2(il[2], il[3]), pack_bf16x2(il[4], il[5]), pack_bf16x2(il[6], il[7]));
    return c;
}

}  // namespace smdd
