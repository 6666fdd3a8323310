// Device side of the work queues of the many-problem epochs (see WorkQueue in smdd_internal.h).
#pragma once

#include "smdd_internal.h"

namespace smdd {

// Next work item of the CTA (thread 0 takes it, everyone reads it); -1 once the queue is empty.  The
// leading barrier makes the previous item's shared memory free before anything of the next one starts.
__device__ __forceinline__ int queue_next(const WorkQueue &q, int &member, int &tile) {
    __shared__ int s_item;
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(q.counter, 1u);
    __syncthreads();
    const int w = s_item;
    if (w >= q.total) return -1;
    int lo = 0, hi = q.n - 1;   // the member: the largest m with start[m] <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(q.start + mid) <= w) lo = mid;
        else hi = mid - 1;
    }
    member = lo;
    tile = w - __ldg(q.start + lo);
    return w;
}

// The argument record of the current item -> shared memory (the body then reads its fields there, as a
// plain launch reads them from the parameter space); the caller syncs before the body runs.
template <class A>
__device__ __forceinline__ void queue_args(const A *src, A &dst) {
    static_assert(sizeof(A) % 4 == 0, "records are copied in 4-byte words");
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(A) / 4); i += blockDim.x) d[i] = __ldg(s + i);
}

// resident CTAs per SM of a kernel times the SMs, at most `items`
template <class K>
int queue_grid(K kern, int threads, size_t smem, int items) {
    int per_sm = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    const long long g = (long long)(per_sm > 0 ? per_sm : 1) * (nsm > 0 ? nsm : 1);
    return (int)(g < items ? g : (items > 0 ? items : 1));
}

}  // namespace smdd
