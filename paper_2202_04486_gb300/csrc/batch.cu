// Many independent MDD problems: whole SGD epochs of every member replayed from one CUDA graph.
//
// One epoch of member m is ceil(ns/nb) SGD steps (Eq. 6 on consecutive slices of a source
// permutation, the last slice partial).  The graph holds, in order:
//   k_epoch_begin  -- for every member, row (e % n_perm) of its permutation table -> its index buffer,
//                     e read from the batch's device epoch counter;
//   the steps      -- MDC_BATCH_BRANCHES: each member's steps in sequence on one of n_branches parallel
//                     branches, as the plan's own launches;
//                     MDC_BATCH_QUEUE: the epoch in waves, wave w holding step w of every member that has
//                     one; every stage of a wave (model transform in wave 0, forward product, residual
//                     step, adjoint product, update) is one launch per kernel family of persistent CTAs
//                     that take (problem, tile) items from a device work queue until it is empty;
//   k_epoch_end    -- the step losses -> row (e % loss_rows) of each member's loss table, then e += 1.
// Only device-side state changes between replays, so the same graph serves every epoch.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "smdd_internal.h"

using namespace smdd;

namespace {

struct EpochSlot {
    const int32_t *perm;   // [n_perm][ns]
    int32_t *cur_idx;      // [ns]: this epoch's order
    const double *cur_loss;// [steps]: written by the residual kernels of this epoch
    double *loss;          // [loss_rows][steps] or null
    int n_perm, ns, steps, loss_rows;
};

__global__ void k_epoch_begin(const EpochSlot *slots, int n, const long long *epoch) {
    const int m = blockIdx.x;
    if (m >= n) return;
    const EpochSlot s = slots[m];
    const long long e = *epoch;
    const int32_t *row = s.perm + (long long)(e % s.n_perm) * s.ns;
    for (int i = threadIdx.x; i < s.ns; i += blockDim.x) s.cur_idx[i] = row[i];
}

// one block: every member's losses, then the counter (after all reads of it in this block)
__global__ void k_epoch_end(const EpochSlot *slots, int n, long long *epoch) {
    const long long e = *epoch;
    for (int m = 0; m < n; ++m) {
        const EpochSlot s = slots[m];
        if (!s.loss) continue;
        double *row = s.loss + (long long)(e % s.loss_rows) * s.steps;
        for (int i = threadIdx.x; i < s.steps; i += blockDim.x) row[i] = s.cur_loss[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) *epoch = e + 1;
}

__global__ void k_set_epoch(long long *epoch, long long v) { *epoch = v; }

double member_cost(const PlanShape &sh, int nb) {
    // per-epoch work estimate used to balance the branches: products + transforms of every step
    const double steps = (sh.ns + nb - 1) / nb;
    const double gemm = 16.0 * nb * sh.nr * (double)sh.nv * sh.nf;
    double lg = 0;
    for (int v = sh.nfft; v > 1; v >>= 1) lg += 1;
    const double fft = 5.0 * sh.nfft * lg * ((double)sh.nr * sh.nv + (double)nb * sh.nv);
    return steps * (gemm + fft);
}

// One launch of the work-queue epoch: stage kind, kernel family, and the queue it drains.
struct QLaunch {
    int kind;            // 0 model transform, 1 forward product, 2 residual, 3 adjoint product, 4 update
    int M, variant;      // trace kernels: FFT length / 2 and variant
    int key;             // forward: batch block NB; adjoint: reciprocity
    std::vector<int> members;
    std::vector<const void *> recs;
    std::vector<int> tiles;
    WorkQueue q;
};

// Group the records of one stage by kernel family into launches (members in order).
void add_stage(std::vector<QLaunch> &out, int kind, const std::vector<int> &ms, const std::vector<StepRecords> &rec) {
    std::vector<QLaunch> stage;
    for (size_t i = 0; i < ms.size(); ++i) {
        const StepRecords &r = rec[i];
        int M = 0, var = 0, key = 0, tiles = 0;
        const void *rp = nullptr;
        switch (kind) {
            case 0: M = r.M; var = r.variant; tiles = r.rfft_tiles; rp = &r.rfft; break;
            case 1: key = r.fwd_nb; tiles = r.fwd_tiles; rp = &r.fwd; break;
            case 2: M = r.M; var = r.variant; tiles = r.resid_tiles; rp = &r.resid; break;
            case 3: key = r.recip ? 1 : 0; tiles = r.adj_tiles; rp = &r.adj; break;
            default: M = r.M; var = r.variant; tiles = r.upd_tiles; rp = &r.upd; break;
        }
        if (tiles <= 0) continue;
        QLaunch *L = nullptr;
        for (auto &x : stage)
            if (x.M == M && x.variant == var && x.key == key) L = &x;
        if (!L) {
            stage.push_back(QLaunch{kind, M, var, key, {}, {}, {}, WorkQueue{}});
            L = &stage.back();
        }
        L->members.push_back(ms[i]);
        L->recs.push_back(rp);
        L->tiles.push_back(tiles);
    }
    for (auto &x : stage) out.push_back(std::move(x));
}

}  // namespace

struct mdc_batch_s {
    int device = 0;
    int n = 0, n_branches = 0, mode = MDC_BATCH_BRANCHES;
    void *queue_mem = nullptr;       // device: argument records, tile prefix sums, queue counters
    std::vector<smdd_member> members;
    std::vector<int> steps;
    EpochSlot *slots = nullptr;      // device [n]
    long long *epoch = nullptr;      // device counter
    std::vector<int32_t *> cur_idx;  // device, per member
    std::vector<double *> cur_loss;  // device, per member
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
};

extern "C" {

int mdc_batch_destroy(mdc_batch_t b) {
    if (!b) return MDC_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto q : b->cur_idx) cudaFree(q);
    for (auto q : b->cur_loss) cudaFree(q);
    cudaFree(b->queue_mem);
    cudaFree(b->slots);
    cudaFree(b->epoch);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    delete b;
    return MDC_OK;
}

int mdc_batch_create(mdc_batch_t *out, const smdd_member *members, int n, int n_branches, void *stream) {
    return mdc_batch_create_ex(out, members, n, MDC_BATCH_BRANCHES, n_branches, stream);
}

int mdc_batch_create_ex(mdc_batch_t *out, const smdd_member *members, int n, int mode, int n_branches, void *stream) {
    if (!out || !members || n < 1) return MDC_ERR_INVALID_ARG;
    if (mode != MDC_BATCH_BRANCHES && mode != MDC_BATCH_QUEUE) return MDC_ERR_INVALID_ARG;
    if (mode == MDC_BATCH_BRANCHES && (n_branches < 1 || n_branches > 64)) return MDC_ERR_INVALID_ARG;
    if (mode == MDC_BATCH_QUEUE) n_branches = 1;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MDC_ERR_CUDA;
    // validation: every member on this device, no plan twice, sizes and flags in range
    std::vector<PlanShape> shapes(n);
    for (int m = 0; m < n; ++m) {
        const smdd_member &mb = members[m];
        if (!mb.plan || !mb.X || !mb.U_obs || !mb.perm || mb.n_perm < 1) return MDC_ERR_INVALID_ARG;
        for (int i = 0; i < 4; ++i)
            if (mb.reserved[i] != 0) return MDC_ERR_INVALID_ARG;
        if (mb.flags & ~(SMDD_RECIPROCITY | SMDD_SYMMETRIC)) return MDC_ERR_INVALID_ARG;
        if (mb.loss && mb.loss_rows < 1) return MDC_ERR_INVALID_ARG;
        shapes[m] = plan_shape(mb.plan);
        if (shapes[m].device != dev) return MDC_ERR_INVALID_ARG;
        if (mb.nb < 1) return MDC_ERR_INVALID_ARG;
        if (mb.nb > shapes[m].nbmax) return MDC_ERR_SHAPE;
        if ((mb.flags & SMDD_RECIPROCITY) && shapes[m].nr != shapes[m].nv) return MDC_ERR_SHAPE;
        for (int q = 0; q < m; ++q)
            if (members[q].plan == mb.plan) return MDC_ERR_INVALID_ARG;
    }
    mdc_batch_s *b = new (std::nothrow) mdc_batch_s();
    if (!b) return MDC_ERR_OOM;
    b->device = dev;
    b->n = n;
    b->mode = mode;
    b->n_branches = std::min(n_branches, n);
    b->members.assign(members, members + n);
    b->steps.resize(n);
    b->cur_idx.assign(n, nullptr);
    b->cur_loss.assign(n, nullptr);
    bool ok = cudaMalloc(&b->slots, n * sizeof(EpochSlot)) == cudaSuccess &&
              cudaMalloc(&b->epoch, sizeof(long long)) == cudaSuccess;
    std::vector<EpochSlot> hs(n);
    for (int m = 0; ok && m < n; ++m) {
        const smdd_member &mb = members[m];
        b->steps[m] = (shapes[m].ns + mb.nb - 1) / mb.nb;
        ok = cudaMalloc(&b->cur_idx[m], shapes[m].ns * sizeof(int32_t)) == cudaSuccess &&
             cudaMalloc(&b->cur_loss[m], b->steps[m] * sizeof(double)) == cudaSuccess;
        hs[m].perm = mb.perm;
        hs[m].cur_idx = b->cur_idx[m];
        hs[m].cur_loss = b->cur_loss[m];
        hs[m].loss = mb.loss;
        hs[m].n_perm = mb.n_perm;
        hs[m].ns = shapes[m].ns;
        hs[m].steps = b->steps[m];
        hs[m].loss_rows = mb.loss ? mb.loss_rows : 1;
    }
    if (!ok) {
        cudaGetLastError();
        mdc_batch_destroy(b);
        return MDC_ERR_OOM;
    }
    int rc = MDC_OK;
    if (cudaMemcpyAsync(b->slots, hs.data(), n * sizeof(EpochSlot), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(b->epoch, 0, sizeof(long long), st) != cudaSuccess)
        rc = MDC_ERR_CUDA;
    for (int m = 0; rc == MDC_OK && m < n; ++m)
        if (cudaMemsetAsync(b->cur_idx[m], 0, shapes[m].ns * sizeof(int32_t), st) != cudaSuccess ||
            cudaMemsetAsync(b->cur_loss[m], 0, b->steps[m] * sizeof(double), st) != cudaSuccess)
            rc = MDC_ERR_CUDA;
    if (rc == MDC_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (rc != MDC_OK) {
        mdc_batch_destroy(b);
        return rc;
    }

    // work-queue epoch: the step records of every wave, grouped into launches, uploaded once
    std::vector<std::vector<StepRecords>> wave_recs;
    std::vector<QLaunch> qlaunches;
    unsigned int *qcounters = nullptr;
    int n_counters = 0;
    if (mode == MDC_BATCH_QUEUE) {
        int maxsteps = 0;
        for (int m = 0; m < n; ++m) maxsteps = std::max(maxsteps, b->steps[m]);
        wave_recs.resize(maxsteps);
        for (int w = 0; rc == MDC_OK && w < maxsteps; ++w) {
            std::vector<int> ms;
            for (int m = 0; m < n; ++m)
                if (b->steps[m] > w) ms.push_back(m);
            wave_recs[w].resize(ms.size());
            for (size_t i = 0; rc == MDC_OK && i < ms.size(); ++i) {
                const int m = ms[i];
                const smdd_member &mb = members[m];
                const int nbs = std::min(mb.nb, shapes[m].ns - w * mb.nb);
                rc = plan_step_records(mb.plan, mb.X, mb.U_obs, b->cur_idx[m] + (long long)w * mb.nb, nbs, mb.alpha,
                                       mb.flags, b->cur_loss[m] + w, &wave_recs[w][i]);
            }
            if (rc != MDC_OK) break;
            if (w == 0) add_stage(qlaunches, 0, ms, wave_recs[w]);
            for (int kind = 1; kind <= 4; ++kind) add_stage(qlaunches, kind, ms, wave_recs[w]);
        }
        // device layout: FftArgs records | GemmArgs records | tile prefix sums | queue counters
        size_t nF = 0, nG = 0, nS = 0;
        for (auto &L : qlaunches) {
            (L.kind == 1 || L.kind == 3 ? nG : nF) += L.members.size();
            nS += L.members.size() + 1;
        }
        n_counters = (int)qlaunches.size();
        auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
        const size_t oF = 0, oG = al(oF + nF * sizeof(FftArgs)), oS = al(oG + nG * sizeof(GemmArgs));
        const size_t oC = al(oS + nS * sizeof(int)), total = al(oC + (size_t)n_counters * sizeof(unsigned int));
        std::vector<unsigned char> host(total, 0);
        if (rc == MDC_OK && cudaMalloc(&b->queue_mem, total) != cudaSuccess) {
            cudaGetLastError();
            rc = MDC_ERR_OOM;
        }
        unsigned char *dev = static_cast<unsigned char *>(b->queue_mem);
        size_t iF = 0, iG = 0, iS = 0;
        for (size_t k = 0; rc == MDC_OK && k < qlaunches.size(); ++k) {
            QLaunch &L = qlaunches[k];
            const bool gemm = L.kind == 1 || L.kind == 3;
            const size_t rsz = gemm ? sizeof(GemmArgs) : sizeof(FftArgs);
            const size_t off = gemm ? oG + iG * rsz : oF + iF * rsz;
            for (size_t i = 0; i < L.members.size(); ++i) memcpy(&host[off + i * rsz], L.recs[i], rsz);
            int *st0 = reinterpret_cast<int *>(&host[oS]) + iS;
            int acc = 0;
            for (size_t i = 0; i < L.members.size(); ++i) {
                st0[i] = acc;
                acc += L.tiles[i];
            }
            st0[L.members.size()] = acc;
            L.q.args = dev + off;
            L.q.start = reinterpret_cast<const int *>(dev + oS) + iS;
            L.q.n = (int)L.members.size();
            L.q.total = acc;
            L.q.counter = reinterpret_cast<unsigned int *>(dev + oC) + k;
            (gemm ? iG : iF) += L.members.size();
            iS += L.members.size() + 1;
        }
        if (rc == MDC_OK) {
            qcounters = reinterpret_cast<unsigned int *>(dev + oC);
            if (cudaMemcpyAsync(b->queue_mem, host.data(), total, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = MDC_ERR_CUDA;
        }
        if (rc != MDC_OK) {
            mdc_batch_destroy(b);
            return rc;
        }
    }

    // branches: members in decreasing cost, each onto the branch with the least work so far
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> cost(n);
    for (int m = 0; m < n; ++m) cost[m] = member_cost(shapes[m], members[m].nb);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<std::vector<int>> branch(b->n_branches);
    std::vector<double> load(b->n_branches, 0.0);
    for (int m : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        branch[k].push_back(m);
        load[k] += cost[m];
    }

    // capture one epoch on private streams
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> bs(b->n_branches, nullptr);
    std::vector<cudaEvent_t> join(b->n_branches, nullptr);
    cudaEvent_t fork = nullptr;
    bool streams_ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; streams_ok && k < b->n_branches; ++k)
        streams_ok = cudaStreamCreateWithFlags(&bs[k], cudaStreamNonBlocking) == cudaSuccess &&
                     cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming) == cudaSuccess;
    std::vector<bool> prof(n, false);
    bool capturing = false;
    if (!streams_ok) rc = MDC_ERR_CUDA;
    if (rc == MDC_OK) {
        for (int m = 0; m < n; ++m) prof[m] = plan_begin_capture(members[m].plan);
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = MDC_ERR_CUDA;
        else capturing = true;
    }
    if (rc == MDC_OK) {
        k_epoch_begin<<<n, 256, 0, cap>>>(b->slots, n, b->epoch);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(fork, cap) != cudaSuccess) rc = MDC_ERR_CUDA;
    }
    if (mode == MDC_BATCH_QUEUE && rc == MDC_OK) {
        if (cudaMemsetAsync(qcounters, 0, (size_t)n_counters * sizeof(unsigned int), cap) != cudaSuccess) rc = MDC_ERR_CUDA;
        for (size_t k = 0; rc == MDC_OK && k < qlaunches.size(); ++k) {
            const QLaunch &L = qlaunches[k];
            cudaError_t e = cudaSuccess;
            switch (L.kind) {
                case 0: e = launch_queue_rfft(L.M, L.variant, L.q, cap); break;
                case 1: e = launch_tc_fwd_queue(L.key, L.q, cap); break;
                case 2: e = launch_queue_residual(L.M, L.variant, L.q, cap); break;
                case 3: e = launch_tc_adj_queue(L.key != 0, L.q, cap); break;
                default: e = launch_queue_update(L.M, L.variant, L.q, cap); break;
            }
            if (e != cudaSuccess) rc = MDC_ERR_CUDA;
        }
    }
    for (int k = 0; mode == MDC_BATCH_BRANCHES && rc == MDC_OK && k < b->n_branches; ++k) {
        if (cudaStreamWaitEvent(bs[k], fork, 0) != cudaSuccess) { rc = MDC_ERR_CUDA; break; }
        for (int m : branch[k]) {
            const smdd_member &mb = members[m];
            const int ns = shapes[m].ns;
            for (int s = 0; s < b->steps[m] && rc == MDC_OK; ++s) {
                smdd_params prm;
                memset(&prm, 0, sizeof(prm));
                prm.alpha = mb.alpha;
                prm.flags = mb.flags | SMDD_KEEP_XHAT | (s > 0 ? SMDD_REUSE_XHAT : 0);
                const int nbs = std::min(mb.nb, ns - s * mb.nb);
                rc = smdd_step(mb.plan, mb.X, mb.U_obs, b->cur_idx[m] + (long long)s * mb.nb, nbs, &prm,
                               b->cur_loss[m] + s, bs[k]);
            }
            if (rc != MDC_OK) break;
        }
        if (rc == MDC_OK && cudaEventRecord(join[k], bs[k]) != cudaSuccess) rc = MDC_ERR_CUDA;
        if (rc == MDC_OK && cudaStreamWaitEvent(cap, join[k], 0) != cudaSuccess) rc = MDC_ERR_CUDA;
    }
    if (rc == MDC_OK) {
        k_epoch_end<<<1, 256, 0, cap>>>(b->slots, n, b->epoch);
        if (cudaGetLastError() != cudaSuccess) rc = MDC_ERR_CUDA;
    }
    if (capturing) {
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cap, &g);
        if (e != cudaSuccess || !g) {
            if (rc == MDC_OK) rc = MDC_ERR_CUDA;
            cudaGetLastError();
        }
        b->graph = g;
    }
    for (int m = 0; m < n; ++m) plan_end_capture(members[m].plan, prof[m]);
    if (rc == MDC_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (rc == MDC_OK) {
        size_t nn = 0;
        if (cudaGraphGetNodes(b->graph, nullptr, &nn) != cudaSuccess) rc = MDC_ERR_CUDA;
        std::vector<cudaGraphNode_t> nodes(nn);
        if (rc == MDC_OK && nn && cudaGraphGetNodes(b->graph, nodes.data(), &nn) != cudaSuccess) rc = MDC_ERR_CUDA;
        for (size_t i = 0; rc == MDC_OK && i < nn; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) b->kernels++;
        }
    }
    for (auto e : join)
        if (e) cudaEventDestroy(e);
    for (auto q : bs)
        if (q) cudaStreamDestroy(q);
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    if (rc != MDC_OK) {
        fprintf(stderr, "smdd: capture of the batch epoch failed (%s)\n", mdc_status_string(rc));
        cudaGetLastError();
        mdc_batch_destroy(b);
        return rc;
    }
    *out = b;
    return MDC_OK;
}

int mdc_batch_run(mdc_batch_t b, long long first_epoch, int n_epochs, void *stream) {
    if (!b || first_epoch < 0 || n_epochs < 0) return MDC_ERR_INVALID_ARG;
    if (n_epochs == 0) return MDC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    int rc = MDC_OK;
    k_set_epoch<<<1, 1, 0, st>>>(b->epoch, first_epoch);
    if (cudaGetLastError() != cudaSuccess) rc = MDC_ERR_CUDA;
    for (int e = 0; rc == MDC_OK && e < n_epochs; ++e)
        if (cudaGraphLaunch(b->exec, st) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return rc;
}

int mdc_batch_info(mdc_batch_t b, long long *kernels_per_epoch, int *n_branches) {
    if (!b) return MDC_ERR_INVALID_ARG;
    if (kernels_per_epoch) *kernels_per_epoch = b->kernels;
    if (n_branches) *n_branches = b->n_branches;
    return MDC_OK;
}

}  // extern "C"
