// C ABI of the stochastic MDD hot path: plan management, the operator entry points and the SGD step.
// See include/smdd.h for the contract of every function.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "smdd_fft.cuh"
#include "smdd_internal.h"

using namespace smdd;

namespace {

struct PendingTiming {
    int stage;
    cudaEvent_t e0, e1;
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

#ifndef SMDD_TC_ADJ_TMA
#define SMDD_TC_ADJ_TMA 1   // the split-BF16 adjoint writes its single-written tiles by tensor-map stores
#endif

}  // namespace

namespace smdd {

bool nfft_supported(int nfft) { return (is_pow2(nfft) && nfft >= 64 && nfft <= 8192) || nfft == 3072; }

int default_nfft(int nt) {
    // the shortest supported length >= max(2 nt - 1, 64): powers of two and 3072 = 3 * 2^10
    int n = 64;
    while (n < 2 * nt - 1) n *= 2;
    return (n == 4096 && 2 * nt - 1 <= 3072) ? 3072 : n;
}

}  // namespace smdd

struct mdc_plan_s {
    int device = 0;
    int nt = 0, nr = 0, nv = 0, ns = 0, nbmax = 0, nfft = 0, M = 0, nf = 0;
    int ldr = 0, ldb = 0;
    int prec = MDC_PREC_FP32;
    float scale = 1.f;
    float2 *Dh = nullptr;        // [nf][ns][ldr]
    float2 *Xh = nullptr;        // [nf][nv][ldr]  model spectra, reused for gradient spectra
    float2 *Uh = nullptr;        // [nf][nv][ldb]  batch spectra (prediction, then residual)
    uint8_t *adj_img = nullptr;  // split-BF16 plans: operand images of the adjoint products (null: not held)
    float2 *tw = nullptr;        // twiddle tables of the FFT variants: 0 at 0, 1 at tw1_off, 2 at tw2_off
    int tw1_off = 0, tw2_off = 0;
    float2 *twN = nullptr;       // [M+1]
    double *partials = nullptr;  // residual-kernel block partials
    double *lam = nullptr;       // [nf] power-iteration results, [nf] = max
    unsigned int *counter = nullptr;
    int *status = nullptr;
    int resid_blocks_max = 0;
    const float *xhat_for = nullptr;  // model pointer whose spectrum Xh holds (KEEP_XHAT)
    int xhat_upper_tr = 0;            // > 0: Xh holds a symmetric model's spectra on and above the block
                                      // diagonal of this many traces only (the lower part is read transposed
                                      // by the tile forward product, or copied before another kernel reads it)
    bool profiling = false;
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> event_pool;
    double stage_ms[MDC_NUM_STAGES] = {0};
    long long stage_launches[MDC_NUM_STAGES] = {0};
    long long launches = 0;
    // kernel configuration (see mdc_config)
    int fft_variant = 0;
    int fft_prefetch = 0;        // update: persistent CTAs prefetching the next tile (variants 0/1, M <= 1536)
    int gemm_fwd = MDC_GEMM_SIMT;
    int gemm_adj = MDC_GEMM_SIMT;
    int nf_active = 0;           // band limit of the products (0: every bin)
    long long wait_probe = 0;    // failure-path check of the tensor-core kernels (cycles; 0 = off)
    // host-input steps (smdd_step_host): two device staging slots, filled on a copy stream
    struct HostStage {
        float *U[2] = {nullptr, nullptr};              // [nbmax][nv][nt] batch rows
        int32_t *idx[2] = {nullptr, nullptr};          // [nbmax] batch indices (device)
        int32_t *idx_pinned[2] = {nullptr, nullptr};   // [nbmax] batch indices (pinned host copy)
        double *loss[2] = {nullptr, nullptr};
        cudaEvent_t copied[2] = {nullptr, nullptr};    // the slot's copies landed
        cudaEvent_t consumed[2] = {nullptr, nullptr};  // the slot's step finished with it
        cudaStream_t copy = nullptr;
        int next = 0;
    } *hs = nullptr;
    alignas(64) unsigned char xh_map[128] = {0};   // tensor map of Xh for the streamed forward product
    bool xh_map_ok = false;
    LsqrWork *lsqr = nullptr;    // full-gradient solver workspace, allocated by the first smdd_lsqr
};

namespace {

cudaEvent_t get_event(mdc_plan_s *p) {
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

template <class F>
int launch_stage(mdc_plan_s *p, int stage, cudaStream_t st, F &&fn) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (p->profiling) {
        e0 = get_event(p);
        e1 = get_event(p);
        cudaEventRecord(e0, st);
    }
    const cudaError_t err = fn();
    if (p->profiling) {
        cudaEventRecord(e1, st);
        p->pending.push_back({stage, e0, e1});
    }
    p->launches++;
    p->stage_launches[stage]++;
    if (err != cudaSuccess) {
        fprintf(stderr, "smdd: launch of stage %d failed: %s\n", stage, cudaGetErrorString(err));
        return MDC_ERR_CUDA;
    }
    return MDC_OK;
}

FftArgs base_fft(const mdc_plan_s *p) {
    FftArgs a;
    memset(&a, 0, sizeof(a));
    a.nt = p->nt;
    a.tw = p->tw + (p->fft_variant == 2 ? p->tw2_off : p->fft_variant == 1 ? p->tw1_off : 0);
    a.variant = p->fft_variant;
    a.prefetch = p->fft_prefetch;
    a.twN = p->twN;
    a.s = p->scale / (float)p->nfft;
    a.status = p->status;
    return a;
}

int ti_log2_for(int n_contig, int TR) {
    // as many consecutive traces along the contiguous spectrum axis as the tile holds
    int l = 0;
    while ((1 << (l + 1)) <= TR && (1 << l) < n_contig) ++l;
    return l;
}


// time traces may be read and written as float4: every trace starts on a 16-byte boundary
bool vec4_ok(int nt, const void *p) { return nt % 4 == 0 && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int traces_per_cta(const mdc_plan_s *p) {
    return p->fft_variant == 2 ? fft2_traces_per_cta(p->M) : fft_traces_per_cta(p->M);
}

// model-layout grid: trace (i = r, j = v) of a [nv][nr][nt] array  <->  spectra [nf][nv][ldr]
TraceGrid model_grid(const mdc_plan_s *p, int nouter) {
    TraceGrid g;
    g.ni = p->nr;
    g.nj = nouter;
    g.ti_log2 = ti_log2_for(p->nr, traces_per_cta(p));
    g.tsi = p->nt;
    g.tsj = (long long)p->nr * p->nt;
    g.ssi = 1;
    g.ssj = p->ldr;
    g.ssf = (long long)nouter * p->ldr;
    return g;
}

// batch-layout grid: trace (i = b, j = v) of a [nb][nv][nt] array  <->  spectra [nf][nv][ldb]
TraceGrid batch_grid(const mdc_plan_s *p, int nb) {
    TraceGrid g;
    g.ni = nb;
    g.nj = p->nv;
    g.ti_log2 = ti_log2_for(nb, traces_per_cta(p));
    g.tsi = (long long)p->nv * p->nt;
    g.tsj = p->nt;
    g.ssi = 1;
    g.ssj = p->ldb;
    g.ssf = (long long)p->nv * p->ldb;
    return g;
}

int rfft_model(mdc_plan_s *p, const float *X, cudaStream_t st) {
    p->xhat_upper_tr = 0;   // every bin of every trace
    FftArgs a = base_fft(p);
    a.g = model_grid(p, p->nv);
    a.tin = X;
    a.vec = vec4_ok(p->nt, X);
    a.spec = p->Xh;
    return launch_stage(p, ST_RFFT, st, [&] { return launch_rfft(p->M, a, st); });
}

int gemm_forward(mdc_plan_s *p, const int32_t *idx, int nb, cudaStream_t st) {
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = p->Xh;
    g.Dh = p->Dh;
    g.idx = idx;
    g.C = p->Uh;
    g.nv = p->nv; g.nr = p->nr; g.ns = p->ns; g.nb = nb; g.ldr = p->ldr; g.ldb = p->ldb;
    g.sAf = (long long)p->nv * p->ldr;
    g.sDf = (long long)p->ns * p->ldr;
    g.sCf = (long long)p->nv * p->ldb;
    g.outscale = 1.f;
    g.status = p->status;
    g.nf_active = p->nf_active;
    g.wait_probe = p->wait_probe;
    if (p->xhat_upper_tr > 0) {
        // the spectra below the block diagonal of a symmetric model: read transposed by the tile kernel,
        // else copied into place first
        if (p->gemm_fwd == MDC_GEMM_TC) {
            g.sym_tr = p->xhat_upper_tr;
        } else {
            const int tr = p->xhat_upper_tr;
            p->xhat_upper_tr = 0;
            const int rc = launch_stage(p, ST_GEMM_FWD, st, [&] {
                return launch_mirror_lower(p->Xh, p->nv, p->ldr, (long long)p->nv * p->ldr, p->nf, tr, st);
            });
            if (rc) return rc;
        }
    }
    if (p->gemm_fwd == MDC_GEMM_TC)
        return launch_stage(p, ST_GEMM_FWD, st, [&] { return launch_tc_fwd(g, p->nf, st); });
    if (p->gemm_fwd == MDC_GEMM_TC_STREAM && p->xh_map_ok)
        return launch_stage(p, ST_GEMM_FWD, st, [&] { return launch_tc_fwd_stream(g, p->xh_map, p->nf, st); });
    if (p->gemm_fwd == MDC_GEMM_GEMV && gemv_supported(p->nv) && p->nf_active == 0)
        return launch_stage(p, ST_GEMM_FWD, st, [&] { return launch_gemv_fwd(g, p->nf, st); });
    return launch_stage(p, ST_GEMM_FWD, st, [&] { return launch_cgemm_fwd(g, p->nf, st); });
}

int gemm_adjoint(mdc_plan_s *p, const int32_t *idx, int nb, bool recip, cudaStream_t st, bool no_mirror = false) {
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = p->Uh;
    g.Dh = p->Dh;
    g.idx = idx;
    g.C = p->Xh;
    g.nv = p->nv; g.nr = p->nr; g.ns = p->ns; g.nb = nb; g.ldr = p->ldr; g.ldb = p->ldb;
    g.sAf = (long long)p->nv * p->ldb;
    g.sDf = (long long)p->ns * p->ldr;
    g.sCf = (long long)p->nv * p->ldr;
    g.outscale = recip ? 0.5f : 1.f;
    g.status = p->status;
    g.nf_active = p->nf_active;
    g.wait_probe = p->wait_probe;
    g.no_mirror = (recip && no_mirror) ? 1 : 0;
    if (p->gemm_adj == MDC_GEMM_TC)
        return launch_stage(p, ST_GEMM_ADJ, st, [&] {
            // the operand images of this step's residual spectra and batch rows, then the products from them
            if (p->adj_img && tc_adj_image_bytes(p->nv, p->nr, nb, p->nf) > 0) {
                const cudaError_t e = launch_tc_adj_images(g, p->adj_img, p->nf, st);
                if (e != cudaSuccess) return e;
                g.img = p->adj_img;
                g.img_nkc = (nb + 31) / 32;
            }
            return launch_tc_adj(g, recip, p->nf, st, (SMDD_TC_ADJ_TMA && p->xh_map_ok) ? p->xh_map : nullptr);
        });
    if (p->gemm_adj == MDC_GEMM_GEMV && gemv_supported(p->nv) && !recip && p->nf_active == 0 && nb <= 1024)
        return launch_stage(p, ST_GEMM_ADJ, st, [&] { return launch_gemv_adj(g, p->nf, st); });
    const int tile = p->gemm_adj == MDC_GEMM_SIMT32 ? 32 : p->gemm_adj == MDC_GEMM_SIMT64 ? 64 : 0;
    return launch_stage(p, ST_GEMM_ADJ, st, [&] { return launch_cgemm_adj(g, recip, p->nf, st, tile); });
}

int forward_impl(mdc_plan_s *p, const float *X, const int32_t *idx, int nb, float *U, cudaStream_t st) {
    int rc;
    p->xhat_for = nullptr;
    if ((rc = rfft_model(p, X, st))) return rc;
    if ((rc = gemm_forward(p, idx, nb, st))) return rc;
    FftArgs a = base_fft(p);
    a.g = batch_grid(p, nb);
    a.tout = U;
    a.vec = vec4_ok(p->nt, U);
    a.spec = p->Uh;
    return launch_stage(p, ST_IRFFT_OUT, st, [&] { return launch_irfft_out(p->M, a, st); });
}

// adjoint, with the reciprocity projection 1/2 (G + G^T) when recip
int adjoint_impl(mdc_plan_s *p, const float *R, const int32_t *idx, int nb, float *G, bool recip, cudaStream_t st) {
    int rc;
    p->xhat_for = nullptr;
    {
        FftArgs a = base_fft(p);
        a.g = batch_grid(p, nb);
        a.tin = R;
        a.vec = vec4_ok(p->nt, R);
        a.spec = p->Uh;
        if ((rc = launch_stage(p, ST_RFFT, st, [&] { return launch_rfft(p->M, a, st); }))) return rc;
    }
    if ((rc = gemm_adjoint(p, idx, nb, recip, st))) return rc;
    FftArgs a = base_fft(p);
    a.g = model_grid(p, p->nv);
    a.tout = G;
    a.vec = vec4_ok(p->nt, G);
    a.spec = p->Xh;
    return launch_stage(p, ST_IRFFT_OUT, st, [&] { return launch_irfft_out(p->M, a, st); });
}

int check_common(mdc_plan_s *p, const void *a, const void *b, const int32_t *idx, int nb) {
    if (!p || !a || !b || !idx) return MDC_ERR_INVALID_ARG;
    if (nb < 1) return MDC_ERR_INVALID_ARG;
    if (nb > p->nbmax) return MDC_ERR_SHAPE;
    return MDC_OK;
}

}  // namespace

namespace smdd {

PlanShape plan_shape(const mdc_plan_s *p) {
    PlanShape sh;
    sh.nt = p->nt; sh.nr = p->nr; sh.nv = p->nv; sh.ns = p->ns; sh.nbmax = p->nbmax;
    sh.nfft = p->nfft; sh.nf = p->nf; sh.prec = p->prec; sh.device = p->device;
    return sh;
}

bool plan_begin_capture(mdc_plan_s *p) {
    const bool was = p->profiling;
    p->profiling = false;   // no timing events inside a graph
    p->xhat_for = nullptr;
    return was;
}

void plan_end_capture(mdc_plan_s *p, bool profiling) {
    p->profiling = profiling;
    p->xhat_for = nullptr;  // what the capture recorded has not run
}

}  // namespace smdd

extern "C" {

const char *mdc_status_string(int s) {
    switch (s) {
        case MDC_OK: return "MDC_OK";
        case MDC_ERR_INVALID_ARG: return "MDC_ERR_INVALID_ARG";
        case MDC_ERR_SHAPE: return "MDC_ERR_SHAPE";
        case MDC_ERR_INDEX_RANGE: return "MDC_ERR_INDEX_RANGE";
        case MDC_ERR_OOM: return "MDC_ERR_OOM";
        case MDC_ERR_CUDA: return "MDC_ERR_CUDA";
        case MDC_ERR_TIMEOUT: return "MDC_ERR_TIMEOUT";
        case MDC_ERR_UNSUPPORTED: return "MDC_ERR_UNSUPPORTED";
    }
    return "MDC_ERR_UNKNOWN";
}

const char *mdc_stage_name(int stage) {
    static const char *names[MDC_NUM_STAGES] = {"rfft", "cgemm_fwd", "residual", "cgemm_adj",
                                                "update", "irfft_out", "setup"};
    return (stage >= 0 && stage < MDC_NUM_STAGES) ? names[stage] : "unknown";
}

int mdc_plan_create(mdc_plan_t *out, int nt, int nr, int nv, int ns, int nb_max, int nfft, float scale,
                    const float *D, int precision, void *stream) {
    if (!out || !D) return MDC_ERR_INVALID_ARG;
    *out = nullptr;
    if (nt < 1 || nr < 1 || nv < 1 || ns < 1 || nb_max < 0) return MDC_ERR_INVALID_ARG;
    if (precision != MDC_PREC_FP32 && precision != MDC_PREC_BF16X3) return MDC_ERR_UNSUPPORTED;
    if (!std::isfinite(scale)) return MDC_ERR_INVALID_ARG;
    if (nt > 4096) return MDC_ERR_UNSUPPORTED;
    if (nfft == 0) {
        nfft = default_nfft(nt);
    } else if (!nfft_supported(nfft) || nfft < 2 * nt - 1) {
        return MDC_ERR_UNSUPPORTED;
    }
    if (nb_max == 0) nb_max = ns;
    if (nb_max > 1024) return MDC_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;

    mdc_plan_s *p = new (std::nothrow) mdc_plan_s();
    if (!p) return MDC_ERR_OOM;
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return MDC_ERR_CUDA; }
    p->nt = nt; p->nr = nr; p->nv = nv; p->ns = ns; p->nbmax = nb_max;
    p->nfft = nfft; p->M = nfft / 2; p->nf = nfft / 2 + 1;
    p->ldr = (nr + 1) & ~1;
    p->ldb = (nb_max + 1) & ~1;
    p->scale = scale;
    p->prec = precision;
    p->gemm_fwd = p->gemm_adj = (precision == MDC_PREC_BF16X3) ? MDC_GEMM_TC : MDC_GEMM_SIMT;
    // default FFT: the two-pass form where it measured faster (nfft 2048: update 750 vs 886 us at 301^2)
    p->fft_variant = (nfft == 2048) ? 2 : 0;
    p->tw1_off = ((fft_tw_size(nfft / 2, 0) > 1 ? fft_tw_size(nfft / 2, 0) : 1) + 1) & ~1;
    p->tw2_off = p->tw1_off + (((fft_tw_size(nfft / 2, 1) > 1 ? fft_tw_size(nfft / 2, 1) : 1) + 1) & ~1);

    const int M = p->M, nf = p->nf;
    const size_t szD = (size_t)nf * ns * p->ldr * sizeof(float2);
    const size_t szX = (size_t)nf * nv * p->ldr * sizeof(float2);
    const size_t szU = (size_t)nf * nv * p->ldb * sizeof(float2);
    {
        // the residual kernel of every FFT variant must fit the partials buffer
        const int v_default = p->fft_variant;
        p->fft_variant = 0;
        p->resid_blocks_max = fft_blocks(M, batch_grid(p, nb_max));
        if (fft2_supported(M)) {
            p->fft_variant = 2;
            p->resid_blocks_max = std::max(p->resid_blocks_max, fft2_blocks(M, batch_grid(p, nb_max)));
        }
        p->fft_variant = v_default;
    }
    bool ok = cudaMalloc(&p->Dh, szD) == cudaSuccess && cudaMalloc(&p->Xh, szX) == cudaSuccess &&
              cudaMalloc(&p->Uh, szU) == cudaSuccess && cudaMalloc(&p->tw, (size_t)(p->tw2_off + std::max(fft2_tw_size(M), M) + 2) * sizeof(float2)) == cudaSuccess &&
              cudaMalloc(&p->twN, (M + 1) * sizeof(float2)) == cudaSuccess &&
              cudaMalloc(&p->partials, (size_t)(p->resid_blocks_max + 1) * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&p->lam, (size_t)(nf + 1) * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&p->counter, sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc(&p->status, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        mdc_plan_destroy(p);
        return MDC_ERR_OOM;
    }
    // split-BF16 plans: operand images for the adjoint products of batches up to 64 (the products split their
    // operands themselves where these do not fit)
    if (precision == MDC_PREC_BF16X3) {
        const size_t bytes = tc_adj_image_bytes(nv, nr, nb_max, nf);
        if (bytes > 0 && cudaMalloc(&p->adj_img, bytes) != cudaSuccess) {
            cudaGetLastError();
            p->adj_img = nullptr;
        }
    }
    // per-pass twiddle tables in double precision, rounded once to float
    const double pi = 3.14159265358979323846;
    std::vector<float2> tw, tw1;
    fft_tw_fill(M, tw, 0);
    fft_tw_fill(M, tw1, 1);
    int rc = MDC_OK;
    if (cudaMemcpyAsync(p->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (cudaMemcpyAsync(p->tw + p->tw1_off, tw1.data(), tw1.size() * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = MDC_ERR_CUDA;
    std::vector<float2> tw2;
    if (fft2_supported(M)) {
        fft2_tw_fill(M, tw2);
        if (cudaMemcpyAsync(p->tw + p->tw2_off, tw2.data(), tw2.size() * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = MDC_ERR_CUDA;
    }
    std::vector<float2> twn(M + 1);
    for (int k = 0; k <= M; ++k) {
        const double ang = 2.0 * pi * (double)k / (double)nfft;
        twn[k] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    if (cudaMemcpyAsync(p->twN, twn.data(), (M + 1) * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (cudaMemsetAsync(p->counter, 0, sizeof(unsigned int), st) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (cudaMemsetAsync(p->status, 0, sizeof(int), st) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (cudaMemsetAsync(p->Dh, 0, szD, st) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (cudaMemsetAsync(p->Xh, 0, szX, st) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (cudaMemsetAsync(p->Uh, 0, szU, st) != cudaSuccess) rc = MDC_ERR_CUDA;
    if (rc == MDC_OK && (fft_prepare(M) != cudaSuccess || gemm_prepare() != cudaSuccess)) rc = MDC_ERR_CUDA;
    if (rc == MDC_OK && precision == MDC_PREC_BF16X3 && tc_prepare() != cudaSuccess) rc = MDC_ERR_CUDA;
    if (rc == MDC_OK && precision == MDC_PREC_BF16X3)   // without a map, MDC_GEMM_TC_STREAM is unsupported
        p->xh_map_ok = tc_encode_fwd_map(p->xh_map, p->Xh, nr, nv, p->ldr, p->nf) == cudaSuccess;
    if (rc == MDC_OK) {
        // kernel spectra: D [ns][nr][nt] -> Dh [nf][ns][ldr] (same layout rule as the model)
        FftArgs a = base_fft(p);
        a.g = model_grid(p, ns);
        a.tin = D;
        a.vec = vec4_ok(nt, D);
        a.spec = p->Dh;
        rc = launch_stage(p, ST_SETUP, st, [&] { return launch_rfft(M, a, st); });
    }
    if (rc == MDC_OK) {
        // the host twiddle vectors must outlive the asynchronous copies
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = MDC_ERR_CUDA;
    }
    if (rc != MDC_OK) {
        mdc_plan_destroy(p);
        return rc;
    }
    *out = p;
    return MDC_OK;
}

static void host_stage_free(mdc_plan_s *p) {
    if (!p->hs) return;
    auto &h = *p->hs;
    for (int i = 0; i < 2; ++i) {
        cudaFree(h.U[i]);
        cudaFree(h.idx[i]);
        cudaFree(h.loss[i]);
        cudaFreeHost(h.idx_pinned[i]);
        if (h.copied[i]) cudaEventDestroy(h.copied[i]);
        if (h.consumed[i]) cudaEventDestroy(h.consumed[i]);
    }
    if (h.copy) cudaStreamDestroy(h.copy);
    delete p->hs;
    p->hs = nullptr;
}

static int host_stage_init(mdc_plan_s *p) {
    p->hs = new mdc_plan_s::HostStage;
    auto &h = *p->hs;
    bool ok = cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < 2; ++i) {
        ok = cudaMalloc(&h.U[i], (size_t)p->nbmax * p->nv * p->nt * sizeof(float)) == cudaSuccess &&
             cudaMalloc(&h.idx[i], (size_t)p->nbmax * sizeof(int32_t)) == cudaSuccess &&
             cudaMalloc(&h.loss[i], sizeof(double)) == cudaSuccess &&
             cudaHostAlloc(&h.idx_pinned[i], (size_t)p->nbmax * sizeof(int32_t), cudaHostAllocDefault) == cudaSuccess &&
             cudaEventCreateWithFlags(&h.copied[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&h.consumed[i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        host_stage_free(p);
        return MDC_ERR_OOM;
    }
    return MDC_OK;
}

int mdc_plan_destroy(mdc_plan_t p) {
    if (!p) return MDC_OK;
    DeviceGuard dg(p->device);
    cudaDeviceSynchronize();
    host_stage_free(p);
    cudaFree(p->Dh);
    cudaFree(p->Xh);
    cudaFree(p->Uh);
    cudaFree(p->adj_img);
    cudaFree(p->tw);
    cudaFree(p->twN);
    cudaFree(p->partials);
    cudaFree(p->lam);
    cudaFree(p->counter);
    cudaFree(p->status);
    for (auto &t : p->pending) {
        cudaEventDestroy(t.e0);
        cudaEventDestroy(t.e1);
    }
    for (auto e : p->event_pool) cudaEventDestroy(e);
    delete p->lsqr;
    delete p;
    return MDC_OK;
}

int mdc_plan_info(mdc_plan_t p, int *nfft, int *nf) {
    if (!p) return MDC_ERR_INVALID_ARG;
    if (nfft) *nfft = p->nfft;
    if (nf) *nf = p->nf;
    return MDC_OK;
}

int mdc_plan_sigma2_max(mdc_plan_t p, int n_iter, double *sigma2, void *stream) {
    if (!p || !sigma2 || n_iter < 1) return MDC_ERR_INVALID_ARG;
    if ((size_t)(2 * p->nr + p->ns) * sizeof(float2) > 227 * 1024) return MDC_ERR_UNSUPPORTED;
    DeviceGuard dg(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_stage(p, ST_SETUP, st, [&] {
        return launch_power_iter(p->Dh, p->ns, p->nr, p->ldr, (long long)p->ns * p->ldr, p->nf, n_iter, p->lam, st);
    });
    if (rc) return rc;
    rc = launch_stage(p, ST_SETUP, st, [&] { return launch_max_reduce(p->lam, p->nf, p->lam + p->nf, st); });
    if (rc) return rc;
    double v = 0.0;
    if (cudaMemcpyAsync(&v, p->lam + p->nf, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MDC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MDC_ERR_CUDA;
    *sigma2 = v * (double)p->scale * (double)p->scale;
    return MDC_OK;
}

int mdc_forward(mdc_plan_t p, const float *X, const int32_t *idx, int nb, float *U, void *stream) {
    int rc = check_common(p, X, U, idx, nb);
    if (rc) return rc;
    DeviceGuard dg(p->device);
    return forward_impl(p, X, idx, nb, U, (cudaStream_t)stream);
}

int mdc_adjoint(mdc_plan_t p, const float *R, const int32_t *idx, int nb, float *G, void *stream) {
    int rc = check_common(p, R, G, idx, nb);
    if (rc) return rc;
    DeviceGuard dg(p->device);
    return adjoint_impl(p, R, idx, nb, G, false, (cudaStream_t)stream);
}

int smdd_lsqr(mdc_plan_t p, float *X, const float *U_obs, int n_iter, int flags, const int32_t *mute, double *norms,
              void *stream) {
    if (!p || !X || !U_obs || n_iter < 0) return MDC_ERR_INVALID_ARG;
    if (flags & ~SMDD_RECIPROCITY) return MDC_ERR_INVALID_ARG;
    const bool recip = flags & SMDD_RECIPROCITY;
    if (recip && p->nr != p->nv) return MDC_ERR_SHAPE;
    if (p->nbmax < p->ns) return MDC_ERR_SHAPE;
    DeviceGuard dg(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long nd = (long long)p->ns * p->nv * p->nt, nm = (long long)p->nv * p->nr * p->nt;
    if (!p->lsqr || p->lsqr->nd != nd || p->lsqr->nm != nm) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return MDC_ERR_INVALID_ARG;
        if (!p->lsqr) p->lsqr = new (std::nothrow) LsqrWork();
        if (!p->lsqr) return MDC_ERR_OOM;
        if (p->lsqr->ensure(nd, nm, p->ns) != cudaSuccess) {
            cudaGetLastError();
            return MDC_ERR_OOM;
        }
        std::vector<int32_t> h(p->ns);
        for (int i = 0; i < p->ns; ++i) h[i] = i;
        if (cudaMemcpy(p->lsqr->idx, h.data(), p->ns * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
            return MDC_ERR_CUDA;
    }
    LsqrWork &wk = *p->lsqr;
    int orc = MDC_OK;
    auto fwd = [&](const float *x, float *out) -> cudaError_t {
        orc = forward_impl(p, x, wk.idx, p->ns, out, st);
        return orc ? cudaErrorUnknown : cudaSuccess;
    };
    auto adj = [&](const float *r, float *out) -> cudaError_t {
        orc = adjoint_impl(p, r, wk.idx, p->ns, out, recip, st);
        return orc ? cudaErrorUnknown : cudaSuccess;
    };
    p->xhat_for = nullptr;
    const cudaError_t e = lsqr_run(wk, X, U_obs, nd, nm, p->nt, n_iter, mute, norms, st, fwd, adj, &p->launches);
    if (orc) return orc;
    return e == cudaSuccess ? MDC_OK : MDC_ERR_CUDA;
}

}  // extern "C"

namespace {

// Adam state of one step (Kingma & Ba, Algorithm 1): moments m, v and the scalars of step t
struct AdamArgs {
    float *m = nullptr, *v = nullptr;
    float beta1 = 0.f, beta2 = 0.f, eps = 0.f, c1 = 1.f, c2 = 1.f;
};

// One step; SGD when vel and adam.m are null, N-SGD with vel, Adam with adam.m; mute: causality table or
// null.  Arguments checked by the callers.
int step_impl(mdc_plan_t p, float *X, const float *U_obs, const int32_t *idx, int nb, float alpha, int flags,
              float *vel, float mu, const int32_t *mute, double *loss, cudaStream_t st,
              const AdamArgs &adam = AdamArgs()) {
    int rc = MDC_OK;
    const bool recip = flags & SMDD_RECIPROCITY;
    const bool ext = vel || mute || adam.m;
    // the update's FFT plan: the momentum / mute / Adam update and the upper enumeration of a symmetric
    // model exist for the radix orders only (variant 0 where the plan uses the register FFT)
    const int v_plan = p->fft_variant;
    const int v_upd = ext ? 0 : ((recip && (flags & SMDD_SYMMETRIC) && v_plan == 2) ? 0 : v_plan);
    p->fft_variant = v_upd;
    const TraceGrid mg = model_grid(p, p->nv);
    const bool sym = recip && (flags & SMDD_SYMMETRIC) && (1 << mg.ti_log2) == traces_per_cta(p) &&
                     traces_per_cta(p) <= 32;
    const int tr_upd = traces_per_cta(p);
    p->fft_variant = v_plan;
    // a1: model spectra (or the ones left by the previous step's fused update)
    if (!((flags & SMDD_REUSE_XHAT) && p->xhat_for == X)) {
        if ((rc = rfft_model(p, X, st))) return rc;
    }
    p->xhat_for = nullptr;
    // a2 + a3: gathered kernel rows x model spectra
    if ((rc = gemm_forward(p, idx, nb, st))) return rc;
    // a4 + a5: inverse FFT, window, residual, loss, residual spectra
    {
        FftArgs a = base_fft(p);
        a.g = batch_grid(p, nb);
        a.spec = p->Uh;
        a.uobs = U_obs;
        a.idx = idx;
        a.ns = p->ns;
        a.gathered = (flags & SMDD_UOBS_GATHERED) ? 1 : 0;
        a.uo_si = (long long)p->nv * p->nt;
        a.uo_sj = p->nt;
        a.vec = vec4_ok(p->nt, U_obs);
        a.partials = p->partials;
        a.counter = p->counter;
        a.loss = loss;
        if ((rc = launch_stage(p, ST_RESID, st, [&] { return launch_residual(p->M, a, p->resid_blocks_max, st); })))
            return rc;
    }
    // a6: gradient spectra (with the reciprocity projection folded in; a symmetric model's update reads
    // the upper triangle only, so the mirrored tiles are not written)
    if ((rc = gemm_adjoint(p, idx, nb, recip, st, sym))) return rc;
    // a7 + a8: inverse FFT, window, update, and optionally the spectra of the new model
    {
        const bool keep = flags & SMDD_KEEP_XHAT;
        // grid and twiddle table of the update's FFT plan (v_upd)
        p->fft_variant = v_upd;
        FftArgs a = base_fft(p);
        a.g = mg;
        p->fft_variant = v_plan;
        if (sym) {
            a.g.sym = 1;
            a.prefetch = 0;
        }
        a.tout = X;
        a.vec = vec4_ok(p->nt, X) && (vel == nullptr || vec4_ok(p->nt, vel)) &&
                (adam.m == nullptr || (vec4_ok(p->nt, adam.m) && vec4_ok(p->nt, adam.v)));
        a.spec = p->Xh;
        a.alpha = alpha;
        a.vel = vel;
        a.mu = mu;
        a.mute = mute;
        a.adam_m = adam.m;
        a.adam_v = adam.v;
        a.beta1 = adam.beta1;
        a.beta2 = adam.beta2;
        a.eps = adam.eps;
        a.c1 = adam.c1;
        a.c2 = adam.c2;
        // a symmetric model's spectra below the block diagonal are copies of the ones above it: the tile
        // forward product of the next step reads them transposed, any other kernel needs the copy
        const bool mirror = keep && sym && p->gemm_fwd != MDC_GEMM_TC;
        if ((rc = launch_stage(p, ST_UPDATE, st, [&] {
                 const cudaError_t e = launch_update(p->M, keep, a, st);
                 if (e != cudaSuccess || !mirror) return e;
                 return launch_mirror_lower(p->Xh, p->nv, p->ldr, (long long)p->nv * p->ldr, p->nf, tr_upd, st);
             })))
            return rc;
        if (keep) p->xhat_for = X;
        p->xhat_upper_tr = (keep && sym && !mirror) ? tr_upd : 0;
    }
    return MDC_OK;
}

}  // namespace

namespace smdd {

int plan_step_records(mdc_plan_s *p, float *X, const float *U_obs, const int32_t *idx, int nb, float alpha, int flags,
                      double *loss, StepRecords *r) {
    if (!p || !X || !U_obs || !idx || !r || nb < 1 || nb > p->nbmax) return MDC_ERR_INVALID_ARG;
    if (p->prec != MDC_PREC_BF16X3 || (p->gemm_fwd != MDC_GEMM_TC && p->gemm_fwd != MDC_GEMM_TC_STREAM) ||
        p->gemm_adj != MDC_GEMM_TC || p->nf_active != 0)
        return MDC_ERR_UNSUPPORTED;
    const bool recip = flags & SMDD_RECIPROCITY;
    if (recip && p->nr != p->nv) return MDC_ERR_SHAPE;
    memset(r, 0, sizeof(*r));
    r->M = p->M;
    r->variant = p->fft_variant;
    auto tiles = [&](const TraceGrid &g) {
        return p->fft_variant == 2 ? fft2_blocks(p->M, g) : fft_blocks(p->M, g);
    };
    // model transform
    r->rfft = base_fft(p);
    r->rfft.g = model_grid(p, p->nv);
    r->rfft.tin = X;
    r->rfft.vec = vec4_ok(p->nt, X);
    r->rfft.spec = p->Xh;
    r->rfft_tiles = tiles(r->rfft.g);
    // forward product (as gemm_forward, on the tile kernel)
    GemmArgs &g = r->fwd;
    g.A = p->Xh; g.Dh = p->Dh; g.idx = idx; g.C = p->Uh;
    g.nv = p->nv; g.nr = p->nr; g.ns = p->ns; g.nb = nb; g.ldr = p->ldr; g.ldb = p->ldb;
    g.sAf = (long long)p->nv * p->ldr; g.sDf = (long long)p->ns * p->ldr; g.sCf = (long long)p->nv * p->ldb;
    g.outscale = 1.f;
    g.status = p->status;
    g.wait_probe = p->wait_probe;
    r->fwd_nb = tc_fwd_queue_nb(nb);
    r->fwd_tiles = tc_fwd_tiles(g, p->nf);
    // residual step (as step_impl)
    FftArgs &a = r->resid;
    a = base_fft(p);
    a.g = batch_grid(p, nb);
    a.spec = p->Uh;
    a.uobs = U_obs;
    a.idx = idx;
    a.ns = p->ns;
    a.gathered = (flags & SMDD_UOBS_GATHERED) ? 1 : 0;
    a.uo_si = (long long)p->nv * p->nt;
    a.uo_sj = p->nt;
    a.vec = vec4_ok(p->nt, U_obs);
    a.partials = p->partials;
    a.counter = p->counter;
    a.loss = loss;
    r->resid_tiles = tiles(a.g);
    if (r->resid_tiles <= 0 || r->resid_tiles > p->resid_blocks_max) return MDC_ERR_INVALID_ARG;
    // adjoint product
    GemmArgs &h = r->adj;
    h.A = p->Uh; h.Dh = p->Dh; h.idx = idx; h.C = p->Xh;
    h.nv = p->nv; h.nr = p->nr; h.ns = p->ns; h.nb = nb; h.ldr = p->ldr; h.ldb = p->ldb;
    h.sAf = (long long)p->nv * p->ldb; h.sDf = (long long)p->ns * p->ldr; h.sCf = (long long)p->nv * p->ldr;
    h.outscale = recip ? 0.5f : 1.f;
    h.status = p->status;
    h.wait_probe = p->wait_probe;
    r->adj_tiles = tc_adj_tiles(h, recip, p->nf);
    r->recip = recip;
    // update with the spectra of the new model
    FftArgs &u = r->upd;
    u = base_fft(p);
    u.g = model_grid(p, p->nv);
    u.tout = X;
    u.vec = vec4_ok(p->nt, X);
    u.spec = p->Xh;
    u.alpha = alpha;
    r->upd_tiles = tiles(u.g);
    return (r->rfft_tiles < 0 || r->upd_tiles < 0) ? MDC_ERR_INVALID_ARG : MDC_OK;
}

}  // namespace smdd

extern "C" {

int smdd_step(mdc_plan_t p, float *X, const float *U_obs, const int32_t *idx, int nb, const smdd_params *prm,
              double *loss, void *stream) {
    int rc = check_common(p, X, U_obs, idx, nb);
    if (rc) return rc;
    if (!prm) return MDC_ERR_INVALID_ARG;
    const int flags = prm->flags;
    if (flags & ~(SMDD_RECIPROCITY | SMDD_KEEP_XHAT | SMDD_REUSE_XHAT | SMDD_UOBS_GATHERED | SMDD_SYMMETRIC))
        return MDC_ERR_INVALID_ARG;
    for (int i = 0; i < 6; ++i)
        if (prm->reserved[i] != 0) return MDC_ERR_INVALID_ARG;
    if (!std::isfinite(prm->alpha)) return MDC_ERR_INVALID_ARG;
    if ((flags & SMDD_RECIPROCITY) && p->nr != p->nv) return MDC_ERR_SHAPE;
    DeviceGuard dg(p->device);
    return step_impl(p, X, U_obs, idx, nb, prm->alpha, flags, nullptr, 0.f, nullptr, loss, (cudaStream_t)stream);
}

int smdd_step_host(mdc_plan_t p, float *X, const float *U_host, const int32_t *idx_host, int nb,
                   const smdd_params *prm, double *loss_host, void *stream) {
    int rc = check_common(p, X, U_host, idx_host, nb);
    if (rc) return rc;
    if (!prm) return MDC_ERR_INVALID_ARG;
    const int flags = prm->flags;
    if (flags & ~(SMDD_RECIPROCITY | SMDD_KEEP_XHAT | SMDD_REUSE_XHAT | SMDD_SYMMETRIC)) return MDC_ERR_INVALID_ARG;
    for (int i = 0; i < 6; ++i)
        if (prm->reserved[i] != 0) return MDC_ERR_INVALID_ARG;
    if (!std::isfinite(prm->alpha)) return MDC_ERR_INVALID_ARG;
    if ((flags & SMDD_RECIPROCITY) && p->nr != p->nv) return MDC_ERR_SHAPE;
    for (int b = 0; b < nb; ++b)
        if (idx_host[b] < 0 || idx_host[b] >= p->ns) return MDC_ERR_INDEX_RANGE;
    DeviceGuard dg(p->device);
    if (!p->hs && (rc = host_stage_init(p))) return rc;
    auto &h = *p->hs;
    const int s = h.next;
    h.next ^= 1;
    cudaStream_t st = (cudaStream_t)stream;
    // the pinned index slot was the source of this slot's previous copy (long finished in a pipeline)
    if (cudaEventSynchronize(h.copied[s]) != cudaSuccess) return MDC_ERR_CUDA;
    memcpy(h.idx_pinned[s], idx_host, (size_t)nb * sizeof(int32_t));
    // the device slot is free once the step that used it two calls back has finished
    if (cudaStreamWaitEvent(h.copy, h.consumed[s], 0) != cudaSuccess) return MDC_ERR_CUDA;
    // from the first copy on, every return marks the copies queued so far: the next use of this slot
    // waits for them before it overwrites the pinned index list they read
    bool queued = cudaMemcpyAsync(h.idx[s], h.idx_pinned[s], (size_t)nb * sizeof(int32_t), cudaMemcpyHostToDevice,
                                  h.copy) == cudaSuccess;
    const size_t row = (size_t)p->nv * p->nt;
    for (int b = 0; queued && b < nb;) {
        int e = b + 1;
        while (e < nb && idx_host[e] == idx_host[e - 1] + 1) ++e;   // consecutive sources: one copy
        queued = cudaMemcpyAsync(h.U[s] + (size_t)b * row, U_host + (size_t)idx_host[b] * row,
                                 (size_t)(e - b) * row * sizeof(float), cudaMemcpyHostToDevice, h.copy) == cudaSuccess;
        b = e;
    }
    const bool recorded = cudaEventRecord(h.copied[s], h.copy) == cudaSuccess;
    if (!queued || !recorded || cudaStreamWaitEvent(st, h.copied[s], 0) != cudaSuccess) return MDC_ERR_CUDA;
    rc = step_impl(p, X, h.U[s], h.idx[s], nb, prm->alpha, flags | SMDD_UOBS_GATHERED, nullptr, 0.f, nullptr,
                   loss_host ? h.loss[s] : nullptr, st);
    if (rc == MDC_OK && loss_host &&
        cudaMemcpyAsync(loss_host, h.loss[s], sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = MDC_ERR_CUDA;
    // recorded on failure too: whatever part of the step was queued still reads this slot
    if (cudaEventRecord(h.consumed[s], st) != cudaSuccess && rc == MDC_OK) rc = MDC_ERR_CUDA;
    return rc;
}

int smdd_step_ex(mdc_plan_t p, float *X, const float *U_obs, const int32_t *idx, int nb,
                 const smdd_step_ex_params *prm, double *loss, void *stream) {
    int rc = check_common(p, X, U_obs, idx, nb);
    if (rc) return rc;
    if (!prm) return MDC_ERR_INVALID_ARG;
    const int flags = prm->flags;
    if (flags & ~(SMDD_RECIPROCITY | SMDD_KEEP_XHAT | SMDD_REUSE_XHAT | SMDD_UOBS_GATHERED | SMDD_NESTEROV | SMDD_ADAM |
                  SMDD_SYMMETRIC))
        return MDC_ERR_INVALID_ARG;
    if (prm->reserved != 0) return MDC_ERR_INVALID_ARG;
    if (!std::isfinite(prm->alpha)) return MDC_ERR_INVALID_ARG;
    const bool nesterov = flags & SMDD_NESTEROV, adam = flags & SMDD_ADAM;
    if (nesterov && adam) return MDC_ERR_INVALID_ARG;
    if (nesterov && (!prm->V || !(prm->mu >= 0.f && prm->mu < 1.f))) return MDC_ERR_INVALID_ARG;
    if (adam && (!prm->V || !prm->S || prm->V == prm->S || prm->S == X || prm->t < 1 ||
                 !(prm->beta1 >= 0.f && prm->beta1 < 1.f) || !(prm->beta2 >= 0.f && prm->beta2 < 1.f) ||
                 !(prm->eps > 0.f) || !std::isfinite(prm->eps)))
        return MDC_ERR_INVALID_ARG;
    if (!nesterov && !adam && prm->V) return MDC_ERR_INVALID_ARG;
    if (!adam && (prm->S || prm->t != 0)) return MDC_ERR_INVALID_ARG;
    if (prm->V == X) return MDC_ERR_INVALID_ARG;
    if ((flags & SMDD_RECIPROCITY) && p->nr != p->nv) return MDC_ERR_SHAPE;
    AdamArgs ad;
    if (adam) {
        ad.m = prm->V;
        ad.v = prm->S;
        ad.beta1 = prm->beta1;
        ad.beta2 = prm->beta2;
        ad.eps = prm->eps;
        // bias corrections 1 / (1 - beta^t), formed in double and rounded once
        ad.c1 = (float)(1.0 / (1.0 - std::pow((double)prm->beta1, (double)prm->t)));
        ad.c2 = (float)(1.0 / (1.0 - std::pow((double)prm->beta2, (double)prm->t)));
    }
    DeviceGuard dg(p->device);
    return step_impl(p, X, U_obs, idx, nb, prm->alpha, flags & ~(SMDD_NESTEROV | SMDD_ADAM), nesterov ? prm->V : nullptr,
                     nesterov ? prm->mu : 0.f, prm->mute, loss, (cudaStream_t)stream, ad);
}

int mdc_plan_set_band(mdc_plan_t p, int nf_active) {
    if (!p || nf_active < 0) return MDC_ERR_INVALID_ARG;
    p->nf_active = (nf_active == 0 || nf_active >= p->nf) ? 0 : nf_active;
    p->xhat_for = nullptr;
    return MDC_OK;
}

int mdc_plan_set_wait_probe(mdc_plan_t p, long long cycles) {
    if (!p || cycles < 0 || cycles > 100000000LL) return MDC_ERR_INVALID_ARG;
    p->wait_probe = cycles;
    return MDC_OK;
}

int mdc_plan_get_config(mdc_plan_t p, mdc_config *cfg) {
    if (!p || !cfg) return MDC_ERR_INVALID_ARG;
    memset(cfg, 0, sizeof(*cfg));
    cfg->fft_variant = p->fft_variant;
    cfg->fft_prefetch = p->fft_prefetch;
    cfg->gemm_fwd = p->gemm_fwd;
    cfg->gemm_adj = p->gemm_adj;
    return MDC_OK;
}

int mdc_plan_set_config(mdc_plan_t p, const mdc_config *cfg) {
    if (!p || !cfg) return MDC_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i)
        if (cfg->reserved[i] != 0) return MDC_ERR_INVALID_ARG;
    if (cfg->fft_variant < 0 || cfg->fft_variant > 2) return MDC_ERR_INVALID_ARG;
    if (cfg->fft_prefetch != 0 && cfg->fft_prefetch != 1) return MDC_ERR_INVALID_ARG;
    if (cfg->gemm_fwd != MDC_GEMM_SIMT && cfg->gemm_fwd != MDC_GEMM_TC && cfg->gemm_fwd != MDC_GEMM_GEMV &&
        cfg->gemm_fwd != MDC_GEMM_TC_STREAM)
        return MDC_ERR_INVALID_ARG;
    if (cfg->gemm_adj < MDC_GEMM_SIMT || cfg->gemm_adj > MDC_GEMM_GEMV) return MDC_ERR_INVALID_ARG;
    if ((cfg->gemm_fwd == MDC_GEMM_GEMV || cfg->gemm_adj == MDC_GEMM_GEMV) && !gemv_supported(p->nv))
        return MDC_ERR_UNSUPPORTED;
    if ((cfg->gemm_fwd == MDC_GEMM_TC || cfg->gemm_fwd == MDC_GEMM_TC_STREAM || cfg->gemm_adj == MDC_GEMM_TC) &&
        p->prec != MDC_PREC_BF16X3)
        return MDC_ERR_UNSUPPORTED;
    if (cfg->gemm_fwd == MDC_GEMM_TC_STREAM && !p->xh_map_ok) return MDC_ERR_UNSUPPORTED;
    // the spectra a plan holds are the same for both radix orders: switching keeps them valid
    p->fft_variant = fft_has_variant(p->M, cfg->fft_variant) ? cfg->fft_variant : 0;
    p->fft_prefetch = (fft_pf_supported(p->M) && p->fft_variant != 2) ? cfg->fft_prefetch : 0;
    p->gemm_fwd = cfg->gemm_fwd;
    p->gemm_adj = cfg->gemm_adj;
    return MDC_OK;
}

int mdc_plan_autotune(mdc_plan_t p, int nb, int flags, int reps, mdc_config *best, void *stream) {
    if (!p || nb < 1 || reps < 1) return MDC_ERR_INVALID_ARG;
    if (nb > p->nbmax) return MDC_ERR_SHAPE;
    if (flags & ~(SMDD_RECIPROCITY | SMDD_KEEP_XHAT | SMDD_REUSE_XHAT | SMDD_UOBS_GATHERED | SMDD_SYMMETRIC))
        return MDC_ERR_INVALID_ARG;
    const bool recip = flags & SMDD_RECIPROCITY;
    if (recip && p->nr != p->nv) return MDC_ERR_SHAPE;
    if (reps > 100) reps = 100;
    DeviceGuard dg(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return MDC_ERR_INVALID_ARG;

    // scratch: a source list (sources 0, 1, ... cycling through ns) and a subset of model traces
    const long long trace_bytes = (long long)p->nr * p->nt * (long long)sizeof(float);
    const int nv_sub = (int)std::max(1LL, std::min((long long)p->nv, (64LL << 20) / std::max(1LL, trace_bytes)));
    int32_t *didx = nullptr;
    float *xs = nullptr, *us = nullptr;   // model-trace subset; gathered observed rows of one batch
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MDC_OK;
    std::vector<int32_t> hidx(nb);
    for (int i = 0; i < nb; ++i) hidx[i] = i % p->ns;
    const size_t u_bytes = (size_t)nb * p->nv * p->nt * sizeof(float);
    if (cudaMalloc(&didx, nb * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&xs, (size_t)nv_sub * trace_bytes) != cudaSuccess || cudaMalloc(&us, u_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(didx);
        cudaFree(xs);
        cudaFree(us);
        return MDC_ERR_OOM;
    }
    if (cudaMemcpyAsync(didx, hidx.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(xs, 0, (size_t)nv_sub * trace_bytes, st) != cudaSuccess ||
        cudaMemsetAsync(us, 0, u_bytes, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = MDC_ERR_CUDA;

    // mean device time of reps launches of fn after one warm-up launch; < 0 on failure
    auto time_it = [&](auto &&fn) -> double {
        if (fn() != MDC_OK) return -1.0;
        if (cudaEventRecord(e0, st) != cudaSuccess) return -1.0;
        for (int i = 0; i < reps; ++i)
            if (fn() != MDC_OK) return -1.0;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
        return (double)ms / reps;
    };
    const bool profiling = p->profiling;
    p->profiling = false;
    const int old_v = p->fft_variant, old_f = p->gemm_fwd, old_a = p->gemm_adj, old_pf = p->fft_prefetch;
    int best_v = old_v, best_f = old_f, best_a = old_a;
    if (rc == MDC_OK) {
        // FFT radix order, on the fused update (inverse + forward transform of every trace)
        double tbest = 1e300;
        int best_pf = 0;
        for (int cand = 0; cand < 5 && rc == MDC_OK; ++cand) {
            const int v = cand < 2 ? cand : cand < 4 ? cand - 2 : 2, pf = (cand >= 2 && cand < 4) ? 1 : 0;
            if (!fft_has_variant(p->M, v) || (pf && !fft_pf_supported(p->M))) continue;
            p->fft_variant = v;
            p->fft_prefetch = pf;
            // a step's two trace kernels: the fused update (scaled from the model subset to every model
            // trace) and the residual step of one batch
            const double tu = time_it([&] {
                FftArgs a = base_fft(p);
                a.g = model_grid(p, nv_sub);
                a.tout = xs;
                a.vec = vec4_ok(p->nt, xs);
                a.spec = p->Xh;
                a.alpha = 0.f;
                return launch_stage(p, ST_UPDATE, st, [&] { return launch_update(p->M, true, a, st); });
            });
            const double tr = tu < 0 ? -1.0 : time_it([&] {
                FftArgs a = base_fft(p);
                a.g = batch_grid(p, nb);
                a.spec = p->Uh;
                a.uobs = us;
                a.idx = didx;
                a.ns = p->ns;
                a.gathered = 1;
                a.uo_si = (long long)p->nv * p->nt;
                a.uo_sj = p->nt;
                a.vec = vec4_ok(p->nt, us);
                a.partials = p->partials;
                a.counter = p->counter;
                a.loss = nullptr;
                return launch_stage(p, ST_RESID, st, [&] { return launch_residual(p->M, a, p->resid_blocks_max, st); });
            });
            const double t = (tu < 0 || tr < 0) ? -1.0 : tu * ((double)p->nv / nv_sub) + tr;
            if (t < 0) rc = MDC_ERR_CUDA;
            else if (t < tbest) { tbest = t; best_v = v; best_pf = pf; }
        }
        p->fft_variant = best_v;
        p->fft_prefetch = best_pf;
    }
    if (rc == MDC_OK) {
        double tbest = 1e300;
        const int cand[4] = {MDC_GEMM_SIMT, MDC_GEMM_TC, MDC_GEMM_TC_STREAM, MDC_GEMM_GEMV};
        for (int c : cand) {
            if ((c == MDC_GEMM_TC || c == MDC_GEMM_TC_STREAM) && p->prec != MDC_PREC_BF16X3) continue;
            if (c == MDC_GEMM_TC_STREAM && !p->xh_map_ok) continue;
            if (c == MDC_GEMM_GEMV && !gemv_supported(p->nv)) continue;
            p->gemm_fwd = c;
            const double t = time_it([&] { return gemm_forward(p, didx, nb, st); });
            if (t < 0) { rc = MDC_ERR_CUDA; break; }
            if (t < tbest) { tbest = t; best_f = c; }
        }
    }
    if (rc == MDC_OK) {
        double tbest = 1e300;
        const int cand[4] = {MDC_GEMM_SIMT32, MDC_GEMM_SIMT64, MDC_GEMM_TC, MDC_GEMM_GEMV};
        for (int c : cand) {
            if (c == MDC_GEMM_TC && p->prec != MDC_PREC_BF16X3) continue;
            if (c == MDC_GEMM_GEMV && (!gemv_supported(p->nv) || recip)) continue;
            p->gemm_adj = c;
            const double t = time_it([&] { return gemm_adjoint(p, didx, nb, recip, st); });
            if (t < 0) { rc = MDC_ERR_CUDA; break; }
            if (t < tbest) { tbest = t; best_a = c; }
        }
    }
    p->profiling = profiling;
    p->xhat_for = nullptr;   // the spectral workspaces were overwritten
    if (rc == MDC_OK) {
        p->fft_variant = best_v;
        p->gemm_fwd = best_f;
        p->gemm_adj = best_a;
    } else {
        p->fft_variant = old_v;
        p->fft_prefetch = old_pf;
        p->gemm_fwd = old_f;
        p->gemm_adj = old_a;
    }
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(didx);
    cudaFree(xs);
    cudaFree(us);
    if (rc == MDC_OK && best) mdc_plan_get_config(p, best);
    return rc;
}

int mdc_plan_sync_status(mdc_plan_t p) {
    if (!p) return MDC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return MDC_ERR_CUDA;
    int h = 0;
    if (cudaMemcpy(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MDC_ERR_CUDA;
    if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return MDC_ERR_CUDA;
    return (h & 2) ? MDC_ERR_TIMEOUT : (h & 1) ? MDC_ERR_INDEX_RANGE : MDC_OK;
}

int mdc_plan_set_profiling(mdc_plan_t p, int enable) {
    if (!p) return MDC_ERR_INVALID_ARG;
    p->profiling = enable != 0;
    return MDC_OK;
}

int mdc_plan_stage_times(mdc_plan_t p, double *ms, long long *launches, int reset) {
    if (!p) return MDC_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    for (auto &t : p->pending) {
        if (cudaEventSynchronize(t.e1) != cudaSuccess) return MDC_ERR_CUDA;
        float el = 0.f;
        if (cudaEventElapsedTime(&el, t.e0, t.e1) != cudaSuccess) return MDC_ERR_CUDA;
        p->stage_ms[t.stage] += el;
        p->event_pool.push_back(t.e0);
        p->event_pool.push_back(t.e1);
    }
    p->pending.clear();
    for (int s = 0; s < MDC_NUM_STAGES; ++s) {
        if (ms) ms[s] = p->stage_ms[s];
        if (launches) launches[s] = p->stage_launches[s];
        if (reset) {
            p->stage_ms[s] = 0.0;
            p->stage_launches[s] = 0;
        }
    }
    return MDC_OK;
}

long long mdc_plan_launch_count(mdc_plan_t p) { return p ? p->launches : -1; }

}  // extern "C"
