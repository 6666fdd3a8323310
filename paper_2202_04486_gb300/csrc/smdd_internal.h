// Internal declarations shared by the translation units of libsmdd_gb300.so (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "../../include/smdd.h"

namespace smdd {

enum Stage { ST_RFFT = 0, ST_GEMM_FWD = 1, ST_RESID = 2, ST_GEMM_ADJ = 3, ST_UPDATE = 4, ST_IRFFT_OUT = 5, ST_SETUP = 6 };

// A 2-D grid of time traces and the matching spectra.  Trace (i, j), i < ni, j < nj:
//   time samples at  tin/tout + i*tsi + j*tsj + t          (floats),  t < nt
//   spectrum bin f at spec + f*ssf + i*ssi + j*ssj           (float2), f <= M
// A CTA owns TR traces: 2^ti_log2 consecutive i times TR >> ti_log2 consecutive j.
struct TraceGrid {
    int ni, nj, ti_log2;
    long long tsi, tsj;
    long long ssi, ssj, ssf;
    // 1: only the tiles on or above the block diagonal of a square grid (ni == nj, CTAs of TR traces along
    // i): tile (bi, j) for bi >= j / TR, bi fastest (a symmetric model, see sym_tile_to_full)
    int sym = 0;
};

struct FftArgs {
    TraceGrid g;
    int nt;
    int vec;                 // time traces may be accessed as float4 (nt % 4 == 0, 16-byte aligned base)
    const float *tin;        // time input (rfft)
    float *tout;             // time output (irfft_out) / model in-out (update)
    float2 *spec;            // spectra (read and/or written)
    const float2 *tw;        // per-pass twiddle tables (see tw_off)
    const float2 *twN;       // exp(-2 pi i k / N), k <= M
    float s;                 // epilogue factor scale / N
    float alpha;             // step size (update)
    // residual: observed rows, row(i) = gathered ? i : idx[i]
    const float *uobs;
    const int32_t *idx;
    int ns, gathered;
    long long uo_si, uo_sj;
    double *partials;
    unsigned int *counter;
    double *loss;
    int *status;
    int variant;             // FFT variant: 0 / 1 radix orders of fft_radix, 2 the two-pass FFT (smdd_fft2.cuh)
    // update: Nesterov velocity (null for SGD), momentum, causality mute (first kept sample per
    // model trace, [nv][nr]; null for none)
    float *vel;
    float mu;
    const int32_t *mute;
    // update: Adam moments (null for SGD / N-SGD), decay rates, epsilon and the bias corrections
    // c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t) of step t
    float *adam_m, *adam_v;
    float beta1, beta2, eps, c1, c2;
    int prefetch;            // update: persistent CTAs prefetching the next tile's spectra (M <= 1024)
};

struct GemmArgs {
    const float2 *A;         // forward: model spectra Xh; adjoint: residual spectra Rh
    const float2 *Dh;        // kernel spectra [nf][ns][ldr]
    const int32_t *idx;
    float2 *C;               // forward: Uh; adjoint: Gh
    int nv, nr, ns, nb, ldr, ldb;
    long long sAf, sDf, sCf; // per-frequency strides (float2)
    float outscale;
    int tiles_v, tiles_r;    // adjoint tile grid
    int *status;
    int nf_active;           // band limit: bins f >= nf_active (when > 0) get zero products
    long long wait_probe;    // tensor-core kernels: > 0 = failure-path check (mdc_plan_set_wait_probe), cycles
    int sym_tr;              // forward: > 0 when A holds a symmetric model's spectra only on and above the
                             // sym_tr-block diagonal: element (v, r) with r < sym_tr floor(v / sym_tr) is read
                             // at (r, v)
    const uint8_t *img;      // adjoint, split-BF16 tile kernel: the operand images of k_tc_adj_images (or null:
    int img_nkc;             // the kernel splits its operands itself), their K chunks (32 batch entries each)
    int no_mirror;           // adjoint with reciprocity: skip the mirrored copy of the off-diagonal tiles (the
                             // update of a symmetric model reads the upper tiles and the diagonal ones only;
                             // a diagonal tile still mirrors its upper half, so it stays exactly symmetric)
};

// Zero the output tile [r0, r0+nrows) x [c0, c0+ncols) of a CTA whose frequency bin lies above the
// band limit (inside the matrix bounds rmax x cmax; leading dimension ld).
__device__ __forceinline__ void zero_tile(float2 *C, long long ld, int r0, int nrows, int c0, int ncols, int rmax,
                                          int cmax) {
    for (int e = threadIdx.x; e < nrows * ncols; e += blockDim.x) {
        const int i = e / ncols, j = e % ncols, r = r0 + i, c = c0 + j;
        if (r < rmax && c < cmax) C[(long long)r * ld + c] = make_float2(0.f, 0.f);
    }
}

// A device work queue over the tiles of one kernel's launches for several problems (the work-queue
// epochs of the many-problem runner): item w < total belongs to member m with start[m] <= w < start[m+1]
// and is tile w - start[m] of that member's launch.  The persistent queue kernels take items in order by
// an atomic add on *counter, which must be zero before the launch.
struct WorkQueue {
    const void *args;        // device array of n argument records (FftArgs or GemmArgs)
    const int *start;        // device [n + 1]: exclusive prefix sums of the members' tile counts
    int n, total;
    unsigned int *counter;
};

// Symmetric model: X^[f][v][r] <- X^[f][r][v] for every r < TR floor(v / TR) (the part of the spectra below
// the TR-block diagonal, which the update of a symmetric model leaves unwritten); n = nr = nv
cudaError_t launch_mirror_lower(float2 *spec, int n, int ld, long long ssf, int nf, int TR, cudaStream_t st);
// Number of tiles of the upper enumeration of a square grid of n x n traces with TR traces per CTA along
// i: row j holds the tiles bi = j / TR .. ceil(n / TR) - 1.
__host__ __device__ inline long long sym_tiles(int n, int TR) {
    const long long nbi = (n + TR - 1) / TR, full = n / TR, rem = n % TR;
    // groups g < full of TR rows with nbi - g tiles each, then rem rows of nbi - full tiles
    return (long long)TR * (full * nbi - full * (full - 1) / 2) + rem * (nbi - full);
}

// FFT lengths of the trace kernels: powers of two 64 .. 8192 and 3072 (api.cu)
bool nfft_supported(int nfft);
int default_nfft(int nt);   // the shortest supported length >= max(2 nt - 1, 64)

// launchers (return cudaError_t of the launch)
cudaError_t launch_rfft(int M, const FftArgs &a, cudaStream_t st);
cudaError_t launch_irfft_out(int M, const FftArgs &a, cudaStream_t st);
cudaError_t launch_residual(int M, const FftArgs &a, int nblocks_expected, cudaStream_t st);
cudaError_t launch_update(int M, bool keep_xhat, const FftArgs &a, cudaStream_t st);
int fft_blocks(int M, const TraceGrid &g);
int fft_traces_per_cta(int M);
bool fft_pf_supported(int M);   // the persistent prefetching update exists for complex length M
cudaError_t fft_prepare(int M);                                // opt-in to the dynamic shared memory of size M
int fft_tw_size(int M, int variant = 0);
bool fft_has_variant(int M, int variant);                     // variant 1 exists where it differs from 0
void fft_tw_fill(int M, std::vector<float2> &tw, int variant = 0);   // host: per-pass twiddle tables

// register FFT kernels (radix-order variant 2: two passes for 128 <= M <= 1024, three for M = 1536;
// fft2_kernels.cu)
bool fft2_supported(int M);
int fft2_traces_per_cta(int M);
int fft2_blocks(int M, const TraceGrid &g);
int fft2_tw_size(int M);                             // entries of the variant's twiddle tables
void fft2_tw_fill(int M, std::vector<float2> &tw);   // host: the variant's twiddle tables
cudaError_t fft2_prepare(int M);
cudaError_t launch2_rfft(int M, const FftArgs &a, cudaStream_t st);
cudaError_t launch2_irfft_out(int M, const FftArgs &a, cudaStream_t st);
cudaError_t launch2_residual(int M, const FftArgs &a, int nblocks_expected, cudaStream_t st);
cudaError_t launch2_update(int M, bool keep_xhat, const FftArgs &a, cudaStream_t st);

// work-queue forms of the trace kernels (rfft, residual step, SGD update with the new model's spectra),
// for FFT variant 0, 1 (radix orders) or 2 (register FFT): CTAs resident on every SM, each taking tiles
// from the queue until it is empty.  Tile counts per member: fft_blocks / fft2_blocks of its grid.
cudaError_t launch_queue_rfft(int M, int variant, const WorkQueue &q, cudaStream_t st);
cudaError_t launch_queue_residual(int M, int variant, const WorkQueue &q, cudaStream_t st);
cudaError_t launch_queue_update(int M, int variant, const WorkQueue &q, cudaStream_t st);
cudaError_t launch2_queue_rfft(int M, const WorkQueue &q, cudaStream_t st);
cudaError_t launch2_queue_residual(int M, const WorkQueue &q, cudaStream_t st);
cudaError_t launch2_queue_update(int M, const WorkQueue &q, cudaStream_t st);

cudaError_t launch_cgemm_fwd(const GemmArgs &a, int nf, cudaStream_t st);
cudaError_t launch_cgemm_adj(const GemmArgs &a, bool recip, int nf, cudaStream_t st, int tile = 0);
cudaError_t gemm_prepare();
// few virtual sources (nv <= 8): matrix-vector kernels; no band limit, no reciprocity (adjoint)
bool gemv_supported(int nv);
cudaError_t launch_gemv_fwd(const GemmArgs &a, int nf, cudaStream_t st);
cudaError_t launch_gemv_adj(const GemmArgs &a, int nf, cudaStream_t st);

// split-BF16 tensor-core products (tcgen05)
cudaError_t tc_prepare();
cudaError_t launch_tc_fwd(const GemmArgs &a, int nf, cudaStream_t st);
// streamed forward product fed by the tensor memory accelerator: map = 128-byte tensor map of the
// model spectra written by tc_encode_fwd_map (64-byte aligned host memory)
cudaError_t tc_encode_fwd_map(void *map_out, const float2 *Xh, int nr, int nv, int ldr, int nf);
cudaError_t launch_tc_fwd_stream(const GemmArgs &a, const void *map, int nf, cudaStream_t st);
// map (or null): the 128-byte tensor map of the output (tc_encode_fwd_map of the model-spectra buffer):
// the tile without reciprocity is then written by the tensor memory accelerator
cudaError_t launch_tc_adj(const GemmArgs &a, bool recip, int nf, cudaStream_t st, const void *map = nullptr);
// Operand images of the split-BF16 adjoint (bytes for a problem; 0 where the batch needs more than two K
// chunks), and their construction for one step (residual spectra and gathered kernel rows of a.idx).
size_t tc_adj_image_bytes(int nv, int nr, int nb, int nf);
cudaError_t launch_tc_adj_images(const GemmArgs &a, uint8_t *img, int nf, cudaStream_t st);
// work-queue forms of the tensor-core tile products (persistent CTAs, TMEM allocated once per CTA);
// tile counts per problem: tc_fwd_tiles (NB = tc_fwd_queue_nb(nb) for every member of a launch),
// tc_adj_tiles (which also sets the record's tiles_v / tiles_r)
int tc_fwd_queue_nb(int nb);
int tc_fwd_tiles(const GemmArgs &a, int nf);
int tc_adj_tiles(GemmArgs &a, bool recip, int nf);
cudaError_t launch_tc_fwd_queue(int NB, const WorkQueue &q, cudaStream_t st);
cudaError_t launch_tc_adj_queue(bool recip, const WorkQueue &q, cudaStream_t st);

// plan internals used by the batch runner (api.cu)
struct PlanShape {
    int nt, nr, nv, ns, nbmax, nfft, nf, prec, device;
};

// The launches of one SGD step of a plan (smdd_step with KEEP_XHAT, and REUSE_XHAT unless `first`) as
// argument records with their tile counts, for the work-queue epochs: the model transform (used on the
// first step only), the forward product on the tensor-core tile kernel with batch block fwd_nb, the
// residual step, the adjoint product (tile kernel, reciprocity flag) and the update.  The trace kernels
// run FFT variant `variant` of complex length M.  Returns MDC_ERR_UNSUPPORTED unless the plan's products
// run on the tensor cores (MDC_PREC_BF16X3 with MDC_GEMM_TC or MDC_GEMM_TC_STREAM forward and
// MDC_GEMM_TC adjoint) and no band limit is set.
struct StepRecords {
    int M, variant;
    FftArgs rfft;
    int rfft_tiles;
    GemmArgs fwd;
    int fwd_nb, fwd_tiles;
    FftArgs resid;
    int resid_tiles;
    GemmArgs adj;
    int adj_tiles;
    bool recip;
    FftArgs upd;
    int upd_tiles;
};
int plan_step_records(mdc_plan_s *p, float *X, const float *U_obs, const int32_t *idx, int nb, float alpha, int flags,
                      double *loss, StepRecords *r);
PlanShape plan_shape(const mdc_plan_s *p);
bool plan_begin_capture(mdc_plan_s *p);               // returns the profiling flag it switched off
void plan_end_capture(mdc_plan_s *p, bool profiling);

// LSQR workspace (owned by a plan, allocated on first use) and the iteration (lsqr.cu)
struct LsqrWork {
    float *u = nullptr, *t = nullptr;           // data-size vectors [ns][nv][nt]
    float *v = nullptr, *w = nullptr, *g = nullptr;   // model-size vectors [nv][nr][nt]
    int32_t *idx = nullptr;                     // 0 .. ns-1
    double *partials = nullptr;
    void *scalars = nullptr;
    long long nd = 0, nm = 0;
    cudaError_t ensure(long long n_data, long long n_model, int ns);
    void release();
    ~LsqrWork();
};
using OperatorFn = std::function<cudaError_t(const float *, float *)>;
cudaError_t lsqr_run(LsqrWork &wk, float *x, const float *b, long long nd, long long nm, int nt, int n_iter,
                     const int32_t *mute, double *norms, cudaStream_t st, const OperatorFn &apply_fwd,
                     const OperatorFn &apply_adj, long long *launches);

cudaError_t launch_power_iter(const float2 *Dh, int ns, int nr, int ldr, long long sDf, int nf, int n_iter,
                              double *lam, cudaStream_t st);
cudaError_t launch_max_reduce(const double *lam, int n, double *out, cudaStream_t st);

}  // namespace smdd
