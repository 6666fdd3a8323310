/*
 * smdd.h -- C ABI of the GB300 (sm_103a) stochastic multi-dimensional deconvolution hot path.
 *
 * The operator is the time-domain multi-dimensional convolution (MDC) of Ravasi, Selvan & Luiken,
 * "Stochastic Multi-Dimensional Deconvolution" (arXiv 2202.04486): Eq. 1-2 written in the time domain
 * (the operator P+_t of Eq. 3), applied to a batch of sources (Eq. 5), its adjoint (the
 * cross-correlation of the Synthetic OBC section), and one SGD step on the mini-batch gradient of
 * Eq. 6 with the optional reciprocity preconditioner C_r of Eq. 4.  Appendix A gives the evaluation
 * order used here: FFT along time, one complex matrix product per frequency, inverse FFT.
 *
 * Array conventions.  All arrays are float32, C order, time axis fastest:
 *   D     [ns][nr][nt]  down-going wavefield p+ (source s, receiver r)
 *   X     [nv][nr][nt]  reflection response r_t (virtual source v, receiver r)
 *   U_obs [ns][nv][nt]  observed up-going wavefield p- (source s, virtual source v)
 *   U     [nb][nv][nt]  MDC output for the sources idx[0..nb)
 *   R     [nb][nv][nt]  residual / adjoint input for the sources idx[0..nb)
 *   G     [nv][nr][nt]  adjoint output
 * with
 *   U[b][v][t] = scale * sum_r sum_{tau=0..t} D[idx[b]][r][tau] * X[v][r][t-tau]          (forward)
 *   G[v][r][tau] = scale * sum_b sum_{t=tau..nt-1} D[idx[b]][r][t-tau] * R[b][v][t]       (adjoint)
 * i.e. causal linear convolution truncated to the nt recorded samples (the FFT length nfft is at
 * least 2*nt-1, so no circular wrap-around reaches [0, nt)).
 *
 * Memory and streams.  Every array pointer is DEVICE memory owned by the caller unless stated
 * otherwise; the plan owns its own workspaces (spectrum of D, model/gradient spectra, batch spectra).
 * Calls are asynchronous on the given stream (a cudaStream_t passed as void*; NULL is the legacy
 * default stream).  A plan must not be used by two calls that may overlap on the GPU (its workspaces
 * are shared); issue all calls on one plan to one stream, or order the streams.
 *
 * Errors.  Every call returns an mdc_status.  Host-detectable errors (null pointers, bad sizes,
 * nb > nb_max, shape mismatch for reciprocity) are returned immediately and nothing is launched.
 * Device-detected errors (a source index outside [0, ns)) are recorded in the plan's status word:
 * the offending rows are treated as zero and the error is returned by mdc_plan_sync_status().
 * Nothing traps and no C++ exception crosses this interface.
 */
#ifndef SMDD_H
#define SMDD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdc_plan_s *mdc_plan_t;

typedef enum {
    MDC_OK = 0,
    MDC_ERR_INVALID_ARG = 1,   /* null pointer, non-positive size, bad flag */
    MDC_ERR_SHAPE = 2,         /* e.g. reciprocity requested with nr != nv, nb > nb_max */
    MDC_ERR_INDEX_RANGE = 3,   /* a source index outside [0, ns) was seen on the device */
    MDC_ERR_OOM = 4,           /* device allocation failed in mdc_plan_create */
    MDC_ERR_CUDA = 5,          /* a CUDA runtime call or kernel launch failed */
    MDC_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (tensor-core products) */
    MDC_ERR_UNSUPPORTED = 7    /* size outside the supported range (nt > 4096, an unsupported nfft) */
} mdc_status;

/* Arithmetic of the per-frequency products (the FFTs are FP32 in both):
 *   MDC_PREC_FP32   : FP32 FMA on the CUDA cores.
 *   MDC_PREC_BF16X3 : tensor cores (tcgen05); each FP32 operand is split into BF16 hi + lo and every real
 *                     product is taken as hi*hi + hi*lo + lo*hi with FP32 accumulation (about 16
 *                     significant bits per operand; relative L2 error of the operator ~1e-5). */
typedef enum { MDC_PREC_FP32 = 0, MDC_PREC_BF16X3 = 1 } mdc_precision;

/* Create a plan for one MDD problem and precompute the spectrum of the down-going wavefield
 * (Appendix A: the kernel is transformed once; the per-frequency matrices Dh_f are ns x nr).
 *   out     : receives the plan handle (host pointer).
 *   nt      : time samples per trace, 1 <= nt <= 4096.
 *   nr, nv, ns : receivers, virtual sources, sources (>= 1).
 *   nb_max  : largest batch size later passed to any call (1 <= nb_max <= 1024; 0 means ns).
 *   nfft    : FFT length; 0 picks the shortest supported length >= max(2*nt-1, 64).  Supported: the
 *             powers of two 64 .. 8192 and 3072 = 3 * 2^10 (chosen for 1025 <= nt <= 1536, where the
 *             power of two would be 4096).  A non-zero value must be supported and >= 2*nt-1.
 *   scale   : multiplies the operator (the discretisation of the receiver integral in Eq. 1; 1 is a
 *             plain sum over receivers).
 *   D       : device pointer, [ns][nr][nt] float32, read during this call only.
 *   precision : MDC_PREC_FP32 or MDC_PREC_BF16X3 (see mdc_precision).
 *   stream  : stream for the precompute; the call returns after it has been enqueued.
 * Allocates about 8*nf*(ns+nv)*nr + 8*nf*nv*nb_max bytes of device memory (nf = nfft/2+1). */
int mdc_plan_create(mdc_plan_t *out, int nt, int nr, int nv, int ns, int nb_max, int nfft,
                    float scale, const float *D, int precision, void *stream);

/* Release a plan and its device memory (synchronises the device first).  NULL is accepted. */
int mdc_plan_destroy(mdc_plan_t plan);

/* Sizes chosen by the plan: FFT length and number of frequency bins (nfft/2+1).  Host pointers,
 * either may be NULL. */
int mdc_plan_info(mdc_plan_t plan, int *nfft, int *nf);

/* Largest squared singular value of the frequency-domain kernel, max over bins f of
 * lambda_max(Dh_f^H Dh_f) * scale^2, by n_iter power iterations per bin (Appendix B: the singular
 * values of the MDC operator are those of the kernel; alpha_max = 2 / sigma^2 for the Landweber
 * iteration).  The result is a lower bound of the exact value that converges as n_iter grows (the
 * products run in FP32, the norms in FP64: the rounding moves it by ~1e-6 relative).  Needs
 * (2*nr + ns) * 8 bytes of shared memory per bin (MDC_ERR_UNSUPPORTED above 227 KiB).
 * Blocks until the value is on the host.  sigma2 is a host pointer. */
int mdc_plan_sigma2_max(mdc_plan_t plan, int n_iter, double *sigma2, void *stream);

/* Forward MDC for a batch of sources (Eq. 1-3 in the time domain, one batch of Eq. 5).
 *   X : [nv][nr][nt] device float32.  idx : device int32[nb], entries in [0, ns), duplicates allowed.
 *   U : [nb][nv][nt] device float32, written.  1 <= nb <= nb_max. */
int mdc_forward(mdc_plan_t plan, const float *X, const int32_t *idx, int nb, float *U, void *stream);

/* Adjoint MDC (cross-correlation with the down-going field; the operator P+^H of Eq. 6).
 *   R : [nb][nv][nt] device float32.  idx as for mdc_forward.  G : [nv][nr][nt] device float32, written. */
int mdc_adjoint(mdc_plan_t plan, const float *R, const int32_t *idx, int nb, float *G, void *stream);

/* smdd_params.flags */
#define SMDD_RECIPROCITY    1   /* apply C_r: the step uses 1/2 (g + g^T) (needs nr == nv) */
#define SMDD_KEEP_XHAT      2   /* after the update, leave the spectrum of the new X in the plan */
#define SMDD_REUSE_XHAT     4   /* start from the spectrum left by the previous KEEP_XHAT step on the
                                   same X pointer (the caller promises X was not modified in between;
                                   ignored if the plan holds no spectrum for this pointer) */
#define SMDD_UOBS_GATHERED  8   /* U_obs is [nb][nv][nt]: the batch rows, already gathered */
#define SMDD_SYMMETRIC      64  /* with SMDD_RECIPROCITY (smdd_step, smdd_step_host, smdd_step_ex, batched epochs):
                                   the caller promises X[v][r] == X[r][v] on entry, and the same of the N-SGD
                                   velocity or the Adam moments (zero starts) -- a symmetric start stays
                                   symmetric under C_r (Eq. 4, X = C_r z) -- so the update transforms only the traces on
                                   and above the diagonal (in blocks of the FFT kernels' traces per CTA) and
                                   writes each result to both (v, r) and (r, v); the result is identical to the
                                   step without the flag on a symmetric X.  On a non-symmetric X the lower
                                   triangle is overwritten by the mirrored upper one.  Without
                                   SMDD_RECIPROCITY it is ignored. */

typedef struct {
    float alpha;        /* step size (Appendix B: a fraction of 2 / sigma^2) */
    int flags;          /* SMDD_* bits */
    int reserved[6];    /* must be zero */
} smdd_params;

/* One stochastic MDD step on the batch idx (Eq. 6 and the SGD update):
 *   R = P_B X - U_obs[idx],  loss = 1/2 ||R||^2 (accumulated in float64),
 *   g = P_B^H R,  X <- X - alpha * C(g),  C = C_r (reciprocity flag) or the identity.
 *   X     : [nv][nr][nt] device float32, updated in place.
 *   U_obs : [ns][nv][nt] (or [nb][nv][nt] with SMDD_UOBS_GATHERED) device float32.
 *   idx   : device int32[nb].   params : host pointer.
 *   loss  : device float64 scalar written with 1/2 ||R||^2, or NULL. */
int smdd_step(mdc_plan_t plan, float *X, const float *U_obs, const int32_t *idx, int nb,
              const smdd_params *params, double *loss, void *stream);

/* smdd_step_host: the step of smdd_step with the batch taken from host memory (a data-loader step).
 *   U_obs_host : [ns][nv][nt] host float32 (pinned, for the copies to be asynchronous).
 *   idx_host   : host int32[nb]; checked on the host (MDC_ERR_INDEX_RANGE before anything is queued)
 *                and copied at once, so the caller may reuse it when the call returns.
 *   loss_host  : host float64 written asynchronously with 1/2 ||R||^2 (pinned memory; valid once
 *                `stream` has passed the step), or NULL.
 *   flags      : SMDD_RECIPROCITY, SMDD_KEEP_XHAT, SMDD_REUSE_XHAT, SMDD_SYMMETRIC.
 * The plan copies the index list and the nb rows U_obs_host[idx[b]] (consecutive sources as one copy)
 * into one of two device staging slots on a copy stream of its own, then queues the step on `stream`
 * behind them: the copies of a call overlap the step of the previous call, and a slot is refilled only
 * after the step two calls back has finished with it.  The rows of U_obs_host must stay unchanged until
 * the step has run.  The staging slots (2 nb_max nv nt floats) are allocated by the first call
 * (MDC_ERR_OOM if that fails). */
int smdd_step_host(mdc_plan_t plan, float *X, const float *U_obs_host, const int32_t *idx_host, int nb,
                   const smdd_params *params, double *loss_host, void *stream);

/* smdd_step_ex: the same step with the N-SGD solver, the Adam update and the causality preconditioner.
 * N-SGD is SGD with Nesterov momentum in the form of Sutskever et al. (2013) -- the solver the paper
 * reports as converging fastest -- written on the look-ahead point: with g the preconditioned batch
 * gradient evaluated at X,
 *   V <- mu V - alpha g,   X <- X + mu V - alpha g.
 * The causality preconditioner C_c of Eq. 4 (the space-time mask that mutes the reflection response
 * above the direct arrival) is a per-trace first kept sample: g is set to zero on samples
 * t < mute[v][r], so a model that starts zero there stays zero there.  The chain C = C_r C_c applies
 * reciprocity first; with SMDD_RECIPROCITY the mute table must be symmetric (mute[v][r] == mute[r][v]),
 * so that the two projections commute and X stays in the range of C. */
#define SMDD_NESTEROV       16  /* smdd_step_ex only: momentum with velocity state V */
/* Adam (Kingma & Ba 2015, Algorithm 1; the paper itself uses SGD and N-SGD) on the preconditioned batch
 * gradient g, element-wise, with moment arrays m = V and v = S and step count t >= 1:
 *   m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
 *   X <- X - alpha * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
 * The bias corrections are formed in double precision on the host and rounded to float once; the
 * element-wise arithmetic is float32.  Muted samples see g = 0, so a model and moments that start zero
 * there stay zero there; with reciprocity a symmetric start stays symmetric. */
#define SMDD_ADAM           32  /* smdd_step_ex only: Adam with moments V (first) and S (second) */

typedef struct {
    float alpha;            /* step size */
    int flags;              /* SMDD_* bits, SMDD_NESTEROV or SMDD_ADAM included */
    float mu;               /* momentum, 0 <= mu < 1 (SMDD_NESTEROV) */
    int t;                  /* SMDD_ADAM: step count, 1 for the first step (bias corrections); else 0 */
    float *V;               /* SMDD_NESTEROV: velocity; SMDD_ADAM: first moment m.  [nv][nr][nt] device
                               float32, updated in place (start from zeros); NULL otherwise; never X */
    const int32_t *mute;    /* causality mute: device int32[nv][nr], first kept sample per model trace; or NULL */
    float *S;               /* SMDD_ADAM: second moment v, [nv][nr][nt] device float32 (start from zeros),
                               distinct from X and V; NULL otherwise */
    float beta1, beta2;     /* SMDD_ADAM: moment decay rates in [0, 1) (Kingma & Ba: 0.9, 0.999) */
    float eps;              /* SMDD_ADAM: > 0, added to the root of the corrected second moment */
    int reserved;           /* zero */
} smdd_step_ex_params;

int smdd_step_ex(mdc_plan_t plan, float *X, const float *U_obs, const int32_t *idx, int nb,
                 const smdd_step_ex_params *params, double *loss, void *stream);

/* Full-gradient MDD by LSQR (Paige & Saunders 1982): the baseline the paper compares stochastic MDD
 * against (the Synthetic OBC example's "10 iterations of LSQR"), on the preconditioned operator
 * A = P C with P the MDC over every source (Eq. 3) and C = C_r C_c (Eq. 4; each optional):
 *   X     : [nv][nr][nt] device float32; the starting model on entry (it must lie in the range of C,
 *           e.g. zero), the LSQR solution after n_iter iterations on return.
 *   U_obs : [ns][nv][nt] device float32.
 *   flags : 0 or SMDD_RECIPROCITY.   mute : causality table as in smdd_step_ex, or NULL.
 *   norms : device float64[n_iter + 1] (or NULL): LSQR's estimates of ||U_obs - A X|| at the start and
 *           after every iteration.
 * The plan must have been made with nb_max >= ns (all sources form one batch).  Vectors are FP32, norms
 * and the recurrence FP64, all on the device: the call enqueues a fixed sequence of launches and does not
 * synchronise.  The first call allocates a workspace of 2 data-size and 3 model-size FP32 vectors, kept
 * by the plan until it is destroyed (that call must not be made during a stream capture). */
int smdd_lsqr(mdc_plan_t plan, float *X, const float *U_obs, int n_iter, int flags, const int32_t *mute,
              double *norms, void *stream);

/* Forward MDC without any device allocation (the paper has no counterpart: this exists for callers
 * that may not call cudaMalloc/cudaFree -- code whose device memory is owned by another allocator or
 * pool, or loops that cannot afford an allocation's latency and implicit synchronisation).
 * Computes the same U as mdc_forward on a plan made with the same nt, nr, nv, ns, scale and D, with
 * nfft the default length.  Every intermediate lives in one static 64 MiB device array that the library
 * holds on each device where this function has been used, until the process exits.
 *   D [ns][nr][nt], X [nv][nr][nt], idx int32[nb], U [nb][nv][nt]: device pointers owned by the caller.
 *   dev_status: device int, required (MDC_ERR_INVALID_ARG when NULL): set to 1 if an index lies outside
 *               [0, ns), whose rows of U are then zero; the caller zeroes it and reads it after the stream
 *               has passed the call.
 *   stream: as elsewhere.
 * Returns MDC_ERR_UNSUPPORTED, launching nothing, when the intermediates of the problem need more than
 * the 64 MiB: 8 * (nfft/2+1) * (ns*ldr + nv*ldr + nv*ldb) bytes plus the twiddle tables, with ldr and ldb
 * nr and nb rounded up to even.  Shapes are not checked here (there is no plan): the caller must pass
 * arrays of exactly the sizes above.
 * The first call on a device looks up the array's device address (once per device) and must therefore
 * not be the first call made during a stream capture.  All calls share the array: two calls that can
 * overlap on the GPU (other streams, other host threads) race with each other and must be serialised
 * by the caller. */
int mdc_forward_static(int nt, int nr, int nv, int ns, float scale, const float *D, const float *X,
                       const int32_t *idx, int nb, float *U, int *dev_status, void *stream);

/* ---------------------------------------------------------------------------------------------
 * Kernel configuration and autotuning.  Every configuration computes the same operator; they differ
 * in speed only.  The FFT radix order and the kernel of each per-frequency product are the choices.
 * A plan made with MDC_PREC_BF16X3 may run the FP32 FMA kernels for a product (they are more
 * accurate than the split-BF16 bound); the tensor-core kernels are allowed for such plans only.
 * ------------------------------------------------------------------------------------------- */
#define MDC_GEMM_SIMT    0   /* FP32 FMA kernels on the CUDA cores (adjoint: tile chosen by size) */
#define MDC_GEMM_SIMT32  1   /* adjoint only: FP32 FMA, 32 x 32 output tiles */
#define MDC_GEMM_SIMT64  2   /* adjoint only: FP32 FMA, 64 x 64 output tiles */
#define MDC_GEMM_TC      3   /* split-BF16 tcgen05 kernels (MDC_PREC_BF16X3 plans only) */
#define MDC_GEMM_GEMV    4   /* FP32 matrix-vector kernels for few virtual sources (nv <= 8): a warp or a
                                thread streams each gathered kernel row once.  Used where allowed: with
                                a band limit, and for the adjoint with reciprocity, the call runs
                                MDC_GEMM_SIMT instead. */
#define MDC_GEMM_TC_STREAM 5 /* forward only: the split-BF16 tcgen05 product as a persistent kernel (one
                                CTA per SM) fed by tiled copies of the tensor memory accelerator
                                (MDC_PREC_BF16X3 plans only; MDC_ERR_UNSUPPORTED where the driver
                                gives no tensor-map encoder) */

typedef struct {
    int fft_variant;   /* 0: default radix order of the FFT plan; 1: the reversed order (accepted for
                          every size, identical to 0 where all radices are equal); 2: the register FFT:
                          two passes with 32 values per thread and one shared-memory exchange per
                          transform for FFT lengths 256 .. 2048, three passes (48 * 4 * 8) with 48
                          values per thread and two exchanges for 3072; elsewhere 2 means 0.  Steps
                          with N-SGD, Adam or the causality mute run variant 0 whatever is set. */
    int gemm_fwd;      /* MDC_GEMM_SIMT, MDC_GEMM_TC, MDC_GEMM_GEMV or MDC_GEMM_TC_STREAM */
    int gemm_adj;      /* MDC_GEMM_SIMT, MDC_GEMM_SIMT32, MDC_GEMM_SIMT64 or MDC_GEMM_TC */
    int fft_prefetch;  /* 1: the update runs as persistent CTAs that prefetch the next tile's gradient
                          spectra while transforming the current one (variants 0 and 1, nfft <= 3072;
                          elsewhere 0) */
    int reserved[4];   /* zero */
} mdc_config;

/* The plan's current configuration (host pointer).  New plans start with fft_variant 2 for nfft 2048
 * and 0 otherwise, fft_prefetch 0, and the kernels of their precision (SIMT for FP32, TC for BF16X3). */
int mdc_plan_get_config(mdc_plan_t plan, mdc_config *cfg);
/* Set the configuration.  MDC_ERR_INVALID_ARG for an unknown value, MDC_ERR_UNSUPPORTED for
 * MDC_GEMM_TC on an FP32 plan.  Must not be called while work of the plan may still run on the GPU
 * with the old configuration in a captured graph that is later replayed (a graph keeps the kernels
 * it captured). */
int mdc_plan_set_config(mdc_plan_t plan, const mdc_config *cfg);
/* Autotune: time every candidate of each choice on this plan's sizes, with batch size nb and the
 * step flags (SMDD_RECIPROCITY changes the adjoint), reps timed launches each after one warm-up, and
 * keep the fastest.  The FFT candidates are timed on a step's two trace kernels: the fused update over a
 * subset of at most 64 MiB of model traces (scaled to all of them) plus the residual step of one batch.  best (host, may be NULL) receives the chosen configuration.
 * Uses temporary device memory (cudaMalloc), overwrites the plan's spectral workspaces, synchronises
 * the stream, and must not be called during a stream capture. */
int mdc_plan_autotune(mdc_plan_t plan, int nb, int flags, int reps, mdc_config *best, void *stream);

/* Band limit (approximate; the paper has no counterpart): only the bins f < nf_active take part in the
 * per-frequency products of every later call, the others get zero products (the FFTs still run at full
 * length, so the operator is the exact one restricted to the band).  For band-limited data -- the Ricker
 * wavelet of the synthetic workloads has no energy above ~3 f0 -- this skips the empty bins; the error
 * against the exact operator is the energy of the data above the band.  0 (or >= nf) restores every bin. */
int mdc_plan_set_band(mdc_plan_t plan, int nf_active);

/* ---------------------------------------------------------------------------------------------
 * Many independent problems.  The paper solves one MDD problem at a time and has no counterpart;
 * this serves workloads with many problems of uneven sizes (one per receiver line, frequency band or
 * survey patch).  A batch holds members, each with its own plan, model, data, source permutations
 * and step size, and runs whole SGD epochs of every member per call.  mdc_batch_create captures one
 * epoch of all members into a CUDA graph -- every step of every member, the members spread over
 * parallel branches (longest first, each onto the least loaded branch) so that small problems share
 * the GPU -- and mdc_batch_run replays it.  Each step is the smdd_step of the member with
 * SMDD_KEEP_XHAT, and SMDD_REUSE_XHAT after the first step of the epoch.
 * ------------------------------------------------------------------------------------------- */
typedef struct mdc_batch_s *mdc_batch_t;

typedef struct {
    mdc_plan_t plan;          /* the member's plan: no other batch or call may use it while the batch lives */
    float *X;                 /* [nv][nr][nt] device, the model, updated in place */
    const float *U_obs;       /* [ns][nv][nt] device */
    const int32_t *perm;      /* device int32[n_perm][ns]: epoch e visits the sources in row e % n_perm */
    int n_perm;               /* >= 1 */
    int nb;                   /* batch size, 1 .. nb_max of the plan: ceil(ns / nb) steps per epoch, the last partial */
    float alpha;              /* step size */
    int flags;                /* 0, SMDD_RECIPROCITY, or SMDD_RECIPROCITY | SMDD_SYMMETRIC (a symmetric start) */
    double *loss;             /* device float64[loss_rows][ceil(ns/nb)], or NULL: epoch e writes its step
                                 losses 1/2 ||R||^2 into row e % loss_rows */
    int loss_rows;            /* >= 1 when loss is given */
    int reserved[4];          /* zero */
} smdd_member;

/* Validate the members (host array of n; copied), allocate the per-member epoch buffers and capture
 * the epoch graph with n_branches parallel branches (1 .. 64; more branches than members is clamped).
 * stream orders the initialisation; the call returns after it is done.  Nothing runs on the members'
 * arrays until mdc_batch_run. */
int mdc_batch_create(mdc_batch_t *out, const smdd_member *members, int n, int n_branches, void *stream);

/* The same with the layout of the epoch chosen by mode:
 *   MDC_BATCH_BRANCHES : as mdc_batch_create (each member's steps as its plan's own launches, members on
 *                        n_branches parallel graph branches);
 *   MDC_BATCH_QUEUE    : persistent kernels with device work queues.  The epoch runs in waves, wave w
 *                        holding step w of every member that has one (members have ceil(ns/nb) steps);
 *                        each stage of a wave -- the model transform (wave 0), the forward product, the
 *                        residual step, the adjoint product, the update -- is one launch per kernel family
 *                        (FFT length and variant; product kernel) of CTAs resident on every SM, which take
 *                        (problem, tile) items from a queue in device memory by atomic counter until it is
 *                        empty.  The same steps and arithmetic as the branch layout (results equal bit for
 *                        bit).  n_branches is ignored.  Every member's plan must be MDC_PREC_BF16X3 with
 *                        tensor-core products (MDC_GEMM_TC or MDC_GEMM_TC_STREAM forward -- run on the tile
 *                        kernel --, MDC_GEMM_TC adjoint) and no band limit, else MDC_ERR_UNSUPPORTED. */
#define MDC_BATCH_BRANCHES 0
#define MDC_BATCH_QUEUE    1
int mdc_batch_create_ex(mdc_batch_t *out, const smdd_member *members, int n, int mode, int n_branches, void *stream);
/* Run epochs first_epoch .. first_epoch + n_epochs - 1 of every member on stream (asynchronous). */
int mdc_batch_run(mdc_batch_t batch, long long first_epoch, int n_epochs, void *stream);
/* Kernel launches in one replay of the epoch graph, and the branch count (host pointers, may be NULL). */
int mdc_batch_info(mdc_batch_t batch, long long *kernels_per_epoch, int *n_branches);
/* Release the graph and the batch's buffers (synchronises the device first; the plans stay). */
int mdc_batch_destroy(mdc_batch_t batch);

/* Failure-path check of the bounded waits (the paper has no counterpart; Eq. 2 and 6 are what the
 * checked kernels compute).  Every mbarrier wait of the split-BF16 product kernels is bounded (about a
 * second of SM clock); a CTA whose wait gives up records MDC_ERR_TIMEOUT in the plan's status word,
 * writes no products, lets products still in flight finish (one more bounded wait), frees its tensor
 * memory and returns, so the context stays usable.  With cycles > 0 every CTA of the tile kernels
 * (MDC_GEMM_TC; the streamed forward kernel ignores it) first waits on an mbarrier that nothing arrives
 * on, for `cycles` SM clock cycles, before any copy or product is issued, and then takes that path: the
 * call's products are not written (the spectral workspaces keep their previous contents) and
 * mdc_plan_sync_status returns MDC_ERR_TIMEOUT.  0 (the default) turns it off.
 * MDC_ERR_INVALID_ARG for cycles < 0 or > 1e8.  Captured graphs keep the value they were captured with. */
int mdc_plan_set_wait_probe(mdc_plan_t plan, long long cycles);

/* Wait for all work of this plan's device, then return and clear the device-side status word
 * (MDC_OK, MDC_ERR_INDEX_RANGE, or MDC_ERR_TIMEOUT when a bounded wait of a tensor-core kernel gave up). */
int mdc_plan_sync_status(mdc_plan_t plan);

/* Human-readable name of a status code (static string). */
const char *mdc_status_string(int status);

/* Stage timing and launch counting, for measurement.  When enabled, every kernel launch of the plan
 * is bracketed by CUDA events recorded on the launch stream.  mdc_plan_stage_times() waits for those
 * events and returns, per stage, the summed device milliseconds and the number of launches since the
 * last reset (arrays of MDC_NUM_STAGES entries, host pointers; either may be NULL). */
#define MDC_NUM_STAGES 7   /* rfft, cgemm_fwd, residual, cgemm_adj, update, irfft_out, setup */
int mdc_plan_set_profiling(mdc_plan_t plan, int enable);
int mdc_plan_stage_times(mdc_plan_t plan, double *ms, long long *launches, int reset);
const char *mdc_stage_name(int stage);
/* Total kernel launches made by this plan since creation (host counter). */
long long mdc_plan_launch_count(mdc_plan_t plan);

/* Arithmetic-peak probe, for the roofline of the FP32 path.  Launches one kernel of `blocks` blocks of
 * 256 threads on `stream` in which every thread runs 8 independent fused multiply-add chains for
 * `iters` rounds (kind 0: FP32 fmaf, kind 1: FP64 fma) and writes one value to sink[thread]; the
 * caller times the launch (CUDA events on `stream`) and divides *flops (host pointer, may be NULL;
 * 2 flops per multiply-add) by the duration.  sink: device buffer of blocks * 256 elements of 4 bytes
 * (kind 0) or 8 bytes (kind 1), owned by the caller.  iters must be a positive multiple of 16.
 * Returns MDC_ERR_INVALID_ARG for a bad argument, MDC_ERR_CUDA if the launch fails. */
int mdc_alu_probe(int kind, int blocks, int iters, void *sink, double *flops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SMDD_H */
