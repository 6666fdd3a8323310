// Full-gradient MDD by LSQR (Paige & Saunders 1982), the baseline the paper compares stochastic MDD
// against: every source at once, on the preconditioned operator A = P C (Eq. 3-4).
//
// The vectors are FP32 device arrays, every norm is reduced in FP64 with a fixed order (per-block
// partials, then one block), and the scalar recurrence of the bidiagonalisation and of the plane
// rotations runs on the device (one thread), so an iteration is a fixed sequence of launches with no
// host round trip.  The operator's forward and adjoint are the plan's own kernels with nb = ns.
#include <cmath>
#include <cstring>

#include "smdd_internal.h"

namespace smdd {

namespace {

constexpr int VEC_THREADS = 256;
constexpr int VEC_BLOCKS = 2 * 152;   // a multiple of the SM count; grid-stride loops

// LSQR scalars (device)
struct LsqrScalars {
    double alpha, beta, rho_bar, phi_bar;
    double cx, cw;        // x += cx w;  w = v - cw w
    double inv;           // 1 / (the norm just reduced), 0 for a zero vector
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// one FP64 partial of sum(a^2) per block (fixed assignment of elements to blocks and threads)
__global__ void __launch_bounds__(VEC_THREADS) k_sumsq_partials(const float *__restrict__ a, long long n,
                                                                  double *__restrict__ partials) {
    __shared__ double red[VEC_THREADS / 32];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)VEC_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * VEC_THREADS) {
        const double x = a[i];
        s += x * x;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < VEC_THREADS / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// the norm from the partials, in block order, then the scalar step `what`:
//   0: beta_1 = ||u||, phi_bar = beta                       (start)
//   1: alpha_1 = ||v||, rho_bar = alpha                     (start)
//   2: beta = ||u||                                          (iteration, after u = A v - alpha u)
//   3: alpha = ||v||, then the plane rotation; norms[it] = phi_bar   (iteration, after v = A^T u - beta v)
__global__ void k_norm_step(const double *__restrict__ partials, int nparts, LsqrScalars *sc, int what,
                            double *norms, int it) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nparts; ++b) t += partials[b];
    const double nrm = sqrt(t);
    sc->inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    if (what == 0) {
        sc->beta = nrm;
        sc->phi_bar = nrm;
        if (norms) norms[0] = nrm;
    } else if (what == 1) {
        sc->alpha = nrm;
        sc->rho_bar = nrm;
    } else if (what == 2) {
        sc->beta = nrm;
    } else {
        sc->alpha = nrm;
        const double rho = hypot(sc->rho_bar, sc->beta);
        const double c = rho > 0.0 ? sc->rho_bar / rho : 0.0, s = rho > 0.0 ? sc->beta / rho : 0.0;
        const double theta = s * nrm;
        const double phi = c * sc->phi_bar;
        sc->rho_bar = -c * nrm;
        sc->phi_bar = s * sc->phi_bar;
        sc->cx = rho > 0.0 ? phi / rho : 0.0;
        sc->cw = rho > 0.0 ? theta / rho : 0.0;
        if (norms) norms[it] = sc->phi_bar;
    }
}

// a *= inv (the reciprocal of the last norm)
__global__ void __launch_bounds__(VEC_THREADS) k_scale_inv(float *__restrict__ a, long long n, const LsqrScalars *sc) {
    const float inv = (float)sc->inv;
    for (long long i = blockIdx.x * (long long)VEC_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * VEC_THREADS)
        a[i] *= inv;
}

// y = t - coef * y   (coef = alpha or beta from the scalars; which = 0: alpha, 1: beta), optional
// causality mute on model-layout vectors (traces of nt samples, mute[trace])
__global__ void __launch_bounds__(VEC_THREADS) k_sub_scaled(float *__restrict__ y, const float *__restrict__ t, long long n,
                                                              const LsqrScalars *sc, int which, const int32_t *__restrict__ mute,
                                                              int nt) {
    const float cf = (float)(which ? sc->beta : sc->alpha);
    for (long long i = blockIdx.x * (long long)VEC_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * VEC_THREADS) {
        float tv = t[i];
        if (mute && (int)(i % nt) < mute[i / nt]) tv = 0.f;
        y[i] = tv - cf * y[i];
    }
}

// u = b - u  (start: the residual of x0)
__global__ void __launch_bounds__(VEC_THREADS) k_rsub(float *__restrict__ u, const float *__restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)VEC_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * VEC_THREADS)
        u[i] = b[i] - u[i];
}

// v = g (with the mute)
__global__ void __launch_bounds__(VEC_THREADS) k_first_v(float *__restrict__ v, const float *__restrict__ g, long long n,
                                                           const int32_t *__restrict__ mute, int nt) {
    for (long long i = blockIdx.x * (long long)VEC_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * VEC_THREADS) {
        float gv = g[i];
        if (mute && (int)(i % nt) < mute[i / nt]) gv = 0.f;
        v[i] = gv;
    }
}

// v *= inv; then x += cx w; w = v - cw w   (the normalisation of v fused with the solution update)
__global__ void __launch_bounds__(VEC_THREADS) k_update_xw(float *__restrict__ x, float *__restrict__ w, float *__restrict__ v,
                                                             long long n, const LsqrScalars *sc) {
    const float inv = (float)sc->inv, cx = (float)sc->cx, cw = (float)sc->cw;
    for (long long i = blockIdx.x * (long long)VEC_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * VEC_THREADS) {
        const float vv = v[i] * inv;
        const float wv = w[i];
        v[i] = vv;
        x[i] = fmaf(cx, wv, x[i]);
        w[i] = fmaf(-cw, wv, vv);
    }
}

__global__ void __launch_bounds__(VEC_THREADS) k_copy(float *__restrict__ y, const float *__restrict__ x, long long n) {
    for (long long i = blockIdx.x * (long long)VEC_THREADS + threadIdx.x; i < n; i += (long long)gridDim.x * VEC_THREADS)
        y[i] = x[i];
}

}  // namespace

LsqrWork::~LsqrWork() { release(); }

void LsqrWork::release() {
    cudaFree(u);
    cudaFree(t);
    cudaFree(v);
    cudaFree(w);
    cudaFree(g);
    cudaFree(idx);
    cudaFree(partials);
    cudaFree(scalars);
    u = t = v = w = g = nullptr;
    idx = nullptr;
    partials = nullptr;
    scalars = nullptr;
    nd = nm = 0;
}

cudaError_t LsqrWork::ensure(long long n_data, long long n_model, int ns) {
    if (u && n_data == nd && n_model == nm) return cudaSuccess;
    release();
    cudaError_t e;
    if ((e = cudaMalloc(&u, n_data * sizeof(float))) || (e = cudaMalloc(&t, n_data * sizeof(float))) ||
        (e = cudaMalloc(&v, n_model * sizeof(float))) || (e = cudaMalloc(&w, n_model * sizeof(float))) ||
        (e = cudaMalloc(&g, n_model * sizeof(float))) || (e = cudaMalloc(&idx, ns * sizeof(int32_t))) ||
        (e = cudaMalloc(&partials, VEC_BLOCKS * sizeof(double))) || (e = cudaMalloc(&scalars, sizeof(LsqrScalars)))) {
        release();
        return e;
    }
    nd = n_data;
    nm = n_model;
    return cudaSuccess;
}

// The LSQR iteration; apply_fwd(x, out) and apply_adj(r, out) launch the plan's operator (all
// sources; the adjoint with the reciprocity projection when asked), mute is the causality table or null.
cudaError_t lsqr_run(LsqrWork &wk, float *x, const float *b, long long nd, long long nm, int nt, int n_iter,
                     const int32_t *mute, double *norms, cudaStream_t st, const OperatorFn &apply_fwd,
                     const OperatorFn &apply_adj, long long *launches) {
    LsqrScalars *sc = reinterpret_cast<LsqrScalars *>(wk.scalars);
    long long nl = 0;
    auto norm_step = [&](const float *a, long long n, int what, int it) {
        k_sumsq_partials<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(a, n, wk.partials);
        k_norm_step<<<1, 32, 0, st>>>(wk.partials, VEC_BLOCKS, sc, what, norms, it);
        nl += 2;
        return cudaGetLastError();
    };
    cudaError_t e;
    // u = b - A x0; beta = ||u||; u /= beta
    if ((e = apply_fwd(x, wk.u))) return e;
    k_rsub<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(wk.u, b, nd);
    ++nl;
    if ((e = norm_step(wk.u, nd, 0, 0))) return e;
    k_scale_inv<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(wk.u, nd, sc);
    ++nl;
    // v = C A^T u; alpha = ||v||; v /= alpha; w = v
    if ((e = apply_adj(wk.u, wk.g))) return e;
    k_first_v<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(wk.v, wk.g, nm, mute, nt);
    ++nl;
    if ((e = norm_step(wk.v, nm, 1, 0))) return e;
    k_scale_inv<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(wk.v, nm, sc);
    k_copy<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(wk.w, wk.v, nm);
    nl += 2;
    for (int it = 1; it <= n_iter; ++it) {
        // u = A v - alpha u; beta = ||u||; u /= beta
        if ((e = apply_fwd(wk.v, wk.t))) return e;
        k_sub_scaled<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(wk.u, wk.t, nd, sc, 0, nullptr, nt);
        ++nl;
        if ((e = norm_step(wk.u, nd, 2, it))) return e;
        k_scale_inv<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(wk.u, nd, sc);
        ++nl;
        // v = C A^T u - beta v; alpha = ||v||; rotation; v /= alpha; x, w updates
        if ((e = apply_adj(wk.u, wk.g))) return e;
        k_sub_scaled<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(wk.v, wk.g, nm, sc, 1, mute, nt);
        ++nl;
        if ((e = norm_step(wk.v, nm, 3, it))) return e;
        k_update_xw<<<VEC_BLOCKS, VEC_THREADS, 0, st>>>(x, wk.w, wk.v, nm, sc);
        ++nl;
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
}

}  // namespace smdd
