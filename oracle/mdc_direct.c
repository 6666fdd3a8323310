/*
 * TEST INFRASTRUCTURE ONLY.  This file is part of the parity oracle for the stochastic MDD hot path:
 * plain, slow, FP64 direct time-domain sums, written from the definitions in the paper.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Conventions (time axis fastest, all arrays float64, C order):
 *   D[s][r][t]   down-going wavefield p+ (Eq. 1-2, time domain)            ns x nr x nt
 *   X[v][r][t]   reflection response r_t, receiver r / virtual source v  nv x nr x nt
 *   U[b][j][t]   predicted up-going wavefield for batch source idx[b] and virtual source vsel[j]
 *   R[b][v][t]   residual for batch source idx[b]                        nb x nv x nt
 *   G[j][r][t]   adjoint output for virtual source vsel[j]                 nvsel x nr x nt
 *
 * The forward operator is the multi-dimensional convolution of Eq. 1/2 written in the time domain
 * (the operator P+_t of Eq. 3, restricted to the sources of a batch as in Eq. 5): a causal linear
 * convolution along time, summed over receivers, truncated to the nt recorded samples.  The adjoint is
 * its transpose, i.e. the cross-correlation of the residual with the down-going wavefield (Synthetic
 * OBC section: "the adjoint ... cross-correlation"), as used by the gradient of Eq. 6.
 *
 * Both functions return 0 on success and -1 on an invalid argument (index out of range, bad size).
 */
#include <stdint.h>
#include <stddef.h>

/* U[b][j][t] = scale * sum_r sum_{tau=0..t} D[idx[b]][r][tau] * X[vsel[j]][r][t - tau],  t in [0, nt) */
int oracle_mdc_forward(int nt, int nr, int nv, int ns,
                       const double *D, const double *X,
                       const int32_t *idx, int nb,
                       const int32_t *vsel, int nvsel,
                       double scale, double *U)
{
    if (nt <= 0 || nr <= 0 || nv <= 0 || ns <= 0 || nb < 0 || nvsel < 0) return -1;
    for (int b = 0; b < nb; ++b) if (idx[b] < 0 || idx[b] >= ns) return -1;
    for (int j = 0; j < nvsel; ++j) if (vsel[j] < 0 || vsel[j] >= nv) return -1;

    long npair = (long)nb * nvsel;
#pragma omp parallel for schedule(dynamic, 1)
    for (long p = 0; p < npair; ++p) {
        int b = (int)(p / nvsel), j = (int)(p % nvsel);
        const double *Ds = D + (size_t)idx[b] * nr * nt;
        const double *Xv = X + (size_t)vsel[j] * nr * nt;
        double *Ub = U + ((size_t)b * nvsel + j) * nt;
        for (int t = 0; t < nt; ++t) {
            double acc = 0.0;
            for (int r = 0; r < nr; ++r) {
                const double *d = Ds + (size_t)r * nt;
                const double *x = Xv + (size_t)r * nt;
                for (int tau = 0; tau <= t; ++tau) acc += d[tau] * x[t - tau];
            }
            Ub[t] = scale * acc;
        }
    }
    return 0;
}

/* G[j][r][tau] = scale * sum_b sum_{t=tau..nt-1} D[idx[b]][r][t - tau] * R[b][vsel[j]][t],  tau in [0, nt) */
int oracle_mdc_adjoint(int nt, int nr, int nv, int ns,
                       const double *D, const double *R,
                       const int32_t *idx, int nb,
                       const int32_t *vsel, int nvsel,
                       double scale, double *G)
{
    if (nt <= 0 || nr <= 0 || nv <= 0 || ns <= 0 || nb < 0 || nvsel < 0) return -1;
    for (int b = 0; b < nb; ++b) if (idx[b] < 0 || idx[b] >= ns) return -1;
    for (int j = 0; j < nvsel; ++j) if (vsel[j] < 0 || vsel[j] >= nv) return -1;

    long ntr = (long)nvsel * nr;
#pragma omp parallel for schedule(dynamic, 1)
    for (long p = 0; p < ntr; ++p) {
        int j = (int)(p / nr), r = (int)(p % nr);
        double *g = G + ((size_t)j * nr + r) * nt;
        for (int tau = 0; tau < nt; ++tau) {
            double acc = 0.0;
            for (int b = 0; b < nb; ++b) {
                const double *d = D + ((size_t)idx[b] * nr + r) * nt;
                const double *res = R + ((size_t)b * nv + vsel[j]) * nt;
                for (int t = tau; t < nt; ++t) acc += d[t - tau] * res[t];
            }
            g[tau] = scale * acc;
        }
    }
    return 0;
}

/* Number of OpenMP threads the two functions above use (1 when built without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of OpenMP threads of the two functions above (for timing the oracle single-threaded
 * and on every core; no effect without OpenMP). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
