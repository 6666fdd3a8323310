// Spectra of a symmetric model (reciprocity, Eq. 4: X = C_r z with C_r = (I + T) / 2 keeps X[v][r] = X[r][v]
// from a symmetric start).  The update of such a model transforms only the traces on and above the
// TR-block diagonal (fft_kernels.cuh).  The forward product of the next step reads whole rows of the model
// spectra: the split-BF16 tile kernel reads the part below the block diagonal transposed, and for any
// other product kernel that part is filled here first by a transposed copy, per frequency bin:
//   X^[f][v][r] = X^[f][r][v]   for r < TR floor(v / TR).
// Tiles of 32 x 32 bins below (or on) the 32-block diagonal go through shared memory, read and written
// as rows of 256 bytes.
#include "smdd_internal.h"

namespace smdd {

namespace {

constexpr int MB = 32;          // tile edge
constexpr int MTHREADS = 256;   // 32 x 8

// block pair p -> (a, b), a >= b: p = a (a + 1) / 2 + b
__device__ __forceinline__ void pair_of(int p, int &a, int &b) {
    int q = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
    while (q > 0 && q * (q + 1) / 2 > p) --q;
    while ((q + 1) * (q + 2) / 2 <= p) ++q;
    a = q;
    b = p - q * (q + 1) / 2;
}

__global__ void __launch_bounds__(MTHREADS) k_mirror_lower(float2 *__restrict__ spec, int n, int ld, long long ssf,
                                                           int nf, int TR) {
    __shared__ float2 tile[MB][MB + 1];
    int a, b;   // destination rows v in block a, columns r in block b (a >= b)
    pair_of(blockIdx.x, a, b);
    const int tx = threadIdx.x % MB, ty = threadIdx.x / MB;
    for (int f = blockIdx.y; f < nf; f += gridDim.y) {
        float2 *S = spec + (long long)f * ssf;
        // source rows r = MB b + i, columns v = MB a + tx
#pragma unroll
        for (int i = ty; i < MB; i += MTHREADS / MB) {
            const int r = MB * b + i, v = MB * a + tx;
            if (r < n && v < n) tile[i][tx] = S[(long long)r * ld + v];
        }
        __syncthreads();
#pragma unroll
        for (int i = ty; i < MB; i += MTHREADS / MB) {
            const int v = MB * a + i, r = MB * b + tx;
            if (v < n && r < n && r < TR * (v / TR)) S[(long long)v * ld + r] = tile[tx][i];
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_mirror_lower(float2 *spec, int n, int ld, long long ssf, int nf, int TR, cudaStream_t st) {
    if (n <= 0 || nf <= 0 || TR <= 0 || MB % TR != 0) return cudaErrorInvalidValue;
    const int nblk = (n + MB - 1) / MB;
    const long long pairs = (long long)nblk * (nblk + 1) / 2;
    if (pairs > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int gy = nf < 64 ? nf : 64;
    k_mirror_lower<<<dim3((unsigned)pairs, gy), MTHREADS, 0, st>>>(spec, n, ld, ssf, nf, TR);
    return cudaGetLastError();
}

}  // namespace smdd
