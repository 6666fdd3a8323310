// Allocation-free variant of the forward operator, for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc or cudaFree: code running under a memory manager that owns
// every device allocation of the process (a framework's caching allocator, a fixed pool carved out of
// a shared or embedded GPU), or latency-critical loops where the implicit device synchronisation and
// the unbounded latency of an allocation are not acceptable.  mdc_plan_create allocates its
// workspaces, so those callers cannot use the plan API.  mdc_forward_static computes the same forward
// MDC as mdc_forward, but keeps every intermediate (kernel spectra, model spectra, batch spectra,
// twiddle tables) in one file-scope device array of fixed size instead.
//
// The array is a static __device__ object: every GPU on which this part of the library is used holds
// it until the process exits.  In host code its name is only a host-side stand-in, never a device
// address: handing it to a kernel would fault, or silently use the wrong memory where the GPU can
// reach host memory.  The device address is therefore looked up with cudaGetSymbolAddress, once per
// device, with that device current, by the first call made on the device.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "smdd_fft.cuh"
#include "smdd_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (looked up once per device), or nullptr.
void *scratch_address(int dev) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

// twiddle tables of the FFT kernels, computed on the device in double precision
__global__ void k_fill_twiddles(float2 *tw, int ntw, float2 *twN, int M) {
    const int nfft = 2 * M;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntw + M + 1; i += gridDim.x * blockDim.x) {
        if (i < ntw) {
            // locate the pass table holding entry i: [r][k] with span Ns and radix R
            for (int inv = 0; inv < 2; ++inv)
                for (int p = 1; p < smdd::fft_npass(M); ++p) {
                    const int NS = smdd::dir_span(M, inv, p), R = smdd::dir_radix(M, inv, p);
                    const int off = smdd::tw_off(M, inv, p);
                    if (i >= off && i < off + NS * R) {
                        const int r = (i - off) / NS, k = (i - off) % NS;
                        double s, c;
                        sincospi(2.0 * (double)(r * k) / (double)(NS * R), &s, &c);
                        tw[i] = make_float2((float)c, (float)-s);
                    }
                }
        } else {
            const int k = i - ntw;
            double s, c;
            sincospi(2.0 * (double)k / (double)nfft, &s, &c);
            twN[k] = make_float2((float)c, (float)-s);
        }
    }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int mdc_forward_static(int nt, int nr, int nv, int ns, float scale, const float *D, const float *X,
                                  const int32_t *idx, int nb, float *U, int *dev_status, void *stream) {
    using namespace smdd;
    if (!D || !X || !idx || !U || !dev_status) return MDC_ERR_INVALID_ARG;
    if (nt < 1 || nr < 1 || nv < 1 || ns < 1 || nb < 1 || !std::isfinite(scale)) return MDC_ERR_INVALID_ARG;
    if (nt > 4096 || nb > 1024) return MDC_ERR_UNSUPPORTED;
    const int nfft = default_nfft(nt);
    const int M = nfft / 2, nf = M + 1;
    const int ldr = (nr + 1) & ~1, ldb = (nb + 1) & ~1;

    // scratch layout: twiddles | kernel spectra | model spectra | batch spectra
    const size_t o_tw = 0;
    const size_t o_twn = align256(o_tw + (size_t)fft_tw_size(M) * sizeof(float2));
    const size_t o_dh = align256(o_twn + (size_t)(M + 1) * sizeof(float2));
    const size_t o_xh = align256(o_dh + (size_t)nf * ns * ldr * sizeof(float2));
    const size_t o_uh = align256(o_xh + (size_t)nf * nv * ldr * sizeof(float2));
    const size_t need = align256(o_uh + (size_t)nf * nv * ldb * sizeof(float2));
    if (need > kScratchBytes) {   // the problem does not fit the static scratch
        fprintf(stderr, "mdc_forward_static: this problem needs %zu bytes of scratch; the static scratch holds %zu\n",
                need, kScratchBytes);
        return MDC_ERR_UNSUPPORTED;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MDC_ERR_CUDA;
    unsigned char *base = static_cast<unsigned char *>(scratch_address(dev));
    if (!base) return MDC_ERR_CUDA;
    if (fft_prepare(M) != cudaSuccess || gemm_prepare() != cudaSuccess) return MDC_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;

    float2 *tw = reinterpret_cast<float2 *>(base + o_tw);
    float2 *twN = reinterpret_cast<float2 *>(base + o_twn);
    float2 *Dh = reinterpret_cast<float2 *>(base + o_dh);
    float2 *Xh = reinterpret_cast<float2 *>(base + o_xh);
    float2 *Uh = reinterpret_cast<float2 *>(base + o_uh);
    int *status = dev_status;   // the caller's word: index errors are always reported

    const int ntw = fft_tw_size(M);
    k_fill_twiddles<<<(ntw + M + 1 + 255) / 256, 256, 0, st>>>(tw, ntw, twN, M);
    if (cudaGetLastError() != cudaSuccess) return MDC_ERR_CUDA;

    const int tr = fft_traces_per_cta(M);
    auto ti_log2 = [tr](int n) {
        int l = 0;
        while ((1 << (l + 1)) <= tr && (1 << l) < n) ++l;
        return l;
    };
    FftArgs a;
    memset(&a, 0, sizeof(a));
    a.nt = nt;
    a.tw = tw;
    a.twN = twN;
    a.s = scale / (float)nfft;
    a.status = status;
    // kernel spectra of every source: D [ns][nr][nt] -> Dh [nf][ns][ldr]
    a.g.ni = nr; a.g.nj = ns; a.g.ti_log2 = ti_log2(nr);
    a.g.tsi = nt; a.g.tsj = (long long)nr * nt;
    a.g.ssi = 1; a.g.ssj = ldr; a.g.ssf = (long long)ns * ldr;
    a.tin = D;
    a.vec = (nt % 4 == 0) && ((reinterpret_cast<uintptr_t>(D) & 15u) == 0);
    a.spec = Dh;
    if (launch_rfft(M, a, st) != cudaSuccess) return MDC_ERR_CUDA;
    // model spectra: X [nv][nr][nt] -> Xh [nf][nv][ldr]
    a.g.nj = nv; a.g.ssf = (long long)nv * ldr;
    a.tin = X;
    a.vec = (nt % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
    a.spec = Xh;
    if (launch_rfft(M, a, st) != cudaSuccess) return MDC_ERR_CUDA;
    // batch products
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = Xh; g.Dh = Dh; g.idx = idx; g.C = Uh;
    g.nv = nv; g.nr = nr; g.ns = ns; g.nb = nb; g.ldr = ldr; g.ldb = ldb;
    g.sAf = (long long)nv * ldr; g.sDf = (long long)ns * ldr; g.sCf = (long long)nv * ldb;
    g.outscale = 1.f;
    g.status = status;
    if (launch_cgemm_fwd(g, nf, st) != cudaSuccess) return MDC_ERR_CUDA;
    // inverse transforms of the batch: Uh [nf][nv][ldb] -> U [nb][nv][nt]
    FftArgs o = a;
    o.g.ni = nb; o.g.nj = nv; o.g.ti_log2 = ti_log2(nb);
    o.g.tsi = (long long)nv * nt; o.g.tsj = nt;
    o.g.ssi = 1; o.g.ssj = ldb; o.g.ssf = (long long)nv * ldb;
    o.tin = nullptr;
    o.tout = U;
    o.vec = (nt % 4 == 0) && ((reinterpret_cast<uintptr_t>(U) & 15u) == 0);
    o.spec = Uh;
    if (launch_irfft_out(M, o, st) != cudaSuccess) return MDC_ERR_CUDA;
    return MDC_OK;
}
