// Host dispatch of the radix FFT kernels (fft_kernels.cuh) over the complex length M: plan queries,
// twiddle tables, and the launchers, which forward to FftLaunch<M> instantiated in fft_m*.cu.
//
// Appendix A: MDC = FFT along time -> batched per-frequency products -> inverse FFT.
#include "fft_kernels.cuh"

namespace smdd {

extern template struct FftLaunch<32>;
extern template struct FftLaunch<64>;
extern template struct FftLaunch<128>;
extern template struct FftLaunch<256>;
extern template struct FftLaunch<512>;
extern template struct FftLaunch<1024>;
extern template struct FftLaunch<1536>;
extern template struct FftLaunch<2048>;
extern template struct FftLaunch<4096>;

#define SMDD_SWITCH_M(M_, ...)                                    \
    switch (M_) {                                                 \
        case 32: { constexpr int MM = 32; __VA_ARGS__; } break;     \
        case 64: { constexpr int MM = 64; __VA_ARGS__; } break;     \
        case 128: { constexpr int MM = 128; __VA_ARGS__; } break;   \
        case 256: { constexpr int MM = 256; __VA_ARGS__; } break;   \
        case 512: { constexpr int MM = 512; __VA_ARGS__; } break;   \
        case 1024: { constexpr int MM = 1024; __VA_ARGS__; } break; \
        case 1536: { constexpr int MM = 1536; __VA_ARGS__; } break; \
        case 2048: { constexpr int MM = 2048; __VA_ARGS__; } break; \
        case 4096: { constexpr int MM = 4096; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;                    \
    }

bool fft_pf_supported(int M) {
    switch (M) {
        case 32: return pf_fits<32>();
        case 64: return pf_fits<64>();
        case 128: return pf_fits<128>();
        case 256: return pf_fits<256>();
        case 512: return pf_fits<512>();
        case 1024: return pf_fits<1024>();
        case 1536: return pf_fits<1536>();
        case 2048: return pf_fits<2048>();
        case 4096: return pf_fits<4096>();
    }
    return false;
}

int fft_traces_per_cta(int M) {
    switch (M) {
        case 32: return Team<32>::TR;
        case 64: return Team<64>::TR;
        case 128: return Team<128>::TR;
        case 256: return Team<256>::TR;
        case 512: return Team<512>::TR;
        case 1024: return Team<1024>::TR;
        case 1536: return Team<1536>::TR;
        case 2048: return Team<2048>::TR;
        case 4096: return Team<4096>::TR;
    }
    return 0;
}

int fft_blocks(int M, const TraceGrid &g) {
    switch (M) {
        case 32: return blocks_for<32>(g);
        case 64: return blocks_for<64>(g);
        case 128: return blocks_for<128>(g);
        case 256: return blocks_for<256>(g);
        case 512: return blocks_for<512>(g);
        case 1024: return blocks_for<1024>(g);
        case 1536: return blocks_for<1536>(g);
        case 2048: return blocks_for<2048>(g);
        case 4096: return blocks_for<4096>(g);
    }
    return 0;
}

int fft_tw_size(int M, int v) {
    switch (M) {
        case 32: return tw_size(32, v);
        case 64: return tw_size(64, v);
        case 128: return tw_size(128, v);
        case 256: return tw_size(256, v);
        case 512: return tw_size(512, v);
        case 1024: return tw_size(1024, v);
        case 1536: return tw_size(1536, v);
        case 2048: return tw_size(2048, v);
        case 4096: return tw_size(4096, v);
    }
    return 0;
}

bool fft_has_variant(int M, int v) {
    return v == 0 || (v == 1 && fft_variant_distinct(M)) || (v == 2 && fft2_supported(M));
}

void fft_tw_fill(int M, std::vector<float2> &tw, int v) {
    const double pi = 3.14159265358979323846;
    tw.assign(fft_tw_size(M, v) > 0 ? fft_tw_size(M, v) : 1, make_float2(0.f, 0.f));
    for (int inv = 0; inv < 2; ++inv)
        for (int p = 1; p < fft_npass(M); ++p) {
            const int NS = dir_span(M, inv, p, v), R = dir_radix(M, inv, p, v), off = tw_off(M, inv, p, v);
            for (int k = 0; k < NS; ++k)
                for (int r = 0; r < R; ++r) {
                    const double ang = 2.0 * pi * (double)(r * k) / (double)(NS * R);
                    tw[off + r * NS + k] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
                }
        }
}

cudaError_t fft_prepare(int M) {
    if (fft2_supported(M)) {
        const cudaError_t e = fft2_prepare(M);
        if (e != cudaSuccess) return e;
    }
    SMDD_SWITCH_M(M, { return FftLaunch<MM>::prepare(); });
    return cudaSuccess;
}

cudaError_t launch_rfft(int M, const FftArgs &a, cudaStream_t st) {
    if (a.variant == 2) return launch2_rfft(M, a, st);
    SMDD_SWITCH_M(M, { return FftLaunch<MM>::rfft(a, st); });
    return cudaSuccess;
}

cudaError_t launch_irfft_out(int M, const FftArgs &a, cudaStream_t st) {
    if (a.variant == 2) return launch2_irfft_out(M, a, st);
    SMDD_SWITCH_M(M, { return FftLaunch<MM>::irfft_out(a, st); });
    return cudaSuccess;
}

cudaError_t launch_residual(int M, const FftArgs &a, int nblocks_expected, cudaStream_t st) {
    if (a.variant == 2) return launch2_residual(M, a, nblocks_expected, st);
    SMDD_SWITCH_M(M, { return FftLaunch<MM>::residual(a, nblocks_expected, st); });
    return cudaSuccess;
}

cudaError_t launch_update(int M, bool keep, const FftArgs &a, cudaStream_t st) {
    const bool ext = a.vel || a.mute || a.adam_m;
    if (a.g.sym && a.variant == 2) return cudaErrorInvalidValue;   // the upper enumeration: radix plans
    if (a.variant == 2 && !ext) return launch2_update(M, keep, a, st);
    SMDD_SWITCH_M(M, { return FftLaunch<MM>::update(keep, a, st); });
    return cudaSuccess;
}

cudaError_t launch_queue_rfft(int M, int variant, const WorkQueue &q, cudaStream_t st) {
    if (variant == 2) return launch2_queue_rfft(M, q, st);
    SMDD_SWITCH_M(M, { return FftLaunch<MM>::queue_rfft(variant, q, st); });
    return cudaSuccess;
}

cudaError_t launch_queue_residual(int M, int variant, const WorkQueue &q, cudaStream_t st) {
    if (variant == 2) return launch2_queue_residual(M, q, st);
    SMDD_SWITCH_M(M, { return FftLaunch<MM>::queue_residual(variant, q, st); });
    return cudaSuccess;
}

cudaError_t launch_queue_update(int M, int variant, const WorkQueue &q, cudaStream_t st) {
    if (variant == 2) return launch2_queue_update(M, q, st);
    SMDD_SWITCH_M(M, { return FftLaunch<MM>::queue_update(variant, q, st); });
    return cudaSuccess;
}

}  // namespace smdd
