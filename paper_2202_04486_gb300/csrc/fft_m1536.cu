// Instantiation of the radix FFT kernels and their launchers (fft_kernels.cuh) for complex length 1536;
// one translation unit per length so the library compiles in parallel.
#define SMDD_FFT_INSTANTIATE 1
#include "fft_kernels.cuh"

namespace smdd {
template struct FftLaunch<1536>;
}  // namespace smdd
