// Instantiation of the radix FFT kernels and their launchers (fft_kernels.cuh) for complex lengths 32, 64, 128, 256;
// one translation unit per length so the library compiles in parallel.
#define SMDD_FFT_INSTANTIATE 1
#include "fft_kernels.cuh"

namespace smdd {
template struct FftLaunch<32>;
template struct FftLaunch<64>;
template struct FftLaunch<128>;
template struct FftLaunch<256>;
}  // namespace smdd
