// fft_dispatch.h -- kernel-pointer tables of the FFT passes. The passes are instantiated per arithmetic
// type in their own translation units (fft_float.cu, fft_double.cu, fft_df64_*.cu) so that the library
// compiles in parallel; the host code launches them through these pointers with cudaLaunchKernel.
#pragma once
#include "df64.cuh"

namespace lgf {

// Specialised pass (fft_fixed.cuh): kind 1 = xy plane (mode 0 forward, 1 inverse), kind 2 = columns
// (mode 0 forward, 1 inverse, 2 forward + filter + inverse) with C in {16, 32}; N in {8,16,24,32,48,64}.
template <typename FT> const void *fft_fixed_kernel(int kind, int mode, int N, int C);
// Generic pass (fft.cuh, k_fft_pass).
template <typename FT> const void *fft_generic_kernel();

}  // namespace lgf
