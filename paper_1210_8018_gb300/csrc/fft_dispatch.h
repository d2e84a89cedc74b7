// fft_dispatch.h -- kernel-pointer tables of the FFT passes. The passes are instantiated per arithmetic
// type in their own translation units (fft_float.cu, fft_double.cu, fft_df64_*.cu) so that the library
// compiles in parallel; the host code launches them through these pointers with cudaLaunchKernel.
#pragma once
#include <type_traits>

#include "df64.cuh"

namespace lgf {

// Specialised pass (fft_fixed.cuh): kind 1 = xy plane (mode 0 forward, 1 inverse), kind 2 = columns
// (mode 0 forward, 1 inverse, 2 forward + filter + inverse) with C in {16, 32}; N in {8,16,24,32,48,64};
// kind 3 = the float column pass with the filter held in registers (k_fx_tfilter64: N = 64, C = 32, mode 2);
// kind 4 = the float 64 x 64 xy plane pass held in registers (k_fx_plane64; mode 0 forward, 1 inverse).
template <typename FT> const void *fft_fixed_kernel(int kind, int mode, int N, int C);
// Generic pass (fft.cuh, k_fft_pass).
template <typename FT> const void *fft_generic_kernel();

// Packed fields per block of the column pass with the filter (kind 2, mode 2): one (small tiles, more
// resident blocks), except in IEEE double, where four fields share the weights of the FP64 pipe.
template <typename FT> constexpr int filter_fields_per_block() { return std::is_same<FT, double>::value ? 4 : 1; }

// Passes that prefetch the next tile into registers while the current one is transformed: the float z
// passes (forward, inverse; measured at 64^4: 0.19 -> 0.17 ms per pass). The xy pass and the t pass with
// the filter gained nothing from it in float (the t pass lost resident blocks to the extra registers),
// and the double-float and double passes are bound by arithmetic: those take one tile per block.
template <typename FT, int KIND, int MODE> __host__ __device__ constexpr bool prefetch_tiles() {
  return std::is_same<FT, float>::value && KIND == 2 && MODE != 2;
}

}  // namespace lgf
