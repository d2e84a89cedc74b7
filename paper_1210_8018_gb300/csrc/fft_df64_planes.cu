// fft_df64_planes.cu -- the xy-plane passes and the generic passes in df64 (the double state's default).
#include "fft_instances.cuh"

namespace lgf {
const void *fft_df64_columns(int mode, int N, int C);  // fft_df64_columns.cu
template <> const void *fft_fixed_kernel<df64>(int kind, int mode, int N, int C) {
  if (kind == 1) return mode == 0 ? fft_inst::plane<df64, false>(N) : fft_inst::plane<df64, true>(N);
  return fft_df64_columns(mode, N, C);
}
template <> const void *fft_generic_kernel<df64>() { return (const void *)k_fft_pass<df64>; }
}  // namespace lgf
