// fft_double.cu -- the FFT passes in IEEE double (double state with LGF_FFT_NATIVE_F64=1).
#include "fft_instances.cuh"

namespace lgf {
template <> const void *fft_fixed_kernel<double>(int kind, int mode, int N, int C) {
  if (kind == 1) return mode == 0 ? fft_inst::plane<double, false>(N) : fft_inst::plane<double, true>(N);
  return C == 32 ? fft_inst::cols_mode<double, 32>(mode, N) : fft_inst::cols_mode<double, 16>(mode, N);
}
template <> const void *fft_generic_kernel<double>() { return (const void *)k_fft_pass<double>; }
}  // namespace lgf
