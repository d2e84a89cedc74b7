// fft_float.cu -- the FFT passes in float (float stage of the mixed and FP32 schedules).
#include "fft_instances.cuh"

namespace lgf {
template <> const void *fft_fixed_kernel<float>(int kind, int mode, int N, int C) {
  if (kind == 1) return mode == 0 ? fft_inst::plane<float, false>(N) : fft_inst::plane<float, true>(N);
  if (kind == 3) return (const void *)k_fx_tfilter64<float, 32, 256>;  // N = 64, C = 32, mode 2
  if (kind == 4) return mode == 0 ? (const void *)k_fx_plane64<float, false> : (const void *)k_fx_plane64<float, true>;
  return C == 32 ? fft_inst::cols_mode<float, 32>(mode, N) : fft_inst::cols_mode<float, 16>(mode, N);
}
template <> const void *fft_generic_kernel<float>() { return (const void *)k_fft_pass<float>; }
}  // namespace lgf
