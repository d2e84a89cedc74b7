// fft_df64_columns.cu -- the z/t column passes in df64 (compiled apart from the plane passes).
#include "fft_instances.cuh"

namespace lgf {
const void *fft_df64_columns(int mode, int N, int C) {
  return C == 32 ? fft_inst::cols_mode<df64, 32>(mode, N) : fft_inst::cols_mode<df64, 16>(mode, N);
}
}  // namespace lgf
