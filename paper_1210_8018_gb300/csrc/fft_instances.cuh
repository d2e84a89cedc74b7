// fft_instances.cuh -- body of the per-type FFT translation units: defines the kernel-pointer tables of
// fft_dispatch.h for the arithmetic type LGF_FFT_TYPE (which includes instantiating the kernels).
#pragma once
#include "fft_dispatch.h"
#include "fft_fixed.cuh"

namespace lgf {
namespace fft_inst {

constexpr int kThreads = 256;

template <typename T, bool INV> const void *plane(int n) {
  switch (n) {
    case 8: return (const void *)k_fx_plane<T, 8, 8, INV, kThreads>;
    case 16: return (const void *)k_fx_plane<T, 16, 16, INV, kThreads>;
    case 24: return (const void *)k_fx_plane<T, 24, 24, INV, kThreads>;
    case 32: return (const void *)k_fx_plane<T, 32, 32, INV, kThreads>;
    case 48: return (const void *)k_fx_plane<T, 48, 48, INV, kThreads>;
    default: return (const void *)k_fx_plane<T, 64, 64, INV, kThreads>;
  }
}
template <typename T, int C, int MODE> const void *cols(int n) {
  constexpr int F = filter_fields_per_block<T>();
  switch (n) {
    case 8: return (const void *)k_fx_cols<T, 8, C, MODE, kThreads, F>;
    case 16: return (const void *)k_fx_cols<T, 16, C, MODE, kThreads, F>;
    case 24: return (const void *)k_fx_cols<T, 24, C, MODE, kThreads, F>;
    case 32: return (const void *)k_fx_cols<T, 32, C, MODE, kThreads, F>;
    case 48: return (const void *)k_fx_cols<T, 48, C, MODE, kThreads, F>;
    default: return (const void *)k_fx_cols<T, 64, C, MODE, kThreads, F>;
  }
}
template <typename T, int C> const void *cols_mode(int mode, int n) {
  if (mode == 0) return cols<T, C, 0>(n);
  if (mode == 1) return cols<T, C, 1>(n);
  return cols<T, C, 2>(n);
}

}  // namespace fft_inst
}  // namespace lgf

#if defined(LGF_FFT_PLANES) || !defined(LGF_FFT_COLUMNS)
#define LGF_FFT_WITH_PLANES 1
#endif
#if defined(LGF_FFT_COLUMNS) || !defined(LGF_FFT_PLANES)
#define LGF_FFT_WITH_COLUMNS 1
#endif
