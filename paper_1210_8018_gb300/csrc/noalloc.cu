// noalloc.cu -- lgf_delta_noalloc: Delta(x), theta and F of caller-owned links with no allocation at all.
//
// Who needs this: some callers cannot allocate device memory at the moment they want a measurement.
// A framework that owns all device memory through its own pool may forbid or starve foreign
// cudaMalloc calls; a service loop that must not stall cannot afford cudaMalloc, which can synchronize
// the device and take unbounded time; an out-of-memory handler or a diagnostic that runs when the
// device is nearly full has no memory left to ask for. lgf_create/lgf_delta allocate their workspaces
// lazily, so they do not fit these callers. This entry point takes every input and output from the
// caller and keeps its only scratch -- the per-block partial sums of the reduction and one counter --
// in a fixed array that is part of the library image on the device.
//
// The scratch array below is shared by every call in the process on a given device and keeps the
// contents of the last call: the counter is cleared before each launch, the partial sums are
// rewritten by each call. Two calls that run on the GPU at the same time (for instance on two
// streams without ordering) race on it and give wrong results.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lgf.h"
#include "su3.cuh"

namespace {

// One partial (theta, F) pair per block of 256 sites, plus the last-block counter.
constexpr int kNoAllocThreads = 256;
constexpr long long kNoAllocMaxSites = 1LL << 24;  // 16,777,216 sites (e.g. 64^4)
constexpr int kNoAllocMaxBlocks = (int)(kNoAllocMaxSites / kNoAllocThreads);

struct NoAllocScratch {
  double partial[2 * kNoAllocMaxBlocks];  // 1 MiB
  unsigned int ticket;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
NoAllocScratch *g_noalloc_ptr[kMaxDevices] = {nullptr};

using lgf::cx;

__device__ __forceinline__ double warp_sum_na(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void block_sum2_na(double &a, double &b) {
  __shared__ double sa[kNoAllocThreads / 32], sb[kNoAllocThreads / 32];
  a = warp_sum_na(a);
  b = warp_sum_na(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = l < kNoAllocThreads / 32 ? sa[l] : 0.0;
    b = l < kNoAllocThreads / 32 ? sb[l] : 0.0;
    a = warp_sum_na(a);
    b = warp_sum_na(b);
  }
}

__device__ __forceinline__ cx<double> ld_link(const double *U, long long idx) {
  const double2 v = __ldg(reinterpret_cast<const double2 *>(U) + idx);
  return {v.x, v.y};
}

// Same arithmetic as the Delta stencil of the main path (Eqs. 3-5, theta of Eq. 4 and F of Eq. 1 at
// g = 1), but reading the caller's links in their own layout [mu][site][3][3] and reducing through
// the static scratch.
__global__ void __launch_bounds__(kNoAllocThreads)
    k_delta_noalloc(const double *__restrict__ U, double *__restrict__ delta, double *__restrict__ theta_F,
                    NoAllocScratch *scratch, int nx, int ny, int nz, int nt) {
  const long long V = (long long)nx * ny * nz * nt;
  const long long s = (long long)blockIdx.x * kNoAllocThreads + threadIdx.x;
  double th = 0.0, f = 0.0;
  if (s < V) {
    const int n[4] = {nx, ny, nz, nt};
    long long stride[4] = {1, nx, (long long)nx * ny, (long long)nx * ny * nz};
    int c[4];
    long long r = s;
    for (int mu = 0; mu < 4; ++mu) {
      c[mu] = (int)(r % n[mu]);
      r /= n[mu];
    }
    cx<double> B[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) B[e] = {0.0, 0.0};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const long long sb = c[mu] == 0 ? s + (long long)(n[mu] - 1) * stride[mu] : s - stride[mu];
      const long long here = ((long long)mu * V + s) * 9, back = ((long long)mu * V + sb) * 9;
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        const cx<double> h = ld_link(U, here + e), b = ld_link(U, back + e);
        B[e].r += b.r - h.r;
        B[e].i += b.i - h.i;
      }
      f += ld_link(U, here).r + ld_link(U, here + 4).r + ld_link(U, here + 8).r;
    }
    // anti-Hermitian traceless part
    cx<double> D[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) D[3 * i + j] = {B[3 * i + j].r - B[3 * j + i].r, B[3 * i + j].i + B[3 * j + i].i};
    const double tr = (D[0].i + D[4].i + D[8].i) / 3.0;
    D[0].i -= tr;
    D[4].i -= tr;
    D[8].i -= tr;
#pragma unroll
    for (int e = 0; e < 9; ++e) th += D[e].r * D[e].r + D[e].i * D[e].i;
    if (delta) {
      double2 *out = reinterpret_cast<double2 *>(delta) + s * 9;
#pragma unroll
      for (int e = 0; e < 9; ++e) out[e] = make_double2(D[e].r, D[e].i);
    }
  }
  __shared__ bool last;
  block_sum2_na(th, f);
  if (threadIdx.x == 0) {
    scratch->partial[2 * blockIdx.x] = th;
    scratch->partial[2 * blockIdx.x + 1] = f;
    __threadfence();
    last = (atomicAdd(&scratch->ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0, b = 0.0;
  for (unsigned k = threadIdx.x; k < gridDim.x; k += kNoAllocThreads) {
    a += __ldcg(scratch->partial + 2 * k);
    b += __ldcg(scratch->partial + 2 * k + 1);
  }
  __syncthreads();
  block_sum2_na(a, b);
  if (threadIdx.x == 0) {
    theta_F[0] = a / (3.0 * (double)V);
    theta_F[1] = b / (12.0 * (double)V);
    scratch->ticket = 0;
  }
}

// Memory the kernel can use directly on device `dev`: device memory of that device, or managed memory.
// Device memory of another GPU is refused: the kernel would reach it only through peer access, which this
// library never enables.
bool on_device(const void *p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

bool extent_ok(int n) {
  if (n < 2 || n > 1024) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

}  // namespace

// Defined in lgf.cu: sets the message that lgf_last_error(NULL) returns (kept by pointer, no allocation).
void lgf_set_static_error(const char *msg);

extern "C" lgf_status lgf_delta_noalloc(const double *links, int Nx, int Ny, int Nz, int Nt, double *delta,
                                        double *theta_F, void *stream) {
  if (!extent_ok(Nx) || !extent_ok(Ny) || !extent_ok(Nz) || !extent_ok(Nt)) {
    lgf_set_static_error("lattice extents must be in [2, 1024] and products of 2, 3 and 5");
    return LGF_EINVAL;
  }
  const long long V = (long long)Nx * Ny * Nz * Nt;
  if (V > kNoAllocMaxSites) {
    lgf_set_static_error("lattice volume exceeds the 16777216-site limit of the fixed scratch array");
    return LGF_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    lgf_set_static_error("no usable current CUDA device");
    return LGF_ECUDA;
  }
  if (!links || !theta_F || !on_device(links, dev) || !on_device(theta_F, dev) || (delta && !on_device(delta, dev))) {
    lgf_set_static_error("links, delta and theta_F must be device pointers of the current device "
                         "(theta_F and links not NULL)");
    return LGF_EINVAL;
  }
  if (((((uintptr_t)links) | ((uintptr_t)delta)) & 15) || (((uintptr_t)theta_F) & 7)) {
    lgf_set_static_error("links and delta must be 16-byte aligned, theta_F 8-byte aligned");
    return LGF_EINVAL;
  }
  NoAllocScratch *scratch = nullptr;
  {
    // one-time set-up per device, with that device current: the device address of the static array
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        lgf_set_static_error("cudaGetSymbolAddress of the scratch array failed");
        return LGF_ECUDA;
      }
      g_noalloc_ptr[dev] = static_cast<NoAllocScratch *>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the counter must start at zero (the partial sums are fully rewritten)
  if (cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned int), st) != cudaSuccess) {
    lgf_set_static_error("cudaMemsetAsync of the scratch counter failed");
    return LGF_ECUDA;
  }
  const unsigned blocks = (unsigned)((V + kNoAllocThreads - 1) / kNoAllocThreads);
  k_delta_noalloc<<<blocks, kNoAllocThreads, 0, st>>>(links, delta, theta_F, scratch, Nx, Ny, Nz, Nt);
  if (cudaGetLastError() != cudaSuccess) {
    lgf_set_static_error("kernel launch failed");
    return LGF_ECUDA;
  }
  lgf_set_static_error(nullptr);
  return LGF_OK;
}
