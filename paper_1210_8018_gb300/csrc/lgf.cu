// lgf.cu -- host side of the Landau-gauge-fixing library: context, FFT pass planning, the loop of
// Algorithm 1 (Cardoso et al., Lattice 2012) with device-side loop control, the mixed-precision
// handover, and the C ABI declared in include/lgf.h.
#include <cuda_runtime.h>

#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <array>
#include <functional>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lgf.h"
#include "fft.cuh"
#include "fft_dispatch.h"
#include "autograd_kernels.cuh"
#include "mixed_kernels.cuh"
#include "site_kernels.cuh"

using namespace lgf;

namespace {

constexpr int NT = 256;  // threads per block of the per-site kernels
// threads per block of the double gauge update: a, the link and b are staged in 54 KB of shared memory
// per block (four blocks per SM)
constexpr int NT_UPDATE64 = 128;

enum KernelId {
  KID_DELTA = 0,
  KID_FFT_XY_FWD,
  KID_FFT_X_FWD,
  KID_FFT_Y_FWD,
  KID_FFT_Z_FWD,
  KID_FFT_ZT_FILTER,
  KID_FFT_T_FILTER,
  KID_FFT_Z_INV,
  KID_FFT_Y_INV,
  KID_FFT_X_INV,
  KID_FFT_XY_INV,
  KID_GAUGE,
  KID_UPDATE,
  KID_UPDATE_FUSED,
  KID_UPDATE_FUSED_REUNIT,
  KID_GACC_TO_DOUBLE,
  KID_TRANSFORM_FROM,
  KID_TO_PLANES,
  KID_FROM_PLANES,
  KID_SET_IDENTITY,
  KID_DELTA_RESIDUAL,
  KID_UPDATE_RESIDUAL,
  KID_RESIDUAL_GAUGE,
  KID_RESIDUAL_REBUILD,
  KID_RESIDUAL_BASE,
  KID_COUNT
};
// kernel names; the float instance of a kernel is reported with the suffix .f32, the double with .f64
const char *kKernelBase[KID_COUNT] = {"delta_theta",   "fft_xy_fwd",    "fft_x_fwd",      "fft_y_fwd",
                                      "fft_z_fwd",     "fft_zt_filter", "fft_t_filter",   "fft_z_inv",
                                      "fft_y_inv",     "fft_x_inv",     "fft_xy_inv",     "gauge_g",
                                      "gauge_update",  "gauge_update_fused", "gauge_update_fused_reunit",
                                      "gacc_to_double", "handover_transform", "to_planes", "from_planes",
                                      "set_identity",  "delta_residual", "update_residual", "residual_gauge",
                                      "residual_rebuild", "residual_base"};
std::string kKernelNames[2 * KID_COUNT];
template <typename T> int kid(int k) { return std::is_same<T, float>::value ? k + KID_COUNT : k; }

struct Pass {
  PassDesc d;
  int kid;
  size_t smem;
  int threads;
  // specialised passes (fft_fixed.cuh): kind 1 = xy plane, kind 2 = columns along z or t
  int kind = 0;
  int N = 0, C = 0, mode = 0, twmu = 0, ncb = 0, nblocks = 0;
  int64_t rstride = 0, ostride = 0;
  int grid_x = 0;  // blocks launched along x: one wave of the GPU (each block loops over its tiles), or nblocks
};
constexpr int kFixedThreads = 256;
bool fixed_len(int n) { return n == 8 || n == 16 || n == 24 || n == 32 || n == 48 || n == 64; }

template <typename T> struct State {
  T *U = nullptr;  // links, planes
  T *P = nullptr;  // packed Delta / Delta-tilde, 4 planes
  T *G = nullptr;  // g, 9 planes
  float *A = nullptr;  // double path: a = g - 1 in double-float, 9 planes of float4
  void *tw[4] = {nullptr, nullptr, nullptr, nullptr};
  std::vector<Pass> passes;
  FFTTables tables;
};

}  // namespace

struct lgf_ctx {
  int n[4];
  int64_t V;
  int nb = 1;  // configurations of this shape held by the context (a batch group); 1 for lgf_create
  Lattice L;
  int device = 0;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  cudaStream_t copy_stream = nullptr;  // host <-> device copies of links, pipelined with their conversion
  cudaEvent_t cev[9] = {nullptr};      // chunk events of that pipeline (kPipelineChunks + 1)
  std::string err;
  bool poisoned = false;
  int smem_optin = 0;

  State<double> s64;
  State<float> s32;
  double *p2part[4] = {nullptr, nullptr, nullptr, nullptr};
  double wscale = 0;
  AxisFFT ax[4];

  double *Wev = nullptr;    // differentiable functional: eigenvectors of omega (9 planes)
  double *lam = nullptr;    // and its eigenvalues (3 planes of doubles)
  double *U0 = nullptr;     // mixed: input links (double planes) for the handover
  float *Gacc = nullptr;    // mixed/float: accumulated gauge transformation (9 float planes)
  float *Rres = nullptr;    // mixed, residual stage: link residual R (4 x 9 float planes)
  float *Kres = nullptr;    // and K = H - 1 (9 float planes)
  double *staging = nullptr;  // AoS double buffer for host inputs / outputs and single steps
  size_t staging_bytes = 0;
  double *staging2 = nullptr;
  size_t staging2_bytes = 0;
  double *partials = nullptr;
  int nblocks_site = 0;
  int64_t partials_blocks = 0;  // (theta, F) pairs per configuration in partials
  Ctrl *ctrl = nullptr;
  Ctrl ctrl_host{};
  double *hist_dev = nullptr;
  int hist_cap = 0;
  unsigned int *ran_dev = nullptr;  // per-kernel counts of launches that did work (timing mode)

  // session
  bool loaded = false;  // a working state is present
  int load_prec = 0;    // the precision it was loaded with
  int stage = -1;       // LGF_FP64 or LGF_FP32: precision of the live working links
  int since_reunit = 0;
  bool generic_fft = false;  // force the generic FFT passes (tests compare the two families)
  bool fft_df64 = true;      // double state: Fourier filter in df64 (LGF_FFT_NATIVE_F64=1: IEEE double)
  bool residual = true;      // mixed: residual stage after the handover (LGF_RESIDUAL=0: double iterations)
  bool resid_off = false;    // this load: a rebuild made no progress, the double stage continues
  bool handover_fp64 = false;  // mixed handover transform in FP64 instead of 61-bit fixed point
  int num_sms = 1;
  bool fft_persist = true;   // specialised FFT passes as one wave of tile-looping blocks (LGF_FFT_PERSIST=0: off)
  bool tfilter_reg = true;   // float t pass with the filter in registers at Nt = 64 (LGF_TFILTER_REG=0: off)
  bool xy_reg = true;        // float 64 x 64 xy passes in registers (LGF_XY_REG=0: off)
  bool twalk = true;  // float and residual Delta and updates walking along t (LGF_TWALK=0: off; twalk_on)
  int64_t twalk_min_blocks = 2048;  // LGF_TWALK_MIN_BLOCKS
  int handover_split[2] = {2, 2};  // links per site in FP64 (even, odd warps), the rest in fixed point
  int update_split[2] = {2, 2};    // the same for the general (large-step) form of the double update
  bool reunit_fp64 = false;    // float stages: periodic projection onto SU(3) in double instead of float
  bool resid_base_ready = false;  // the float link planes hold the double links rounded (by the handover)
  double resid_theta0 = 0;  // theta of the residual stage's base links
  bool small_step = true;    // double g and update: small-step forms where they apply (LGF_SMALL_STEP=0: never)
  int fixed_cols[2] = {0, 0};  // column width of the specialised passes (double, float); 0 = default
  double prev_theta = 0;  // theta and iteration count at the previous chunk boundary
  int prev_iters = 0;

  // timing
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  std::vector<int> ev_kid;
  size_t ev_used = 0;
  double kms[2 * KID_COUNT] = {0};
  long klaunch[2 * KID_COUNT] = {0};
};

namespace {

thread_local std::string g_last_static_error;
thread_local const char *g_static_literal = nullptr;  // a static message set without allocating

lgf_status fail(lgf_ctx *c, lgf_status st, const std::string &msg) {
  if (c) {
    c->err = msg;
    if (st == LGF_ECUDA) c->poisoned = true;
  } else {
    g_last_static_error = msg;
    g_static_literal = nullptr;
  }
  return st;
}

#define CK(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? LGF_ENOMEM : LGF_ECUDA,                    \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                              \
  } while (0)

#define CKL()                                                                                       \
  do {                                                                                              \
    cudaError_t e_ = cudaGetLastError();                                                            \
    if (e_ != cudaSuccess) return fail(ctx, LGF_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

#define TRY(x)                   \
  do {                           \
    lgf_status s_ = (x);         \
    if (s_ != LGF_OK) return s_; \
  } while (0)

bool factor_ok(int n) {
  if (n < 2 || n > 1024) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

AxisFFT make_axis(int N) {
  AxisFFT a{};
  a.N = N;
  int r = N, k = 0;
  for (int R : {8, 4, 2, 3, 5})
    while (r % R == 0 && !(R == 2 && r % 4 == 0)) {
      a.R[k++] = R;
      r /= R;
    }
  while (r % 2 == 0) {
    a.R[k++] = 2;
    r /= 2;
  }
  a.nst = k;
  return a;
}

// Frequency held at each position after the in-place DIF transform with radices R[0..nst).
void digit_reversed_freq(const AxisFFT &a, std::vector<int> &kpos) {
  kpos.assign(a.N, 0);
  for (int pos = 0; pos < a.N; ++pos) {
    int N = a.N, p = pos, k = 0, mult = 1;
    for (int st = 0; st < a.nst; ++st) {
      const int R = a.R[st];
      const int M = N / R;
      const int r = p / M;  // output index r' of this stage
      k += mult * r;
      mult *= R;
      p %= M;
      N = M;
    }
    kpos[pos] = k;
  }
}

lgf_status timed_begin(lgf_ctx *ctx, int kid) {
  if (!ctx->timing) return LGF_OK;
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    ctx->ev_pool.push_back({a, b});
    ctx->ev_kid.push_back(kid);
  }
  ctx->ev_kid[ctx->ev_used] = kid;
  CK(cudaEventRecord(ctx->ev_pool[ctx->ev_used].first, ctx->stream));
  return LGF_OK;
}
lgf_status timed_end(lgf_ctx *ctx) {
  if (!ctx->timing) return LGF_OK;
  CK(cudaEventRecord(ctx->ev_pool[ctx->ev_used].second, ctx->stream));
  ctx->ev_used++;
  return LGF_OK;
}
lgf_status timed_collect(lgf_ctx *ctx) {
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ctx->ev_pool[i].first, ctx->ev_pool[i].second));
    ctx->kms[ctx->ev_kid[i]] += ms;
    ctx->klaunch[ctx->ev_kid[i]] += 1;
  }
  ctx->ev_used = 0;
  return LGF_OK;
}

template <typename T> lgf_status alloc(lgf_ctx *ctx, T **p, size_t count) {
  if (*p) return LGF_OK;
  CK(cudaMalloc((void **)p, count * sizeof(T)));
  return LGF_OK;
}

// Kernel pointers of the specialised passes (instantiated in the per-type FFT translation units).
template <typename T> const void *fixed_kernel(const Pass &p) { return fft_fixed_kernel<T>(p.kind, p.mode, p.N, p.C); }

// Specialised plan (5 passes: xy forward, z forward, t forward + filter + inverse, z inverse,
// xy inverse) when every extent is one of the fixed lengths and Nx == Ny; false otherwise.
template <typename T> bool plan_fixed(lgf_ctx *ctx, State<T> &S) {
  const int Nx = ctx->n[0], Ny = ctx->n[1], Nz = ctx->n[2], Nt = ctx->n[3];
  for (int mu = 0; mu < 4; ++mu)
    if (!fixed_len(ctx->n[mu])) return false;
  if (Nx != Ny) return false;
  const int pick = ctx->fixed_cols[sizeof(T) == 8 ? 0 : 1];
  const int C = pick ? pick : 32;  // 32-wide column tiles (measured faster than 16 in float and double-float)
  const int64_t Nxy = (int64_t)Nx * Ny, Nxyz = Nxy * Nz;
  if (Nxy % C || Nxyz % C) return false;
  const size_t es = sizeof(cx<T>);
  // filter_fields_per_block<FT>() of the FFT type FT of this state
  const int fields_per_filter_block = (sizeof(T) == 8 && !ctx->fft_df64) ? filter_fields_per_block<double>() : 1;
  std::function<Pass(int, int)> plane = [&](int mode, int kid) {
    Pass p{};
    p.kind = 1;
    p.N = Nx;
    p.mode = mode;
    p.kid = kid;
    p.nblocks = Nz * Nt;
    p.threads = kFixedThreads;
    p.smem = (size_t)(Ny * (Nx + 1) + Nx + Ny) * es;
    return p;
  };
  auto cols = [&](int N, int mode, int64_t rstride, int ncb, int64_t ostride, int nouter, int twmu, int kid) {
    Pass p{};
    p.kind = 2;
    p.N = N;
    p.C = C;
    p.mode = mode;
    p.kid = kid;
    p.rstride = rstride;
    p.ncb = ncb;
    p.ostride = ostride;
    p.nblocks = ncb * nouter;
    p.twmu = twmu;
    p.threads = kFixedThreads;
    p.smem = (size_t)((mode == 2 ? fields_per_filter_block : 1) * N * (C + 1) + N) * es;
    return p;
  };
  if (sizeof(T) == 4 && Nx == 64 && ctx->xy_reg) {
    auto plane_reg = plane;  // the register form of the 64 x 64 plane pass (512 threads, static shared memory)
    plane = [plane_reg](int mode, int kid) {
      Pass p = plane_reg(mode, kid);
      p.kind = 4;
      p.threads = 512;
      p.smem = 0;
      return p;
    };
  }
  S.passes.clear();
  S.passes.push_back(plane(0, KID_FFT_XY_FWD));
  S.passes.push_back(cols(Nz, 0, Nxy, (int)(Nxy / C), Nxyz, Nt, 2, KID_FFT_Z_FWD));
  S.passes.push_back(cols(Nt, 2, Nxyz, (int)(Nxyz / C), 0, 1, 3, KID_FFT_T_FILTER));
  if (sizeof(T) == 4 && Nt == 64 && C == 32 && ctx->tfilter_reg) {
    Pass &p = S.passes.back();  // the register form of the same pass (static shared memory)
    p.kind = 3;
    p.smem = 0;
  }
  S.passes.push_back(cols(Nz, 1, Nxy, (int)(Nxy / C), Nxyz, Nt, 2, KID_FFT_Z_INV));
  S.passes.push_back(plane(1, KID_FFT_XY_INV));
  return true;
}

// Plan the FFT passes for element size es (bytes per complex number).
template <typename T> void plan_passes(lgf_ctx *ctx, State<T> &S) {
  if (!ctx->generic_fft && plan_fixed<T>(ctx, S)) return;
  const int Nx = ctx->n[0], Ny = ctx->n[1], Nz = ctx->n[2], Nt = ctx->n[3];
  const int64_t Nxy = (int64_t)Nx * Ny, Nxyz = Nxy * Nz;
  const size_t es = sizeof(cx<T>);
  const size_t budget = 112 * 1024;  // tile bytes: two blocks per SM
  const int cmin = (int)std::max<size_t>(1, 64 / es);  // aim for >= 64-byte contiguous runs
  auto mk = [&](int d0, int d1, int d2, int64_t g0, int64_t g1, int64_t g2, int nb1, int64_t B1, int64_t B2,
                int nblocks, int nax, int dim0, int mu0, int dim1, int mu1, int mode, int kid) {
    Pass p{};
    p.d.d[0] = d0;
    p.d.d[1] = d1;
    p.d.d[2] = d2;
    p.d.g[0] = g0;
    p.d.g[1] = g1;
    p.d.g[2] = g2;
    p.d.nb1 = nb1;
    p.d.B1 = B1;
    p.d.B2 = B2;
    p.d.nblocks = nblocks;
    p.d.nax = nax;
    p.d.ax_dim[0] = dim0;
    p.d.ax_mu[0] = mu0;
    p.d.ax_dim[1] = dim1;
    p.d.ax_mu[1] = mu1;
    p.d.mode = mode;
    p.kid = kid;
    const int nel = d0 * d1 * d2;
    int twn = ctx->n[mu0] + (nax > 1 ? ctx->n[mu1] : 0);
    p.smem = (size_t)(nel + twn) * es;
    p.threads = nel >= 2048 ? 512 : 256;
    return p;
  };
  auto largest_run = [&](int64_t extent, int64_t per_col_bytes, int cap) {
    int best = 1;
    for (int c = 1; c <= cap && c <= extent; ++c)
      if (extent % c == 0 && (size_t)(c * per_col_bytes) <= budget) best = c;
    return best;
  };
  std::vector<Pass> fwd, mid, inv;
  // x and y
  if ((size_t)Nxy * es <= budget) {
    const int nb = Nz * Nt;
    fwd.push_back(mk(Nx, Ny, 1, 1, Nx, 0, nb, Nxy, 0, nb, 2, 0, 0, 1, 1, 0, KID_FFT_XY_FWD));
    inv.push_back(mk(Nx, Ny, 1, 1, Nx, 0, nb, Nxy, 0, nb, 2, 0, 0, 1, 1, 1, KID_FFT_XY_INV));
  } else {
    const int rows = largest_run(Ny * Nz * Nt, (int64_t)Nx * es, 16);
    const int nbx = (int)(Ny * (int64_t)Nz * Nt / rows);
    fwd.push_back(mk(Nx, rows, 1, 1, Nx, 0, nbx, (int64_t)rows * Nx, 0, nbx, 1, 0, 0, 0, 0, 0, KID_FFT_X_FWD));
    const int cy = largest_run(Nx, (int64_t)Ny * es, 64);
    const int nby = (Nx / cy) * Nz * Nt;
    fwd.push_back(mk(cy, Ny, 1, 1, Nx, 0, Nx / cy, cy, Nxy, nby, 1, 1, 1, 0, 0, 0, KID_FFT_Y_FWD));
    inv.push_back(mk(cy, Ny, 1, 1, Nx, 0, Nx / cy, cy, Nxy, nby, 1, 1, 1, 0, 0, 1, KID_FFT_Y_INV));
    inv.push_back(mk(Nx, rows, 1, 1, Nx, 0, nbx, (int64_t)rows * Nx, 0, nbx, 1, 0, 0, 0, 0, 1, KID_FFT_X_INV));
  }
  // z and t, with the filter
  const int64_t zt_col = (int64_t)Nz * Nt * es;
  int czt = 0;
  for (int c = (int)std::min<int64_t>(Nxy, 64); c >= 1; --c)
    if (Nxy % c == 0 && (size_t)(c * zt_col) <= budget) {
      czt = c;
      break;
    }
  if (czt >= std::min<int64_t>(cmin, Nxy)) {
    const int nb = (int)(Nxy / czt);
    mid.push_back(mk(czt, Nz, Nt, 1, Nxy, Nxyz, nb, czt, 0, nb, 2, 1, 2, 2, 3, 2, KID_FFT_ZT_FILTER));
  } else {
    const int cz = largest_run(Nxy, (int64_t)Nz * es, 64);
    const int nbz = (int)(Nxy / cz) * Nt;
    fwd.push_back(mk(cz, Nz, 1, 1, Nxy, 0, (int)(Nxy / cz), cz, Nxyz, nbz, 1, 1, 2, 0, 0, 0, KID_FFT_Z_FWD));
    const int ct = largest_run(Nxyz, (int64_t)Nt * es, 64);
    const int nbt = (int)(Nxyz / ct);
    mid.push_back(mk(ct, Nt, 1, 1, Nxyz, 0, nbt, ct, 0, nbt, 1, 1, 3, 0, 0, 2, KID_FFT_T_FILTER));
    inv.insert(inv.begin(),
               mk(cz, Nz, 1, 1, Nxy, 0, (int)(Nxy / cz), cz, Nxyz, nbz, 1, 1, 2, 0, 0, 1, KID_FFT_Z_INV));
  }
  S.passes.clear();
  for (auto &p : fwd) S.passes.push_back(p);
  for (auto &p : mid) S.passes.push_back(p);
  for (auto &p : inv) S.passes.push_back(p);
}

// Arithmetic type of the Fourier filter of state T: float for the float state; for the double state
// df64 (two floats) unless the context asks for IEEE double. The packed Delta buffer of the state holds
// that type (16 bytes per complex number for both double and df64).
template <typename T, typename Fn> lgf_status with_fft_type(const lgf_ctx *ctx, Fn &&fn) {
  if constexpr (std::is_same<T, double>::value) {
    if (ctx->fft_df64) return fn(df64{});
    return fn(double{});
  } else {
    return fn(float{});
  }
}

template <typename FT> void fill_twiddles(std::vector<FT> &tw, int N) {
  for (int j = 0; j < N; ++j) {
    // w_N^j = exp(-2 pi i j / N) in long double, rounded to FT
    const long double a = 2.0L * 3.14159265358979323846264338327950288L * (long double)j / (long double)N;
    tw[2 * j] = (FT)std::cos(a);
    tw[2 * j + 1] = (FT)(-std::sin(a));
  }
}
template <> void fill_twiddles<df64>(std::vector<df64> &tw, int N) {
  for (int j = 0; j < N; ++j) {
    const long double a = 2.0L * 3.14159265358979323846264338327950288L * (long double)j / (long double)N;
    const long double c = std::cos(a), sn = -std::sin(a);
    const float ch = (float)c, sh = (float)sn;
    tw[2 * j] = df64{ch, (float)(c - (long double)ch)};
    tw[2 * j + 1] = df64{sh, (float)(sn - (long double)sh)};
  }
}

// Opt the FFT kernels in to the dynamic shared memory each pass needs (the generic kernel: the
// largest of its passes).
// The specialised passes get one wave of blocks (resident blocks per SM x SMs, over the fields and the
// configurations of the launch), each looping over its tiles with the next tile's loads in flight.
template <typename T> lgf_status opt_in_smem(lgf_ctx *ctx, State<T> &S) {
  return with_fft_type<T>(ctx, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    size_t generic_max = 0;
    for (auto &p : S.passes) {
      if (p.kind == 0) generic_max = std::max(generic_max, p.smem);
      else if (p.smem > 48 * 1024)
        CK(cudaFuncSetAttribute(fixed_kernel<FT>(p), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
      if (p.kind != 0) {
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fixed_kernel<FT>(p), p.threads, p.smem));
        const int gy = p.kind == 2 && p.mode == 2 ? 4 / filter_fields_per_block<FT>() : 4;
        const int64_t wave = (int64_t)std::max(per_sm, 1) * ctx->num_sms;
        const int64_t gx = (wave + (int64_t)gy * ctx->nb - 1) / ((int64_t)gy * ctx->nb);
        const bool prefetch = p.kind == 2 ? (p.mode == 0   ? prefetch_tiles<FT, 2, 0>()
                                             : p.mode == 1 ? prefetch_tiles<FT, 2, 1>()
                                                           : prefetch_tiles<FT, 2, 2>())
                                          : prefetch_tiles<FT, 1, 0>();  // kind 1 and 3: one tile per block
        p.grid_x = ctx->fft_persist && prefetch ? (int)std::min<int64_t>(p.nblocks, std::max<int64_t>(gx, 1))
                                                : p.nblocks;
      }
    }
    if (generic_max > 48 * 1024)
      CK(cudaFuncSetAttribute(fft_generic_kernel<FT>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)generic_max));
    return LGF_OK;
  });
}

template <typename T> lgf_status setup_precision(lgf_ctx *ctx, State<T> &S) {
  const int64_t V = ctx->V;
  const size_t nb = (size_t)ctx->nb;
  TRY(alloc(ctx, &S.U, nb * 4 * LinkStore<T>::planes * V * 2));
  TRY(alloc(ctx, &S.P, nb * 4 * V * 2));
  TRY(alloc(ctx, &S.G, nb * 9 * V * 2));
  if constexpr (std::is_same<T, double>::value) TRY(alloc(ctx, &S.A, nb * 9 * V * 4));
  if (!S.tw[0]) {
    for (int mu = 0; mu < 4; ++mu) {
      const int N = ctx->n[mu];
      TRY(with_fft_type<T>(ctx, [&](auto tag) -> lgf_status {
        using FT = decltype(tag);
        std::vector<FT> tw(2 * N);
        fill_twiddles<FT>(tw, N);
        CK(cudaMalloc(&S.tw[mu], sizeof(FT) * 2 * N));
        CK(cudaMemcpy(S.tw[mu], tw.data(), sizeof(FT) * 2 * N, cudaMemcpyHostToDevice));
        return LGF_OK;
      }));
    }
    plan_passes<T>(ctx, S);
    for (int mu = 0; mu < 4; ++mu) {
      S.tables.ax[mu] = ctx->ax[mu];
      S.tables.tw[mu] = S.tw[mu];
      S.tables.p2part[mu] = ctx->p2part[mu];
      S.tables.n[mu] = ctx->n[mu];
    }
    S.tables.wscale = ctx->wscale;
    TRY(opt_in_smem<T>(ctx, S));
    if constexpr (std::is_same<T, double>::value) {
      CK(cudaFuncSetAttribute(k_update<double, NT_UPDATE64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)update_smem_bytes<NT_UPDATE64>()));
      CK(cudaFuncSetAttribute(k_update<double, NT_UPDATE64>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared));
    }
  }
  return LGF_OK;
}

lgf_status ensure_common(lgf_ctx *ctx) {
  if (!ctx->partials) {
    ctx->nblocks_site = (int)((ctx->V + NT * kSitesPerThread - 1) / (NT * kSitesPerThread));
    // one (theta, F) pair per block of the largest reducing grid: the site kernels' nblocks_site, or the
    // t-walking kernels' columns x Nt / 8 blocks (twalk_on)
    ctx->partials_blocks = std::max<int64_t>(
        std::max(ctx->nblocks_site, 1), (ctx->L.stride[3] + NT - 1) / NT * std::max(ctx->n[3] / 8, 1));
    CK(cudaMalloc(&ctx->partials, sizeof(double) * 2 * (size_t)ctx->partials_blocks * ctx->nb));
    CK(cudaMalloc(&ctx->ctrl, sizeof(Ctrl) * ctx->nb));
    CK(cudaMemset(ctx->ctrl, 0, sizeof(Ctrl) * ctx->nb));
  }
  return LGF_OK;
}

lgf_status ensure_staging(lgf_ctx *ctx, double **buf, size_t *have, size_t bytes) {
  if (*have >= bytes) return LGF_OK;
  if (*buf) CK(cudaFree(*buf));
  *buf = nullptr;
  *have = 0;
  CK(cudaMalloc(buf, bytes));
  *have = bytes;
  return LGF_OK;
}

enum PtrKind { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };

// Host memory (pageable, or page-locked), memory the kernels of the context's device can use directly
// (device memory of that device, or managed memory), or device memory of another GPU (rejected: the
// kernels would reach it only through peer access, which the library does not enable).
PtrKind ptr_kind(const void *p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  if (a.type == cudaMemoryTypeManaged) return PTR_DEVICE;
  if (a.type == cudaMemoryTypeDevice) return a.device == device ? PTR_DEVICE : PTR_OTHER_DEVICE;
  return PTR_HOST;
}

// Resolve a caller buffer of `bytes` to a device pointer: device memory as it is, host memory staged
// through `buf` by the copy engine (measured faster than kernels reading page-locked host memory over
// the host link).
lgf_status input_ptr(lgf_ctx *ctx, const double *p, size_t bytes, double **buf, size_t *have, const double **out) {
  if (!p) return fail(ctx, LGF_EINVAL, "null buffer");
  const PtrKind k = ptr_kind(p, ctx->device);
  if (k == PTR_OTHER_DEVICE) return fail(ctx, LGF_EINVAL, "device buffer belongs to another GPU than the context's");
  if (k == PTR_DEVICE) {
    if (((uintptr_t)p) & 15) return fail(ctx, LGF_EINVAL, "device buffers must be 16-byte aligned");
    *out = p;
    return LGF_OK;
  }
  TRY(ensure_staging(ctx, buf, have, bytes));
  CK(cudaMemcpyAsync(*buf, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *out = *buf;
  return LGF_OK;
}

lgf_status output_ptr(lgf_ctx *ctx, double *p, size_t bytes, double **buf, size_t *have, double **dev, bool *host) {
  if (!p) return fail(ctx, LGF_EINVAL, "null buffer");
  const PtrKind k = ptr_kind(p, ctx->device);
  if (k == PTR_OTHER_DEVICE) return fail(ctx, LGF_EINVAL, "device buffer belongs to another GPU than the context's");
  if (k == PTR_DEVICE) {
    if (((uintptr_t)p) & 15) return fail(ctx, LGF_EINVAL, "device buffers must be 16-byte aligned");
    *dev = p;
    *host = false;
    return LGF_OK;
  }
  TRY(ensure_staging(ctx, buf, have, bytes));
  *dev = *buf;
  *host = true;
  return LGF_OK;
}

unsigned grid1(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// The kernels that walk along t give each thread kTwalkSlices consecutive t-slices. They run when Nt allows
// and the launch still has twalk_min_blocks blocks; otherwise the site-order kernels run. Measured: at 64^4
// (8192 blocks) the walking kernels save the second read of each t-neighbour and 9 ms per mixed fix; on
// single lattices with fewer blocks (32^4: 512, 32^3 x 64: 1024) the second read hits L2 anyway and the
// site-order kernels are as fast or faster (32^3 x 64: 28.5 against 29.5 ms); shorter walks (4 or 2 slices,
// more blocks) were slower still.
constexpr int kTwalkSlices = 8;
bool twalk_on(const lgf_ctx *ctx) {
  if (!ctx->twalk || ctx->n[3] % kTwalkSlices) return false;
  const int64_t blocks = (int64_t)grid1(ctx->L.stride[3], NT) * (ctx->n[3] / kTwalkSlices);  // per configuration
  return blocks * ctx->nb >= ctx->twalk_min_blocks && blocks <= ctx->partials_blocks;
}
dim3 twalk_grid(const lgf_ctx *ctx) { return dim3(grid1(ctx->L.stride[3], NT), ctx->n[3] / kTwalkSlices, ctx->nb); }

template <typename T> lgf_status launch_delta(lgf_ctx *ctx, State<T> &S, int counts_update, int check_active) {
  TRY(timed_begin(ctx, kid<T>(KID_DELTA)));
  TRY(with_fft_type<T>(ctx, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    const dim3 grid(ctx->nblocks_site, 1, ctx->nb);
    FT *P = reinterpret_cast<FT *>(S.P);
    if constexpr (std::is_same<T, float>::value) {
      if (twalk_on(ctx))
        k_delta_f32_tw<NT, kTwalkSlices><<<twalk_grid(ctx), NT, 0, ctx->stream>>>(
            S.U, P, ctx->partials, ctx->ctrl, ctx->L, counts_update, check_active, kid<T>(KID_DELTA));
      else
        k_delta_f32<NT><<<grid, NT, 0, ctx->stream>>>(S.U, P, ctx->partials, ctx->ctrl, ctx->L, counts_update,
                                                      check_active, kid<T>(KID_DELTA));
    }
    else
      k_delta<T, NT, FT><<<grid, NT, 0, ctx->stream>>>(S.U, P, ctx->partials, ctx->ctrl, ctx->L, counts_update,
                                                       check_active, kid<T>(KID_DELTA));
    CKL();
    return LGF_OK;
  }));
  return timed_end(ctx);
}

template <typename T> lgf_status launch_filter(lgf_ctx *ctx, State<T> &S, T *data_, int check_active) {
  return with_fft_type<T>(ctx, [&](auto tag) -> lgf_status {
  using FT = decltype(tag);
  FT *data = reinterpret_cast<FT *>(data_);
  for (auto &p : S.passes) {
    TRY(timed_begin(ctx, kid<T>(p.kid)));
    const int tk = kid<T>(p.kid);
    if (p.kind == 0) {
      dim3 grid(p.d.nblocks, 4, ctx->nb);
      int64_t V = ctx->V;
      PassDesc pd = p.d;
      FFTTables tb = S.tables;
      const Ctrl *c = ctx->ctrl;
      void *args[] = {&data, &V, &pd, &tb, &c, &check_active, (void *)&tk};
      CK(cudaLaunchKernel(fft_generic_kernel<FT>(), grid, dim3(p.threads), args, p.smem, ctx->stream));
    } else if (p.kind == 1 || p.kind == 4) {
      dim3 grid(p.grid_x > 0 ? p.grid_x : p.nblocks, 4, ctx->nb);
      int64_t V = ctx->V;
      FFTTables tb = S.tables;
      const Ctrl *c = ctx->ctrl;
      int nt = p.nblocks;
      void *args[] = {&data, &V, &tb, &c, &check_active, (void *)&tk, &nt};
      CK(cudaLaunchKernel(fixed_kernel<FT>(p), grid, dim3(p.threads), args, p.smem, ctx->stream));
    } else {
      dim3 grid(p.grid_x > 0 ? p.grid_x : p.nblocks, p.mode == 2 ? 4 / filter_fields_per_block<FT>() : 4, ctx->nb);
      int64_t V = ctx->V, rs = p.rstride, os = p.ostride;
      int ncb = p.ncb, twmu = p.twmu, nt = p.nblocks;
      FFTTables tb = S.tables;
      const Ctrl *c = ctx->ctrl;
      void *args[] = {&data, &V, &rs, &ncb, &os, &tb, &c, &check_active, (void *)&tk, &twmu, &nt};
      CK(cudaLaunchKernel(fixed_kernel<FT>(p), grid, dim3(p.threads), args, p.smem, ctx->stream));
    }
    CKL();
    TRY(timed_end(ctx));
  }
  return LGF_OK;
  });
}

template <typename T> lgf_status launch_gauge(lgf_ctx *ctx, State<T> &S, double alpha, int check_active) {
  TRY(timed_begin(ctx, kid<T>(KID_GAUGE)));
  TRY(with_fft_type<T>(ctx, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    k_gauge<T, NT, FT><<<dim3(grid1(ctx->V, NT), 1, ctx->nb), NT, 0, ctx->stream>>>(
        reinterpret_cast<const FT *>(S.P), S.G, S.A, (T)(0.5 * alpha), ctx->V, ctx->ctrl, check_active, kid<T>(KID_GAUGE),
        ctx->small_step ? 1 : 0);
    CKL();
    return LGF_OK;
  }));
  return timed_end(ctx);
}

template <typename T> lgf_status launch_update(lgf_ctx *ctx, State<T> &S, int check_active) {
  TRY(timed_begin(ctx, kid<T>(KID_UPDATE)));
  if constexpr (std::is_same<T, double>::value) {
    k_update<double, NT_UPDATE64><<<dim3(grid1(ctx->V, NT_UPDATE64), 1, ctx->nb), NT_UPDATE64,
                                    update_smem_bytes<NT_UPDATE64>(), ctx->stream>>>(
        S.U, S.G, S.A, ctx->L, ctx->ctrl, check_active, kid<T>(KID_UPDATE), ctx->small_step ? 1 : 0,
        ctx->update_split[0], ctx->update_split[1]);
  } else {
    k_update<T, NT><<<dim3(grid1(ctx->V, NT), 1, ctx->nb), NT, 0, ctx->stream>>>(S.U, S.G, nullptr, ctx->L, ctx->ctrl,
                                                                               check_active, kid<T>(KID_UPDATE), 0, 0, 0);
  }
  CKL();
  return timed_end(ctx);
}

// One iteration of the loop of Algorithm 1 on state S (kernels return at once once the loop stops).
template <typename T> lgf_status launch_iteration(lgf_ctx *ctx, State<T> &S, double alpha) {
  TRY(launch_filter<T>(ctx, S, S.P, 1));
  TRY(launch_gauge<T>(ctx, S, alpha, 1));
  TRY(launch_update<T>(ctx, S, 1));
  return launch_delta<T>(ctx, S, 1, 1);
}

// Double-stage iteration with the FFT in float (mixed option fft32_final): Delta in double stored
// packed in float, float FFT passes, g formed in double from the float Delta-tilde, double update.
lgf_status launch_delta_d2f(lgf_ctx *ctx, int counts_update, int check_active) {
  TRY(timed_begin(ctx, kid<double>(KID_DELTA)));
  k_delta<double, NT, float><<<dim3(ctx->nblocks_site, 1, ctx->nb), NT, 0, ctx->stream>>>(
      ctx->s64.U, ctx->s32.P, ctx->partials, ctx->ctrl, ctx->L, counts_update, check_active, kid<double>(KID_DELTA));
  CKL();
  return timed_end(ctx);
}
lgf_status launch_iteration_fft32(lgf_ctx *ctx, double alpha) {
  TRY(launch_filter<float>(ctx, ctx->s32, ctx->s32.P, 2));
  TRY(timed_begin(ctx, kid<double>(KID_GAUGE)));
  k_gauge<double, NT, float><<<dim3(grid1(ctx->V, NT), 1, ctx->nb), NT, 0, ctx->stream>>>(
      ctx->s32.P, ctx->s64.G, ctx->s64.A, 0.5 * alpha, ctx->V, ctx->ctrl, 1, kid<double>(KID_GAUGE),
      ctx->small_step ? 1 : 0);
  CKL();
  TRY(timed_end(ctx));
  TRY(launch_update<double>(ctx, ctx->s64, 1));
  return launch_delta_d2f(ctx, 1, 1);
}

// One iteration of the float stage (FP32 / mixed): g is rebuilt inside the update, which also
// accumulates G and, every reunit_period iterations, reprojects G and the new links onto SU(3).
lgf_status launch_iteration_float(lgf_ctx *ctx, double alpha, bool reunit) {
  State<float> &S = ctx->s32;
  TRY(launch_filter<float>(ctx, S, S.P, 1));
  const int kidx = kid<float>(reunit ? KID_UPDATE_FUSED_REUNIT : KID_UPDATE_FUSED);
  TRY(timed_begin(ctx, kidx));
  const dim3 grid(grid1(ctx->V, NT), 1, ctx->nb);
  const float ha = (float)(0.5 * alpha);
  if (twalk_on(ctx)) {
    constexpr int TCH = kTwalkSlices;
    if (reunit && ctx->reunit_fp64)
      k_update_fused_f32_tw<NT, 2, TCH><<<twalk_grid(ctx), NT, 0, ctx->stream>>>(S.U, S.P, ctx->Gacc, ha, ctx->L,
                                                                                 ctx->ctrl, kidx);
    else if (reunit)
      k_update_fused_f32_tw<NT, 1, TCH><<<twalk_grid(ctx), NT, 0, ctx->stream>>>(S.U, S.P, ctx->Gacc, ha, ctx->L,
                                                                                 ctx->ctrl, kidx);
    else
      k_update_fused_f32_tw<NT, 0, TCH><<<twalk_grid(ctx), NT, 0, ctx->stream>>>(S.U, S.P, ctx->Gacc, ha, ctx->L,
                                                                                 ctx->ctrl, kidx);
  } else if (reunit && ctx->reunit_fp64)
    k_update_fused_f32<NT, 2><<<grid, NT, 0, ctx->stream>>>(S.U, S.P, ctx->Gacc, ha, ctx->L, ctx->ctrl, kidx);
  else if (reunit)
    k_update_fused_f32<NT, 1><<<grid, NT, 0, ctx->stream>>>(S.U, S.P, ctx->Gacc, ha, ctx->L, ctx->ctrl, kidx);
  else
    k_update_fused_f32<NT, 0><<<grid, NT, 0, ctx->stream>>>(S.U, S.P, ctx->Gacc, ha, ctx->L, ctx->ctrl, kidx);
  CKL();
  TRY(timed_end(ctx));
  return launch_delta<float>(ctx, S, 1, 1);
}

lgf_status read_ctrl(lgf_ctx *ctx) {
  CK(cudaMemcpyAsync(&ctx->ctrl_host, ctx->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->timing) TRY(timed_collect(ctx));
  return LGF_OK;
}

lgf_status write_ctrl(lgf_ctx *ctx) {
  ctx->ctrl_host.ran = ctx->timing ? ctx->ran_dev : nullptr;
  CK(cudaMemcpyAsync(ctx->ctrl, &ctx->ctrl_host, sizeof(Ctrl), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LGF_OK;
}

// Mixed handover: G from the float accumulation (reprojected in double), then
// U = G U0 G^+(x+mu) in double precision from the saved input (exact gauge equivalence). With
// write_base, rows 0-1 of U rounded to float also go to the float link planes (the residual stage's
// base; the float stage's links are not needed after the handover).
lgf_status handover(lgf_ctx *ctx, bool write_base = false) {
  TRY(setup_precision<double>(ctx, ctx->s64));
  TRY(timed_begin(ctx, kid<double>(KID_GACC_TO_DOUBLE)));
  k_gacc_to_double<NT><<<grid1(ctx->V, NT), NT, 0, ctx->stream>>>(ctx->Gacc, ctx->s64.G, ctx->V);
  CKL();
  TRY(timed_end(ctx));
  TRY(timed_begin(ctx, kid<double>(KID_TRANSFORM_FROM)));
  if (ctx->handover_fp64)
    k_transform_from<NT><<<grid1(ctx->V, NT), NT, 0, ctx->stream>>>(ctx->U0, ctx->s64.U, ctx->s64.G, ctx->L,
                                                                   write_base ? ctx->s32.U : nullptr);
  else
    k_transform_from_q<NT><<<grid1(ctx->V, NT), NT, 0, ctx->stream>>>(ctx->U0, ctx->s64.U, ctx->s64.G, ctx->L,
                                                                     write_base ? ctx->s32.U : nullptr,
                                                                     ctx->handover_split[0], ctx->handover_split[1]);
  CKL();
  ctx->resid_base_ready = write_base;
  return timed_end(ctx);
}

// Residual stage of the mixed schedule (mixed_kernels.cuh), stage code kHostStageResidual on the host and
// kStageResidual in the loop control. Entered from the double state: s64.U holds the base links U_h,
// s64.P their packed Delta, s64.G the transformation G with U_h = G U0 G^+, and the loop control their
// theta and F.
constexpr int kHostStageResidual = 3;

lgf_status launch_delta_residual(lgf_ctx *ctx, int counts_update) {
  TRY(timed_begin(ctx, kid<float>(KID_DELTA_RESIDUAL)));
  TRY(with_fft_type<double>(ctx, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    if (twalk_on(ctx))
      k_delta_residual_tw<NT, FT, kTwalkSlices><<<twalk_grid(ctx), NT, 0, ctx->stream>>>(
          ctx->Rres, reinterpret_cast<const FT *>(ctx->s64.P), ctx->s32.P, ctx->partials, ctx->ctrl, ctx->L,
          counts_update, kid<float>(KID_DELTA_RESIDUAL));
    else
      k_delta_residual<NT, FT><<<dim3(ctx->nblocks_site, 1, ctx->nb), NT, 0, ctx->stream>>>(
          ctx->Rres, reinterpret_cast<const FT *>(ctx->s64.P), ctx->s32.P, ctx->partials, ctx->ctrl, ctx->L,
          counts_update, kid<float>(KID_DELTA_RESIDUAL));
    CKL();
    return LGF_OK;
  }));
  return timed_end(ctx);
}

lgf_status residual_begin(lgf_ctx *ctx) {
  const int64_t V = ctx->V;
  TRY(setup_precision<float>(ctx, ctx->s32));
  TRY(alloc(ctx, &ctx->Rres, (size_t)36 * V * 2));
  TRY(alloc(ctx, &ctx->Kres, (size_t)9 * V * 2));
  if (!ctx->resid_base_ready) {
    TRY(timed_begin(ctx, kid<float>(KID_RESIDUAL_BASE)));
    k_narrow_link_planes<<<grid1((int64_t)4 * V, NT), NT, 0, ctx->stream>>>(ctx->s64.U, ctx->s32.U, V, 0, 4 * V);
    CKL();
    TRY(timed_end(ctx));
  }
  ctx->resid_base_ready = false;
  CK(cudaMemsetAsync(ctx->Rres, 0, sizeof(float) * 72 * (size_t)V, ctx->stream));
  CK(cudaMemsetAsync(ctx->Kres, 0, sizeof(float) * 18 * (size_t)V, ctx->stream));
  Ctrl &c = ctx->ctrl_host;
  ctx->resid_theta0 = c.theta;
  ctx->stage = kHostStageResidual;
  ctx->prev_theta = 0;
  c.f_base = c.F;
  c.stage = kStageResidual;
  c.active = 1;
  TRY(write_ctrl(ctx));
  TRY(launch_delta_residual(ctx, 0));  // Delta = Delta(U_h) packed in float, and theta, F
  return read_ctrl(ctx);
}

lgf_status launch_iteration_residual(lgf_ctx *ctx, double alpha) {
  TRY(launch_filter<float>(ctx, ctx->s32, ctx->s32.P, 3));
  TRY(timed_begin(ctx, kid<float>(KID_UPDATE_RESIDUAL)));
  if (twalk_on(ctx))
    k_update_residual_tw<NT, kTwalkSlices><<<twalk_grid(ctx), NT, 0, ctx->stream>>>(
        ctx->s32.U, ctx->Rres, ctx->Kres, ctx->s32.P, (float)(0.5 * alpha), ctx->L, ctx->ctrl,
        kid<float>(KID_UPDATE_RESIDUAL));
  else
    k_update_residual<NT><<<dim3(grid1(ctx->V, NT), 1, ctx->nb), NT, 0, ctx->stream>>>(
        ctx->s32.U, ctx->Rres, ctx->Kres, ctx->s32.P, (float)(0.5 * alpha), ctx->L, ctx->ctrl,
        kid<float>(KID_UPDATE_RESIDUAL));
  CKL();
  TRY(timed_end(ctx));
  return launch_delta_residual(ctx, 1);
}

// End of the residual stage: H = proj(1 + K) in double, U_h -> H U_h H^+(x + mu) in place by the double
// update (small-step form: exact to FP64 rounding for H close to 1), and Delta, theta and F of the
// rebuilt links in double. Leaves the double state.
lgf_status residual_rebuild(lgf_ctx *ctx) {
  State<double> &S = ctx->s64;
  TRY(timed_begin(ctx, kid<double>(KID_RESIDUAL_GAUGE)));
  k_residual_gauge<NT><<<grid1(ctx->V, NT), NT, 0, ctx->stream>>>(ctx->Kres, S.G, S.A, ctx->V);
  CKL();
  TRY(timed_end(ctx));
  TRY(timed_begin(ctx, kid<double>(KID_RESIDUAL_REBUILD)));
  k_update<double, NT_UPDATE64><<<dim3(grid1(ctx->V, NT_UPDATE64), 1, 1), NT_UPDATE64, update_smem_bytes<NT_UPDATE64>(),
                                  ctx->stream>>>(S.U, S.G, S.A, ctx->L, ctx->ctrl, 0, kid<double>(KID_RESIDUAL_REBUILD),
                                                 ctx->small_step ? 1 : 0, ctx->update_split[0], ctx->update_split[1]);
  CKL();
  TRY(timed_end(ctx));
  Ctrl &c = ctx->ctrl_host;
  ctx->stage = LGF_FP64;
  ctx->prev_theta = 0;
  c.stage = 1;
  c.active = 1;
  TRY(write_ctrl(ctx));
  TRY(launch_delta<double>(ctx, ctx->s64, 0, 0));
  return read_ctrl(ctx);
}

// Timed wrappers of the layout conversions used by load and store.
// nmat = 4: links (stored with LinkStore<T>::planes planes); nmat = 1: a site field of 9 planes.
template <typename T> lgf_status to_planes(lgf_ctx *ctx, const double *src, T *dst, int nmat) {
  TRY(timed_begin(ctx, kid<T>(KID_TO_PLANES)));
  const int np = nmat == 4 ? LinkStore<T>::planes : 9;
  k_aos_to_planes<T><<<grid1((int64_t)nmat * ctx->V, NT), NT, 0, ctx->stream>>>(src, dst, ctx->V, nmat, np, 0,
                                                                                (int64_t)nmat * ctx->V);
  CKL();
  return timed_end(ctx);
}
template <typename T> lgf_status from_planes(lgf_ctx *ctx, const T *src, double *dst, int nmat) {
  TRY(timed_begin(ctx, kid<T>(KID_FROM_PLANES)));
  const int np = nmat == 4 ? LinkStore<T>::planes : 9;
  k_planes_to_aos<T><<<grid1((int64_t)nmat * ctx->V, NT), NT, 0, ctx->stream>>>(src, dst, ctx->V, nmat, np, 0,
                                                                                (int64_t)nmat * ctx->V);
  CKL();
  return timed_end(ctx);
}

// Links from the caller's layout into the working planes for `precision`, for the links i0 .. i0 + n - 1 of
// the 4V (mu-major): FP64 -> double planes; MIXED -> the double planes U0 kept for the handover and the float
// links narrowed from them; FP32 -> float planes.
lgf_status convert_links_in(lgf_ctx *ctx, const double *src, int precision, int64_t i0, int64_t n) {
  const int64_t V = ctx->V;
  if (precision == LGF_FP64) {
    TRY(timed_begin(ctx, kid<double>(KID_TO_PLANES)));
    k_aos_to_planes<double><<<grid1(n, NT), NT, 0, ctx->stream>>>(src, ctx->s64.U, V, 4, 9, i0, n);
    CKL();
    return timed_end(ctx);
  }
  if (precision == LGF_MIXED) {
    TRY(timed_begin(ctx, kid<double>(KID_TO_PLANES)));
    k_aos_to_planes<double><<<grid1(n, NT), NT, 0, ctx->stream>>>(src, ctx->U0, V, 4, 9, i0, n);
    CKL();
    TRY(timed_end(ctx));
    TRY(timed_begin(ctx, kid<float>(KID_TO_PLANES)));
    k_narrow_link_planes<<<grid1(n, NT), NT, 0, ctx->stream>>>(ctx->U0, ctx->s32.U, V, i0, n);
    CKL();
    return timed_end(ctx);
  }
  TRY(timed_begin(ctx, kid<float>(KID_TO_PLANES)));
  k_aos_to_planes<float><<<grid1(n, NT), NT, 0, ctx->stream>>>(src, ctx->s32.U, V, 4, LinkStore<float>::planes, i0, n);
  CKL();
  return timed_end(ctx);
}

// Working planes (double, or float with row 2 rebuilt) -> the caller's layout, links i0 .. i0 + n - 1.
lgf_status convert_links_out(lgf_ctx *ctx, bool from_float, double *dst, int64_t i0, int64_t n) {
  const int64_t V = ctx->V;
  if (from_float) {
    TRY(timed_begin(ctx, kid<float>(KID_FROM_PLANES)));
    k_planes_to_aos<float><<<grid1(n, NT), NT, 0, ctx->stream>>>(ctx->s32.U, dst, V, 4, LinkStore<float>::planes, i0,
                                                                  n);
  } else {
    TRY(timed_begin(ctx, kid<double>(KID_FROM_PLANES)));
    k_planes_to_aos<double><<<grid1(n, NT), NT, 0, ctx->stream>>>(ctx->s64.U, dst, V, 4, 9, i0, n);
  }
  CKL();
  return timed_end(ctx);
}

// Host links are moved in chunks: the copy engine works on a second stream, and each chunk is converted on
// the working stream as soon as it has arrived (loading) or copied out as soon as it has been converted
// (storing), so the conversions overlap the copies. Links below kPipelineMinBytes go in one chunk.
constexpr int kPipelineChunks = 8;
constexpr size_t kPipelineMinBytes = (size_t)64 << 20;

lgf_status ensure_copy_stream(lgf_ctx *ctx) {
  if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  for (int c = 0; c <= kPipelineChunks; ++c)
    if (!ctx->cev[c]) CK(cudaEventCreateWithFlags(&ctx->cev[c], cudaEventDisableTiming));
  return LGF_OK;
}

lgf_status load_host_links(lgf_ctx *ctx, const double *host, int precision) {
  const int64_t nl = 4 * ctx->V;
  const size_t bytes = (size_t)nl * 144;
  TRY(ensure_staging(ctx, &ctx->staging, &ctx->staging_bytes, bytes));
  TRY(ensure_copy_stream(ctx));
  const int nc = bytes >= kPipelineMinBytes ? kPipelineChunks : 1;
  // the copies overwrite the staging buffer only after the working stream's earlier work on it
  CK(cudaEventRecord(ctx->cev[kPipelineChunks], ctx->stream));
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->cev[kPipelineChunks], 0));
  for (int c = 0; c < nc; ++c) {
    const int64_t i0 = nl * c / nc, i1 = nl * (c + 1) / nc;
    CK(cudaMemcpyAsync(ctx->staging + i0 * 18, host + i0 * 18, (size_t)(i1 - i0) * 144, cudaMemcpyHostToDevice,
                       ctx->copy_stream));
    CK(cudaEventRecord(ctx->cev[c], ctx->copy_stream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->cev[c], 0));
    TRY(convert_links_in(ctx, ctx->staging, precision, i0, i1 - i0));
  }
  return LGF_OK;
}

lgf_status store_host_links(lgf_ctx *ctx, bool from_float, double *host) {
  const int64_t nl = 4 * ctx->V;
  const size_t bytes = (size_t)nl * 144;
  TRY(ensure_staging(ctx, &ctx->staging, &ctx->staging_bytes, bytes));
  TRY(ensure_copy_stream(ctx));
  const int nc = bytes >= kPipelineMinBytes ? kPipelineChunks : 1;
  for (int c = 0; c < nc; ++c) {
    const int64_t i0 = nl * c / nc, i1 = nl * (c + 1) / nc;
    TRY(convert_links_out(ctx, from_float, ctx->staging, i0, i1 - i0));
    CK(cudaEventRecord(ctx->cev[c], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->cev[c], 0));
    CK(cudaMemcpyAsync(host + i0 * 18, ctx->staging + i0 * 18, (size_t)(i1 - i0) * 144, cudaMemcpyDeviceToHost,
                       ctx->copy_stream));
  }
  // later work on the working stream (which may reuse the staging buffer) follows the copies
  CK(cudaEventRecord(ctx->cev[kPipelineChunks], ctx->copy_stream));
  CK(cudaStreamWaitEvent(ctx->stream, ctx->cev[kPipelineChunks], 0));
  return LGF_OK;
}

lgf_status upload_hist(lgf_ctx *ctx, const lgf_options *opt) {
  ctx->ctrl_host.hist = nullptr;
  ctx->ctrl_host.hist_len = 0;
  if (opt && opt->history && opt->history_len > 0) {
    if (opt->history_len > ctx->hist_cap) {
      if (ctx->hist_dev) CK(cudaFree(ctx->hist_dev));
      ctx->hist_dev = nullptr;
      CK(cudaMalloc(&ctx->hist_dev, sizeof(double) * 2 * opt->history_len));
      ctx->hist_cap = opt->history_len;
    }
    CK(cudaMemsetAsync(ctx->hist_dev, 0, sizeof(double) * 2 * opt->history_len, ctx->stream));
    ctx->ctrl_host.hist = ctx->hist_dev;
    ctx->ctrl_host.hist_len = opt->history_len;
  }
  return LGF_OK;
}

lgf_status check_ctx(lgf_ctx *ctx) {
  if (!ctx) return fail(nullptr, LGF_EINVAL, "null context");
  if (ctx->poisoned) return LGF_ECUDA;
  CK(cudaSetDevice(ctx->device));
  return LGF_OK;
}

}  // namespace

// Library-internal (not exported): lets other translation units of the library report a message
// through lgf_last_error(NULL).
// msg must be a string with static storage (it is kept by pointer; nothing is allocated). NULL clears it.
__attribute__((visibility("hidden"))) void lgf_set_static_error(const char *msg) { g_static_literal = msg; }

static lgf_status create_ctx(const int n[4], int nb, lgf_ctx **out);

// ============================================== C ABI ===============================================
extern "C" {

void lgf_default_options(lgf_options *opt) {
  if (!opt) return;
  opt->fft32_final = 0;
  opt->precision = LGF_FP64;
  opt->theta_switch = 1e-11;
  opt->reunit_period = 16;
  opt->max_iter = 100000;
  opt->history = nullptr;
  opt->history_len = 0;
}

lgf_status lgf_create(int Nx, int Ny, int Nz, int Nt, lgf_ctx **out) {
  const int n[4] = {Nx, Ny, Nz, Nt};
  return create_ctx(n, 1, out);
}

}  // extern "C"

// A context for nb configurations of one lattice shape (nb = 1 for lgf_create).
static lgf_status create_ctx(const int n[4], int nb, lgf_ctx **out) {
  if (!out) return fail(nullptr, LGF_EINVAL, "null output pointer");
  *out = nullptr;
  const int Nx = n[0], Ny = n[1], Nz = n[2], Nt = n[3];
  for (int mu = 0; mu < 4; ++mu)
    if (!factor_ok(n[mu]))
      return fail(nullptr, LGF_EINVAL, "lattice extents must be in [2, 1024] and products of 2, 3 and 5");
  // site indices are decomposed with 32-bit arithmetic in the kernels (such a lattice needs over 1 TB of
  // links in any case)
  if ((int64_t)Nx * Ny * Nz * Nt >= ((int64_t)1 << 31))
    return fail(nullptr, LGF_EINVAL, "the lattice volume must be below 2^31 sites");
  lgf_ctx *ctx = new lgf_ctx();
  ctx->nb = nb;
  for (int mu = 0; mu < 4; ++mu) ctx->n[mu] = n[mu];
  ctx->V = (int64_t)Nx * Ny * Nz * Nt;
  ctx->L.V = ctx->V;
  int64_t st = 1;
  for (int mu = 0; mu < 4; ++mu) {
    ctx->L.n[mu] = n[mu];
    ctx->L.stride[mu] = st;
    st *= n[mu];
  }
  auto bail = [&](lgf_status s, const std::string &m) {
    g_last_static_error = m;
    g_static_literal = nullptr;
    delete ctx;
    return s;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(LGF_ECUDA, "no CUDA device");
  if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(LGF_ECUDA, "cudaStreamCreate failed");
  ctx->stream = ctx->own_stream;
  {
    // LGF_GENERIC_FFT=1 forces the generic FFT passes (used by the tests to check both families)
    const char *g = std::getenv("LGF_GENERIC_FFT");
    ctx->generic_fft = g && g[0] == '1';
    const char *nf = std::getenv("LGF_FFT_NATIVE_F64");
    ctx->fft_df64 = !(nf && nf[0] == '1');
    const char *ss = std::getenv("LGF_SMALL_STEP");
    ctx->small_step = !(ss && ss[0] == '0');
    const char *rs = std::getenv("LGF_RESIDUAL");
    ctx->residual = !(rs && rs[0] == '0');
    const char *hf = std::getenv("LGF_HANDOVER_FP64");
    ctx->handover_fp64 = hf && hf[0] == '1';
    // LGF_HANDOVER_SPLIT=ab (two digits 0-4): links per site that the handover transform forms in FP64 in
    // even and in odd warps, the others in 61-bit fixed point (default 22; 00 is fixed point alone)
    const char *hs = std::getenv("LGF_HANDOVER_SPLIT");
    if (hs && hs[0] >= '0' && hs[0] <= '4' && hs[1] >= '0' && hs[1] <= '4') {
      ctx->handover_split[0] = hs[0] - '0';
      ctx->handover_split[1] = hs[1] - '0';
    }
    // LGF_UPDATE_SPLIT=ab: the same for the general (large-step) form of the double update (default 22;
    // 44 is FP64 alone, 00 fixed point alone)
    const char *us = std::getenv("LGF_UPDATE_SPLIT");
    if (us && us[0] >= '0' && us[0] <= '4' && us[1] >= '0' && us[1] <= '4') {
      ctx->update_split[0] = us[0] - '0';
      ctx->update_split[1] = us[1] - '0';
    }
    const char *rf = std::getenv("LGF_REUNIT_FP64");
    ctx->reunit_fp64 = rf && rf[0] == '1';
  }
  cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (ctx->num_sms < 1) ctx->num_sms = 1;
  {
    const char *fp = std::getenv("LGF_FFT_PERSIST");
    ctx->fft_persist = !(fp && fp[0] == '0');
    const char *tr = std::getenv("LGF_TFILTER_REG");
    ctx->tfilter_reg = !(tr && tr[0] == '0');
    const char *xr = std::getenv("LGF_XY_REG");
    ctx->xy_reg = !(xr && xr[0] == '0');
    const char *tw = std::getenv("LGF_TWALK");
    ctx->twalk = !(tw && tw[0] == '0');
    const char *tmb = std::getenv("LGF_TWALK_MIN_BLOCKS");
    if (tmb) ctx->twalk_min_blocks = std::atoll(tmb);
  }
  // p^2 tables (position -> 4 sin^2(pi k / N)) and the filter scale p^2_max / V
  double p2max = 0;
  for (int mu = 0; mu < 4; ++mu) {
    ctx->ax[mu] = make_axis(n[mu]);
    std::vector<int> kpos;
    digit_reversed_freq(ctx->ax[mu], kpos);
    std::vector<double> part(n[mu]);
    for (int p = 0; p < n[mu]; ++p) {
      const double sn = std::sin(M_PI * (double)kpos[p] / (double)n[mu]);
      part[p] = 4.0 * sn * sn;
    }
    const double sm = std::sin(M_PI * (double)(n[mu] / 2) / (double)n[mu]);
    p2max += 4.0 * sm * sm;
    if (cudaMalloc(&ctx->p2part[mu], sizeof(double) * n[mu]) != cudaSuccess ||
        cudaMemcpy(ctx->p2part[mu], part.data(), sizeof(double) * n[mu], cudaMemcpyHostToDevice) != cudaSuccess) {
      lgf_destroy(ctx);
      g_last_static_error = "allocation of FFT tables failed";
      g_static_literal = nullptr;
      return LGF_ENOMEM;
    }
  }
  ctx->wscale = p2max / (double)ctx->V;
  *out = ctx;
  return LGF_OK;
}

extern "C" {

void lgf_destroy(lgf_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  auto fr = [](void *p) {
    if (p) cudaFree(p);
  };
  fr(ctx->s64.U);
  fr(ctx->s64.P);
  fr(ctx->s64.G);
  fr(ctx->s64.A);
  fr(ctx->s32.U);
  fr(ctx->s32.P);
  fr(ctx->s32.G);
  for (int mu = 0; mu < 4; ++mu) {
    fr(ctx->s64.tw[mu]);
    fr(ctx->s32.tw[mu]);
    fr(ctx->p2part[mu]);
  }
  fr(ctx->U0);
  fr(ctx->Wev);
  fr(ctx->lam);
  fr(ctx->Gacc);
  fr(ctx->Rres);
  fr(ctx->Kres);
  fr(ctx->staging);
  fr(ctx->staging2);
  fr(ctx->partials);
  fr(ctx->ctrl);
  fr(ctx->hist_dev);
  fr(ctx->ran_dev);
  for (auto &e : ctx->ev_pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  for (auto e : ctx->cev)
    if (e) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  delete ctx;
}

const char *lgf_last_error(const lgf_ctx *ctx) {
  if (!ctx) return g_static_literal ? g_static_literal : g_last_static_error.c_str();
  return ctx->err.c_str();
}

lgf_status lgf_set_stream(lgf_ctx *ctx, void *stream) {
  TRY(check_ctx(ctx));
  ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
  return LGF_OK;
}

lgf_status lgf_load(lgf_ctx *ctx, const double *links, int precision) {
  TRY(check_ctx(ctx));
  if (precision != LGF_FP64 && precision != LGF_MIXED && precision != LGF_FP32)
    return fail(ctx, LGF_EINVAL, "unknown precision");
  TRY(ensure_common(ctx));
  const int64_t V = ctx->V;
  if (!links) return fail(ctx, LGF_EINVAL, "null buffer");
  const PtrKind kind = ptr_kind(links, ctx->device);
  if (kind == PTR_OTHER_DEVICE) return fail(ctx, LGF_EINVAL, "device buffer belongs to another GPU than the context's");
  if (kind == PTR_DEVICE && (((uintptr_t)links) & 15))
    return fail(ctx, LGF_EINVAL, "device buffers must be 16-byte aligned");
  memset(&ctx->ctrl_host, 0, sizeof(Ctrl));
  ctx->ctrl_host.active = 1;
  ctx->ctrl_host.limit = 0;
  ctx->ctrl_host.threshold = 0;
  ctx->ctrl_host.stage = precision == LGF_FP64 ? 1 : 0;
  TRY(write_ctrl(ctx));
  if (precision == LGF_FP64) {
    TRY(setup_precision<double>(ctx, ctx->s64));
  } else {
    TRY(setup_precision<float>(ctx, ctx->s32));
    TRY(alloc(ctx, &ctx->Gacc, (size_t)ctx->nb * 6 * V * 2));
    // mixed: the caller's links are read once, into the double planes kept for the handover, and the
    // float links are narrowed from those
    if (precision == LGF_MIXED) TRY(alloc(ctx, &ctx->U0, (size_t)ctx->nb * 4 * 9 * V * 2));
  }
  if (kind == PTR_HOST) TRY(load_host_links(ctx, links, precision));
  else TRY(convert_links_in(ctx, links, precision, 0, 4 * V));
  if (precision == LGF_FP64) {
    TRY(launch_delta<double>(ctx, ctx->s64, 0, 0));
    ctx->stage = LGF_FP64;
  } else {
    TRY(timed_begin(ctx, kid<float>(KID_SET_IDENTITY)));
    k_set_identity<<<grid1(V, NT), NT, 0, ctx->stream>>>(ctx->Gacc, V);
    CKL();
    TRY(timed_end(ctx));
    TRY(launch_delta<float>(ctx, ctx->s32, 0, 0));
    ctx->stage = LGF_FP32;
  }
  TRY(read_ctrl(ctx));
  ctx->loaded = true;
  ctx->load_prec = precision;
  ctx->since_reunit = 0;
  ctx->prev_theta = 0;
  ctx->prev_iters = 0;
  ctx->resid_off = false;
  return LGF_OK;
}

lgf_status lgf_iterate(lgf_ctx *ctx, int max_new, double alpha, double eps, const lgf_options *opt, double *theta,
                       double *F, int *iters) {
  TRY(check_ctx(ctx));
  if (!ctx->loaded) return fail(ctx, LGF_EINVAL, "lgf_iterate before lgf_load");
  if (max_new < 0 || !(alpha > 0) || !(eps >= 0)) return fail(ctx, LGF_EINVAL, "bad max_new, alpha or eps");
  lgf_options o;
  lgf_default_options(&o);
  if (opt) o = *opt;
  if (o.reunit_period < 1) o.reunit_period = 1;
  TRY(upload_hist(ctx, opt));
  if (ctx->ctrl_host.hist && ctx->ctrl_host.iters < ctx->ctrl_host.hist_len) {
    // record the state the call starts from
    double h[2] = {ctx->ctrl_host.theta, ctx->ctrl_host.F};
    CK(cudaMemcpyAsync(ctx->ctrl_host.hist + 2 * ctx->ctrl_host.iters, h, sizeof h, cudaMemcpyHostToDevice,
                       ctx->stream));
  }
  const int target = ctx->ctrl_host.iters + max_new;
  lgf_status result = LGF_ENOCONV;
  for (;;) {
    const bool float_stage = ctx->stage == LGF_FP32;
    const bool mixed_float = float_stage && ctx->load_prec == LGF_MIXED;
    const bool resid_stage = ctx->stage == kHostStageResidual;
    // the residual stage stops a little below eps: its float theta is checked again in double after
    // the rebuild
    const double thr = mixed_float ? std::max(eps, o.theta_switch) : resid_stage ? 0.8 * eps : eps;
    Ctrl &c = ctx->ctrl_host;
    if (c.status == 5) {
      result = LGF_ENONFINITE;
      break;
    }
    // the mixed schedule past the handover continues in the residual stage while theta >= eps
    if (ctx->stage == LGF_FP64 && ctx->load_prec == LGF_MIXED && ctx->residual && !o.fft32_final &&
        !ctx->resid_off && !(c.theta < eps) && c.iters < target) {
      TRY(residual_begin(ctx));
      continue;
    }
    // a float or residual stage that no longer lowers theta over a chunk of iterations has reached what
    // its float arithmetic resolves: it hands over (or rebuilds) at once
    const bool stalled = (mixed_float || resid_stage) && ctx->prev_theta > 0 && ctx->prev_iters < c.iters &&
                         !(c.theta < ctx->prev_theta);
    if (c.theta < thr || c.iters >= target || stalled) {
      if (resid_stage) {
        // rebuild the double links; without progress over the stage the double iterations take over
        const double theta0 = ctx->resid_theta0;
        TRY(residual_rebuild(ctx));
        if (!(ctx->ctrl_host.theta < theta0)) ctx->resid_off = true;
        continue;
      }
      if (mixed_float && (c.theta < thr || stalled)) {
        // hand over to double precision: rebuild the links from the input and G, then Delta, theta, F
        TRY(handover(ctx, ctx->residual && !o.fft32_final));
        ctx->stage = LGF_FP64;
        ctx->prev_theta = 0;
        c.active = 1;
        c.stage = 1;
        TRY(write_ctrl(ctx));
        if (o.fft32_final) TRY(launch_delta_d2f(ctx, 0, 0));
        else TRY(launch_delta<double>(ctx, ctx->s64, 0, 0));
        TRY(read_ctrl(ctx));
        continue;
      }
      result = (c.theta < eps) ? LGF_OK : LGF_ENOCONV;
      break;
    }
    c.threshold = thr;
    c.limit = target;
    c.active = 1;
    TRY(write_ctrl(ctx));
    // a chunk of iterations without host round trips; kernels return at once after the loop stops.
    // The chunk is sized from the observed geometric convergence rate so that few launches are idle.
    int chunk = 8;
    if (ctx->prev_theta > 0 && c.theta > 0 && c.theta < ctx->prev_theta && ctx->prev_iters < c.iters) {
      const double rate = std::pow(c.theta / ctx->prev_theta, 1.0 / (c.iters - ctx->prev_iters));
      const double need = std::ceil(std::log(thr / c.theta) / std::log(rate));
      if (need >= 1 && need < chunk) chunk = (int)need;
    }
    ctx->prev_theta = c.theta;
    ctx->prev_iters = c.iters;
    for (int k = 0; k < chunk; ++k) {
      if (resid_stage) {
        TRY(launch_iteration_residual(ctx, alpha));
      } else if (float_stage) {
        const bool reunit = ++ctx->since_reunit >= o.reunit_period;
        if (reunit) ctx->since_reunit = 0;
        TRY(launch_iteration_float(ctx, alpha, reunit));
      } else if (o.fft32_final && ctx->load_prec == LGF_MIXED) {
        TRY(launch_iteration_fft32(ctx, alpha));
      } else {
        TRY(launch_iteration<double>(ctx, ctx->s64, alpha));
      }
    }
    TRY(read_ctrl(ctx));
  }
  if (theta) *theta = ctx->ctrl_host.theta;
  if (F) *F = ctx->ctrl_host.F;
  if (iters) *iters = ctx->ctrl_host.iters;
  if (opt && opt->history && opt->history_len > 0) {
    CK(cudaMemcpyAsync(opt->history, ctx->hist_dev, sizeof(double) * 2 * opt->history_len, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (result == LGF_ENONFINITE) return fail(ctx, LGF_ENONFINITE, "theta or F is not finite");
  return result;
}

lgf_status lgf_store(lgf_ctx *ctx, double *links) {
  TRY(check_ctx(ctx));
  if (!ctx->loaded) return fail(ctx, LGF_EINVAL, "lgf_store before lgf_load");
  const int64_t V = ctx->V;
  if (!links) return fail(ctx, LGF_EINVAL, "null buffer");
  const PtrKind kind = ptr_kind(links, ctx->device);
  if (kind == PTR_OTHER_DEVICE) return fail(ctx, LGF_EINVAL, "device buffer belongs to another GPU than the context's");
  if (kind == PTR_DEVICE && (((uintptr_t)links) & 15))
    return fail(ctx, LGF_EINVAL, "device buffers must be 16-byte aligned");
  if (ctx->stage == kHostStageResidual) TRY(residual_rebuild(ctx));
  bool from_float = false;
  if (ctx->stage != LGF_FP64) {
    if (ctx->load_prec == LGF_MIXED) TRY(handover(ctx));
    else from_float = true;
  }
  if (kind == PTR_HOST) TRY(store_host_links(ctx, from_float, links));
  else TRY(convert_links_out(ctx, from_float, links, 0, 4 * V));
  CK(cudaStreamSynchronize(ctx->stream));
  return LGF_OK;
}

lgf_status lgf_fix(lgf_ctx *ctx, double *links, double alpha, double eps, const lgf_options *opt, double *theta_out,
                   double *F_out, int *iters_out) {
  lgf_options o;
  lgf_default_options(&o);
  if (opt) o = *opt;
  TRY(lgf_load(ctx, links, o.precision));
  double th = 0, F = 0;
  int it = 0;
  lgf_status st = lgf_iterate(ctx, o.max_iter, alpha, eps, &o, &th, &F, &it);
  if (st != LGF_OK && st != LGF_ENOCONV) return st;
  TRY(lgf_store(ctx, links));
  if (theta_out) *theta_out = th;
  if (F_out) *F_out = F;
  if (iters_out) *iters_out = it;
  return st;
}

lgf_status lgf_measure(lgf_ctx *ctx, const double *links, double *theta, double *F, double *plaq) {
  TRY(check_ctx(ctx));
  TRY(ensure_common(ctx));
  TRY(setup_precision<double>(ctx, ctx->s64));
  const int64_t V = ctx->V;
  const double *src = nullptr;
  TRY(input_ptr(ctx, links, (size_t)4 * V * 9 * 16, &ctx->staging, &ctx->staging_bytes, &src));
  k_aos_to_planes<double><<<grid1(4 * V, NT), NT, 0, ctx->stream>>>(src, ctx->s64.U, V, 4, 9, 0, 4 * V);
  CKL();
  memset(&ctx->ctrl_host, 0, sizeof(Ctrl));
  TRY(write_ctrl(ctx));
  TRY(launch_delta<double>(ctx, ctx->s64, 0, 0));
  if (plaq) {
    // stream-ordered after the Delta reduction, which leaves the last-block counter at zero
    k_plaquette<double, NT><<<ctx->nblocks_site, NT, 0, ctx->stream>>>(ctx->s64.U, ctx->partials, ctx->ctrl, ctx->L);
    CKL();
  }
  TRY(read_ctrl(ctx));
  if (theta) *theta = ctx->ctrl_host.theta;
  if (F) *F = ctx->ctrl_host.F;
  if (plaq) *plaq = ctx->ctrl_host.plaq;
  ctx->loaded = false;  // the working links were overwritten
  return LGF_OK;
}

}  // extern "C"

// ---------------------------------- single steps ----------------------------------
// Full site matrices <-> the state's packed buffer (in the state's FFT type).
template <typename T> static lgf_status pack_field(lgf_ctx *ctx, State<T> &S, const double *src) {
  return with_fft_type<T>(ctx, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    k_pack_antiherm<FT><<<grid1(ctx->V, NT), NT, 0, ctx->stream>>>(src, reinterpret_cast<FT *>(S.P), ctx->V);
    CKL();
    return LGF_OK;
  });
}
template <typename T> static lgf_status unpack_field(lgf_ctx *ctx, State<T> &S, double *dst) {
  return with_fft_type<T>(ctx, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    k_unpack_antiherm<FT><<<grid1(ctx->V, NT), NT, 0, ctx->stream>>>(reinterpret_cast<const FT *>(S.P), dst, ctx->V);
    CKL();
    return LGF_OK;
  });
}
template <typename T> static lgf_status step_delta(lgf_ctx *ctx, State<T> &S, const double *src, double *dst,
                                                   double *theta, double *F) {
  const int64_t V = ctx->V;
  k_aos_to_planes<T><<<grid1(4 * V, NT), NT, 0, ctx->stream>>>(src, S.U, V, 4, LinkStore<T>::planes, 0, 4 * V);
  CKL();
  memset(&ctx->ctrl_host, 0, sizeof(Ctrl));
  TRY(write_ctrl(ctx));
  if constexpr (std::is_same<T, double>::value) {
    // the caller gets Delta in full FP64: pack it as double, not as the type of the double path's FFT
    k_delta<double, NT, double><<<dim3(ctx->nblocks_site, 1, 1), NT, 0, ctx->stream>>>(
        S.U, S.P, ctx->partials, ctx->ctrl, ctx->L, 0, 0, kid<T>(KID_DELTA));
    CKL();
    k_unpack_antiherm<double><<<grid1(V, NT), NT, 0, ctx->stream>>>(S.P, dst, V);
    CKL();
  } else {
    TRY(launch_delta<T>(ctx, S, 0, 0));
    TRY(unpack_field<T>(ctx, S, dst));
  }
  TRY(read_ctrl(ctx));
  if (theta) *theta = ctx->ctrl_host.theta;
  if (F) *F = ctx->ctrl_host.F;
  return LGF_OK;
}

extern "C" lgf_status lgf_delta(lgf_ctx *ctx, const double *links, double *delta, double *theta, double *F, int precision) {
  TRY(check_ctx(ctx));
  TRY(ensure_common(ctx));
  const int64_t V = ctx->V;
  const double *src = nullptr;
  TRY(input_ptr(ctx, links, (size_t)4 * V * 144, &ctx->staging, &ctx->staging_bytes, &src));
  double *dst = nullptr;
  bool host = false;
  TRY(output_ptr(ctx, delta, (size_t)V * 144, &ctx->staging2, &ctx->staging2_bytes, &dst, &host));
  if (precision == LGF_FP32) {
    TRY(setup_precision<float>(ctx, ctx->s32));
    TRY(step_delta<float>(ctx, ctx->s32, src, dst, theta, F));
  } else {
    TRY(setup_precision<double>(ctx, ctx->s64));
    TRY(step_delta<double>(ctx, ctx->s64, src, dst, theta, F));
  }
  if (host) CK(cudaMemcpyAsync(delta, dst, (size_t)V * 144, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->loaded = false;
  return LGF_OK;
}

template <typename T> static lgf_status step_filter(lgf_ctx *ctx, State<T> &S, const double *src, double *dst) {
  const int64_t V = ctx->V;
  TRY(pack_field<T>(ctx, S, src));
  TRY(launch_filter<T>(ctx, S, S.P, 0));
  TRY(unpack_field<T>(ctx, S, dst));
  (void)V;
  return LGF_OK;
}

extern "C" lgf_status lgf_filter(lgf_ctx *ctx, const double *delta, double *dtilde, int precision) {
  TRY(check_ctx(ctx));
  TRY(ensure_common(ctx));
  const int64_t V = ctx->V;
  const double *src = nullptr;
  TRY(input_ptr(ctx, delta, (size_t)V * 144, &ctx->staging, &ctx->staging_bytes, &src));
  double *dst = nullptr;
  bool host = false;
  TRY(output_ptr(ctx, dtilde, (size_t)V * 144, &ctx->staging2, &ctx->staging2_bytes, &dst, &host));
  if (precision == LGF_FP32) {
    TRY(setup_precision<float>(ctx, ctx->s32));
    TRY(step_filter<float>(ctx, ctx->s32, src, dst));
  } else {
    TRY(setup_precision<double>(ctx, ctx->s64));
    TRY(step_filter<double>(ctx, ctx->s64, src, dst));
  }
  if (host) CK(cudaMemcpyAsync(dtilde, dst, (size_t)V * 144, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->loaded = false;
  return LGF_OK;
}

template <typename T>
static lgf_status step_filter_coeffs(lgf_ctx *ctx, State<T> &S, const double *src, double *dst) {
  TRY(with_fft_type<T>(ctx, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    k_pack_coeffs<FT><<<grid1(ctx->V, NT), NT, 0, ctx->stream>>>(src, reinterpret_cast<FT *>(S.P), ctx->V);
    CKL();
    return LGF_OK;
  }));
  TRY(launch_filter<T>(ctx, S, S.P, 0));
  return with_fft_type<T>(ctx, [&](auto tag) -> lgf_status {
    using FT = decltype(tag);
    k_unpack_coeffs<FT><<<grid1(ctx->V, NT), NT, 0, ctx->stream>>>(reinterpret_cast<const FT *>(S.P), dst, ctx->V);
    CKL();
    return LGF_OK;
  });
}

extern "C" lgf_status lgf_filter_coeffs(lgf_ctx *ctx, const double *coef, double *out, int precision) {
  TRY(check_ctx(ctx));
  TRY(ensure_common(ctx));
  const int64_t V = ctx->V;
  const double *src = nullptr;
  TRY(input_ptr(ctx, coef, (size_t)V * 64, &ctx->staging, &ctx->staging_bytes, &src));
  double *dst = nullptr;
  bool host = false;
  TRY(output_ptr(ctx, out, (size_t)V * 64, &ctx->staging2, &ctx->staging2_bytes, &dst, &host));
  if (precision == LGF_FP32) {
    TRY(setup_precision<float>(ctx, ctx->s32));
    TRY(step_filter_coeffs<float>(ctx, ctx->s32, src, dst));
  } else {
    TRY(setup_precision<double>(ctx, ctx->s64));
    TRY(step_filter_coeffs<double>(ctx, ctx->s64, src, dst));
  }
  if (host) CK(cudaMemcpyAsync(out, dst, (size_t)V * 64, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->loaded = false;
  return LGF_OK;
}

template <typename T> static lgf_status step_gauge(lgf_ctx *ctx, State<T> &S, const double *src, double alpha,
                                                   double *dst) {
  const int64_t V = ctx->V;
  if constexpr (std::is_same<T, double>::value) {
    // Delta-tilde from the caller is taken in full FP64 (packed as double)
    k_pack_antiherm<double><<<grid1(V, NT), NT, 0, ctx->stream>>>(src, S.P, V);
    CKL();
    k_gauge<double, NT, double><<<dim3(grid1(V, NT), 1, 1), NT, 0, ctx->stream>>>(
        S.P, S.G, S.A, 0.5 * alpha, V, ctx->ctrl, 0, kid<T>(KID_GAUGE), ctx->small_step ? 1 : 0);
    CKL();
  } else {
    TRY(pack_field<T>(ctx, S, src));
    TRY(launch_gauge<T>(ctx, S, alpha, 0));
  }
  k_planes_to_aos<T><<<grid1(V, NT), NT, 0, ctx->stream>>>(S.G, dst, V, 1, 9, 0, V);
  CKL();
  return LGF_OK;
}

extern "C" lgf_status lgf_gauge(lgf_ctx *ctx, const double *dtilde, double alpha, double *g, int precision) {
  TRY(check_ctx(ctx));
  TRY(ensure_common(ctx));
  const int64_t V = ctx->V;
  const double *src = nullptr;
  TRY(input_ptr(ctx, dtilde, (size_t)V * 144, &ctx->staging, &ctx->staging_bytes, &src));
  double *dst = nullptr;
  bool host = false;
  TRY(output_ptr(ctx, g, (size_t)V * 144, &ctx->staging2, &ctx->staging2_bytes, &dst, &host));
  if (precision == LGF_FP32) {
    TRY(setup_precision<float>(ctx, ctx->s32));
    TRY(step_gauge<float>(ctx, ctx->s32, src, alpha, dst));
  } else {
    TRY(setup_precision<double>(ctx, ctx->s64));
    TRY(step_gauge<double>(ctx, ctx->s64, src, alpha, dst));
  }
  if (host) CK(cudaMemcpyAsync(g, dst, (size_t)V * 144, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->loaded = false;
  return LGF_OK;
}

template <typename T> static lgf_status step_update(lgf_ctx *ctx, State<T> &S, const double *lsrc, const double *gsrc,
                                                    double *dst) {
  const int64_t V = ctx->V;
  k_aos_to_planes<T><<<grid1(4 * V, NT), NT, 0, ctx->stream>>>(lsrc, S.U, V, 4, LinkStore<T>::planes, 0, 4 * V);
  CKL();
  k_aos_to_planes<T><<<grid1(V, NT), NT, 0, ctx->stream>>>(gsrc, S.G, V, 1, 9, 0, V);
  CKL();
  if constexpr (std::is_same<T, double>::value) {
    k_a_from_g<NT><<<grid1(V, NT), NT, 0, ctx->stream>>>(S.G, S.A, V);
    CKL();
  }
  TRY(launch_update<T>(ctx, S, 0));
  k_planes_to_aos<T><<<grid1(4 * V, NT), NT, 0, ctx->stream>>>(S.U, dst, V, 4, LinkStore<T>::planes, 0, 4 * V);
  CKL();
  return LGF_OK;
}

extern "C" lgf_status lgf_update(lgf_ctx *ctx, double *links, const double *g, int precision) {
  TRY(check_ctx(ctx));
  TRY(ensure_common(ctx));
  const int64_t V = ctx->V;
  double *ldev = nullptr;
  bool host = false;
  TRY(output_ptr(ctx, links, (size_t)4 * V * 144, &ctx->staging, &ctx->staging_bytes, &ldev, &host));
  if (host) CK(cudaMemcpyAsync(ldev, links, (size_t)4 * V * 144, cudaMemcpyHostToDevice, ctx->stream));
  const double *gdev = nullptr;
  TRY(input_ptr(ctx, g, (size_t)V * 144, &ctx->staging2, &ctx->staging2_bytes, &gdev));
  if (precision == LGF_FP32) {
    TRY(setup_precision<float>(ctx, ctx->s32));
    TRY(step_update<float>(ctx, ctx->s32, ldev, gdev, ldev));
  } else {
    TRY(setup_precision<double>(ctx, ctx->s64));
    TRY(step_update<double>(ctx, ctx->s64, ldev, gdev, ldev));
  }
  if (host) CK(cudaMemcpyAsync(links, ldev, (size_t)4 * V * 144, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->loaded = false;
  return LGF_OK;
}

// ------------------------------ differentiable functional ------------------------------
// Shared set-up of lgf_functional / lgf_functional_grad: links to planes, omega -> g, W, l.
static lgf_status prepare_functional(lgf_ctx *ctx, const double *links, const double *omega) {
  TRY(check_ctx(ctx));
  TRY(ensure_common(ctx));
  TRY(setup_precision<double>(ctx, ctx->s64));
  const int64_t V = ctx->V;
  TRY(alloc(ctx, &ctx->Wev, (size_t)9 * V * 2));
  TRY(alloc(ctx, &ctx->lam, (size_t)3 * V));
  const double *ldev = nullptr, *odev = nullptr;
  TRY(input_ptr(ctx, links, (size_t)4 * V * 144, &ctx->staging, &ctx->staging_bytes, &ldev));
  TRY(input_ptr(ctx, omega, (size_t)V * 64, &ctx->staging2, &ctx->staging2_bytes, &odev));
  TRY(to_planes<double>(ctx, ldev, ctx->s64.U, 4));
  k_expi<NT><<<grid1(V, NT), NT, 0, ctx->stream>>>(odev, ctx->s64.G, ctx->Wev, ctx->lam, V);
  CKL();
  ctx->loaded = false;  // the working links were overwritten
  return LGF_OK;
}

extern "C" lgf_status lgf_functional(lgf_ctx *ctx, const double *links, const double *omega, double *F,
                                     double *g_out) {
  TRY(prepare_functional(ctx, links, omega));
  const int64_t V = ctx->V;
  memset(&ctx->ctrl_host, 0, sizeof(Ctrl));
  TRY(write_ctrl(ctx));
  k_functional_g<NT><<<ctx->nblocks_site, NT, 0, ctx->stream>>>(ctx->s64.U, ctx->s64.G, ctx->partials, ctx->ctrl,
                                                                ctx->L);
  CKL();
  if (g_out) {
    double *gdev = nullptr;
    bool host = false;
    TRY(output_ptr(ctx, g_out, (size_t)V * 144, &ctx->staging, &ctx->staging_bytes, &gdev, &host));
    TRY(from_planes<double>(ctx, ctx->s64.G, gdev, 1));
    if (host) CK(cudaMemcpyAsync(g_out, gdev, (size_t)V * 144, cudaMemcpyDeviceToHost, ctx->stream));
  }
  TRY(read_ctrl(ctx));
  if (F) *F = ctx->ctrl_host.F;
  return LGF_OK;
}

extern "C" lgf_status lgf_functional_grad(lgf_ctx *ctx, const double *links, const double *omega, double scale,
                                          double *grad) {
  TRY(prepare_functional(ctx, links, omega));
  const int64_t V = ctx->V;
  double *gdev = nullptr;
  bool host = false;
  TRY(output_ptr(ctx, grad, (size_t)V * 64, &ctx->staging, &ctx->staging_bytes, &gdev, &host));
  k_functional_grad<NT><<<grid1(V, NT), NT, 0, ctx->stream>>>(ctx->s64.U, ctx->s64.G, ctx->Wev, ctx->lam, gdev,
                                                              ctx->L, scale);
  CKL();
  if (host) CK(cudaMemcpyAsync(grad, gdev, (size_t)V * 64, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LGF_OK;
}

extern "C" {

lgf_status lgf_enable_timing(lgf_ctx *ctx, int enable) {
  TRY(check_ctx(ctx));
  if (enable && !ctx->ran_dev) {
    CK(cudaMalloc(&ctx->ran_dev, sizeof(unsigned int) * 2 * KID_COUNT));
    CK(cudaMemset(ctx->ran_dev, 0, sizeof(unsigned int) * 2 * KID_COUNT));
  }
  ctx->timing = enable != 0;
  return LGF_OK;
}

lgf_status lgf_kernel_times(lgf_ctx *ctx, const char **name, long *launches, double *ms, int cap, int *count) {
  TRY(check_ctx(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  TRY(timed_collect(ctx));
  if (ctx->ran_dev) {
    // kernels of the loop return at once after the loop has stopped: report the launches that ran
    unsigned int ran[2 * KID_COUNT];
    CK(cudaMemcpy(ran, ctx->ran_dev, sizeof ran, cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->ran_dev, 0, sizeof ran));
    const int loop_kids[] = {KID_DELTA, KID_FFT_XY_FWD, KID_FFT_X_FWD, KID_FFT_Y_FWD, KID_FFT_Z_FWD,
                             KID_FFT_ZT_FILTER, KID_FFT_T_FILTER, KID_FFT_Z_INV, KID_FFT_Y_INV, KID_FFT_X_INV,
                             KID_FFT_XY_INV, KID_GAUGE, KID_UPDATE, KID_UPDATE_FUSED, KID_UPDATE_FUSED_REUNIT,
                             KID_DELTA_RESIDUAL, KID_UPDATE_RESIDUAL};
    for (int k : loop_kids)
      for (int h = 0; h < 2; ++h) {
        const int i = k + h * KID_COUNT;
        if (ctx->klaunch[i] > 0) ctx->klaunch[i] = ran[i];
        if (ctx->klaunch[i] == 0) ctx->kms[i] = 0;
      }
  }
  int k = 0;
  if (kKernelNames[0].empty())
    for (int i = 0; i < 2 * KID_COUNT; ++i)
      kKernelNames[i] = std::string(kKernelBase[i % KID_COUNT]) + (i < KID_COUNT ? ".f64" : ".f32");
  for (int i = 0; i < 2 * KID_COUNT; ++i)
    if (ctx->klaunch[i] > 0) {
      if (k < cap) {
        if (name) name[k] = kKernelNames[i].c_str();
        if (launches) launches[k] = ctx->klaunch[i];
        if (ms) ms[k] = ctx->kms[i];
      }
      ++k;
      ctx->klaunch[i] = 0;
      ctx->kms[i] = 0;
    }
  if (count) *count = k;
  return LGF_OK;
}

}  // extern "C"

#include "batch.cuh"
