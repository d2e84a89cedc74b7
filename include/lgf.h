/*
 * lgf.h -- C ABI of the GB300 (sm_103a) library for Fourier-accelerated steepest-descent Landau gauge
 * fixing of SU(3) lattice gauge fields (Cardoso, Silva, Oliveira, Bicudo, "GPU implementation of a
 * Landau gauge fixing algorithm", Lattice 2012).
 *
 * The method maximises F_U[g] (Eq. 1) on the gauge orbit of U. Each iteration of Algorithm 1 computes
 * Delta(x) (Eqs. 3, 5), theta (Eq. 4) and F, Fourier-filters Delta with p^2_max/p^2 (Eq. 2), forms
 * g(x) = SU(3)-projection of [1 + (alpha/2) Delta-tilde(x)] and applies U_mu(x) -> g(x)U_mu(x)g^+(x+mu).
 * The loop stops when theta < eps (Algorithm 1: "while theta >= eps").
 *
 * Conventions shared by every entry point
 *   Lattice: Nx, Ny, Nz, Nt, periodic; V = Nx*Ny*Nz*Nt; site s = x + Nx*(y + Ny*(z + Nz*t)).
 *   Links (caller-owned): 4*V*9 complex doubles (re, im interleaved), index ((mu*V + s)*3 + i)*3 + j
 *     for direction mu in {x,y,z,t}, row i, column j; i.e. a contiguous complex128 array of shape
 *     (4, Nt, Nz, Ny, Nx, 3, 3). 144 bytes per link, 4*V*144 bytes in all.
 *   Site matrix fields (Delta, Delta-tilde, g): V*9 complex doubles, index (s*3 + i)*3 + j.
 *   Pointers may be device pointers (CUDA global memory of the context's device) or host pointers
 *     (pageable or pinned); the library detects which and copies host data through its own device
 *     buffers. Device pointers must be 16-byte aligned.
 *   Streams: work is issued on the stream given to lgf_set_stream (default: a stream the context
 *     creates). Every call returns only after its results are complete (it synchronizes that stream).
 *   Errors: every call returns an lgf_status; outputs are written only when the call returns LGF_OK
 *     (or LGF_ENOCONV, see lgf_fix). After a CUDA error the context is poisoned and every later call
 *     returns LGF_ECUDA. lgf_last_error gives a message for the last failing call.
 *   Threads: a context must not be used by two threads at once; distinct contexts are independent.
 *   Ownership: the context owns all its device workspaces; the caller owns every buffer it passes.
 */
#ifndef LGF_H
#define LGF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lgf_ctx lgf_ctx;

typedef enum {
  LGF_OK = 0,
  LGF_EINVAL = 1,     /* bad argument: size, pointer, option or call order                  */
  LGF_ENOMEM = 2,     /* a device or pinned allocation failed                                */
  LGF_ECUDA = 3,      /* a CUDA call or kernel failed; the context is poisoned               */
  LGF_ENOCONV = 4,    /* the iteration limit was reached before theta < eps                  */
  LGF_ENONFINITE = 5  /* theta or F became NaN or infinite (e.g. non-finite input links)     */
} lgf_status;

typedef enum {
  LGF_FP64 = 0,  /* every step at double precision: FP64 links and sums (equivalent forms of some
                    steps are listed at lgf_create)                                              */
  LGF_MIXED = 1, /* float links, FFTs and updates (double reductions) until theta <= theta_switch,
                    then a double-precision handover, float iterations on the residual of the
                    handover links, and the double links rebuilt exactly, to theta < eps        */
  LGF_FP32 = 2   /* float links, FFTs and updates throughout (double reductions)                 */
} lgf_precision;

typedef struct {
  int precision;       /* lgf_precision; default LGF_FP64                                          */
  double theta_switch; /* LGF_MIXED: theta at which the float stage hands over; default 1e-11. The
                          float stage also hands over when a chunk of its iterations does not lower
                          theta (the resolution of float links is reached)                          */
  int reunit_period;   /* float stages: links and accumulated transformation reprojected to SU(3)
                          (in float) every this many iterations; default 16                        */
  int max_iter;        /* iteration limit; default 100000                                          */
  double *history;     /* optional host buffer: history[2k] = theta, history[2k+1] = F after k
                          updates (k = 0 is the input), for k < history_len                         */
  int history_len;
  int fft32_final;     /* LGF_MIXED only, default 0: in the double stage run the Fourier filter in
                          float (Delta, g, the update and the theta/F sums stay double; the filter
                          only sets the search direction, so the fixed point is unchanged)         */
} lgf_options;

/* Fill *opt with the defaults listed above. */
void lgf_default_options(lgf_options *opt);

/* Create a context for an Nx x Ny x Nz x Nt lattice on the current CUDA device. Every extent must be
 * >= 2 and a product of the primes 2, 3 and 5, and at most 1024, and the volume must be below 2^31
 * sites. Device memory is allocated lazily by the first call that needs it. Returns LGF_EINVAL for
 * unsupported extents, LGF_ECUDA if no device.
 * Environment switches read here, each selecting an equivalent form of a step (all pass the same
 * tests): LGF_GENERIC_FFT=1 uses the generic FFT passes for every extent; LGF_FFT_NATIVE_F64=1 runs
 * the Fourier filter of the double path in IEEE double instead of double-float; and LGF_SMALL_STEP=0
 * turns off the small-step forms of the double path, which by default apply per warp where the step
 * is small: g = 1 + a formed in double-float when every |(alpha/2) Delta-tilde| < 2^-8, and rows 0-1
 * of the update as U + [a U + (U + a U) b^+] (a = g(x) - 1, b = g(x+mu) - 1) with the bracket in
 * double-float when every |a|, |b| < 2^-7 (row 2 = conj(row0 x row1) in FP64 in both forms). Their
 * errors are at the level of the FP64 rounding of the plain forms. Three switches concern the float
 * stages and LGF_MIXED: LGF_REUNIT_FP64=1 makes the periodic projection of the float links and of the
 * accumulated transformation onto SU(3) double precision instead of float; LGF_HANDOVER_FP64=1 forms the
 * handover links G U0 G^+(x+mu) in FP64 instead of in 64-bit fixed point with 61 fractional bits (exact
 * to FP64 rounding either way); and LGF_RESIDUAL=0 runs double iterations after the handover instead of
 * the residual stage (float iterations on U = U_h + R, with R the float change since the handover, then
 * the double links rebuilt exactly). With LGF_REUNIT_FP64=1, LGF_RESIDUAL=0 and theta_switch = 1e-8
 * the mixed schedule is: float iterations with double reductions and periodic double reprojection until
 * theta <= 1e-8, the handover, and double iterations to theta < eps. */
lgf_status lgf_create(int Nx, int Ny, int Nz, int Nt, lgf_ctx **out);

/* Release every resource of the context (NULL is accepted). */
void lgf_destroy(lgf_ctx *ctx);

/* Message for the last failing call on this context (a static string if ctx is NULL). */
const char *lgf_last_error(const lgf_ctx *ctx);

/* Issue all later work on `stream` (a cudaStream_t; NULL restores the context's own stream, which is
 * non-blocking; pass cudaStreamLegacy to use the legacy default stream). */
lgf_status lgf_set_stream(lgf_ctx *ctx, void *stream);

/* Algorithm 1 in full: fix the links in place to Landau gauge.
 *   links      in/out, the layout above (device or host pointer)
 *   alpha      step size (the paper uses 0.08, after Davies et al.)
 *   eps        stop when theta < eps (the paper: 1e-15)
 *   opt        NULL for the defaults
 *   theta_out, F_out, iters_out   final theta (Eq. 4), F (Eq. 1 at g = 1) and the number of gauge
 *              updates applied (0 if theta < eps on input); any may be NULL
 * Returns LGF_OK on convergence; LGF_ENOCONV when max_iter updates did not reach theta < eps (the
 * links and outputs then hold the last state); LGF_ENONFINITE if theta or F became non-finite. */
lgf_status lgf_fix(lgf_ctx *ctx, double *links, double alpha, double eps, const lgf_options *opt,
                   double *theta_out, double *F_out, int *iters_out);

/* theta (Eq. 4), F (Eq. 1 at g = 1) and the average plaquette (1/3) Re Tr of the 1x1 loop, averaged
 * over sites and the six planes, of the given links. Any output may be NULL. */
lgf_status lgf_measure(lgf_ctx *ctx, const double *links, double *theta, double *F, double *plaq);

/* ---- Session interface: the loop of Algorithm 1 split into load / iterate / store, so that a
 * caller can run a fixed number of iterations, inspect the state, or time the loop. lgf_fix is
 * lgf_load + lgf_iterate + lgf_store. ---- */

/* Load links into the context's working state at the given precision and compute Delta, theta and F
 * of the input (Algorithm 1, first line). Resets the iteration count. With LGF_MIXED the input is kept
 * in double precision for the handover. */
lgf_status lgf_load(lgf_ctx *ctx, const double *links, int precision);

/* Run at most max_new iterations of the loop of Algorithm 1 on the working state, stopping early when
 * theta < eps (and, with LGF_MIXED, handing over to double precision at theta_switch). theta/F/iters
 * report the state after the call (iters counts all updates since lgf_load). opt supplies
 * theta_switch, reunit_period and history; NULL for the defaults. Returns LGF_OK when theta < eps,
 * LGF_ENOCONV when the limit stopped it first, LGF_ENONFINITE on a non-finite theta or F. */
lgf_status lgf_iterate(lgf_ctx *ctx, int max_new, double alpha, double eps, const lgf_options *opt,
                       double *theta, double *F, int *iters);

/* Write the working state back to links (double precision, the layout above). With LGF_MIXED still in
 * its float stage, the links are rebuilt as G(x) U0_mu(x) G^+(x+mu) in double precision from the
 * saved input U0 and the accumulated transformation G, so they stay gauge-equivalent to the input. */
lgf_status lgf_store(lgf_ctx *ctx, double *links);

/* ---- Single steps of one iteration, on caller buffers in the layouts above (used to check each
 * step against a reference implementation; not needed to fix a gauge). All run in double precision
 * unless `precision` says LGF_FP32. ---- */

/* Eqs. 3-5 and Eq. 1: Delta(x) (V*9 complex, out), theta and F of links. */
lgf_status lgf_delta(lgf_ctx *ctx, const double *links, double *delta, double *theta, double *F,
                     int precision);

/* Algorithm 1, FFT block: Delta-tilde = F^-1[ (p^2_max/p^2) F[Delta] ] / V, zero mode set to 0.
 * delta must be anti-Hermitian and traceless at every site (as Eq. 5 makes it); only its upper
 * triangle and diagonal imaginary parts are read. dtilde (out) is written in full. */
lgf_status lgf_filter(lgf_ctx *ctx, const double *delta, double *dtilde, int precision);

/* Eq. 2 to first order plus projection: g(x) = SU(3)-projection of [1 + (alpha/2) Delta-tilde(x)]
 * (Gram-Schmidt on rows 1-2, row 3 = conj(row1 x row2)). Same input rule as lgf_filter. */
lgf_status lgf_gauge(lgf_ctx *ctx, const double *dtilde, double alpha, double *g, int precision);

/* Algorithm 1: U_mu(x) -> g(x) U_mu(x) g^+(x + mu) for all x, mu (links in/out, g in). */
lgf_status lgf_update(lgf_ctx *ctx, double *links, const double *g, int precision);

/* Algorithm 1, FFT block, on an su(3) coefficient field: out[8*s + a] = F^-1[(p^2_max/p^2) F[c^a]](s) / V
 * for each of the eight real fields c^a(s) = coef[8*s + a] (zero mode set to 0). The filter is real and
 * even in k, so each real field stays real, and filtering the coefficients equals filtering the matrix
 * field sum_a c^a M^a element by element for any constant basis M^a (e.g. i T^a). It preconditions the
 * su(3) gradient of lgf_functional_grad the way Algorithm 1 preconditions Delta. coef and out: V*8
 * doubles, site-major, device (16-byte aligned) or host pointers; they may be the same buffer. */
lgf_status lgf_filter_coeffs(lgf_ctx *ctx, const double *coef, double *out, int precision);

/* ---- The functional as a differentiable function of a Lie-algebra field (Eq. 1 at g = exp(i omega)).
 * omega: V*8 doubles, site-major: omega[8*s + a] is the coefficient of T^a = lambda^a/2 (Gell-Mann
 * matrices), so omega(x) = sum_a omega^a T^a is Hermitian and traceless; g(x) = exp(i omega(x)) is
 * formed from a Jacobi eigen-decomposition of omega(x). Pointers may be device or host pointers. ---- */

/* F = F_U[exp(i omega)] (Eq. 1); g_out (V*9 complex, site-field layout) receives g if not NULL. */
lgf_status lgf_functional(lgf_ctx *ctx, const double *links, const double *omega, double *F, double *g_out);

/* grad[8*s + a] = scale * dF/d omega^a(s): the su(3) gradient, i.e. the steepest-ascent direction
 * (Daleckii-Krein adjoint of the exponential applied to the staple of Eq. 1). At omega = 0 it equals
 * -scale * (i / (24 V)) Tr[T^a Delta(s)] with Delta of Eq. 5. */
lgf_status lgf_functional_grad(lgf_ctx *ctx, const double *links, const double *omega, double scale, double *grad);

/* ---- Timing of the loop's kernels: when enabled, lgf_iterate brackets every kernel launch with CUDA
 * events on the working stream and accumulates per-kernel device time. ---- */
lgf_status lgf_enable_timing(lgf_ctx *ctx, int enable);
/* Copy up to `cap` entries: name[i] (static strings), launches[i], total device milliseconds ms[i];
 * *count gets the number of kernels with timing data. Resets the counters. */
lgf_status lgf_kernel_times(lgf_ctx *ctx, const char **name, long *launches, double *ms, int cap,
                            int *count);

/* ---- Ensembles: several configurations of possibly different lattice shapes fixed together.
 * Configurations of equal shape form a group whose kernels are launched once per group for all its
 * configurations; the iteration loop of all groups is captured in a CUDA graph and replayed until every
 * configuration has stopped (each keeps its own loop control, so iteration counts are per
 * configuration). FFT pass shapes are autotuned per (shape, precision) and cached in the JSON file
 * $LGF_TUNE_CACHE (default $HOME/.cache/lgf_fft_tune.json); LGF_AUTOTUNE=0 disables the tuner. ---- */
typedef struct lgf_batch lgf_batch;

/* dims: n x 4 extents (Nx, Ny, Nz, Nt), each as for lgf_create. */
lgf_status lgf_batch_create(int n, const int *dims, lgf_batch **out);
void lgf_batch_destroy(lgf_batch *b);
const char *lgf_batch_last_error(const lgf_batch *b);

/* Algorithm 1 for every configuration: links[i] (device or host pointer, the links layout above) is
 * fixed in place. opt as for lgf_fix (precision, theta_switch, reunit_period -- also the number of
 * iterations per captured graph replay -- and max_iter; history and fft32_final are ignored). theta, F, iters and status
 * (lgf_status per configuration) are arrays of n entries, any may be NULL. Returns LGF_OK when every
 * configuration reached theta < eps, otherwise the first non-OK status. */
lgf_status lgf_batch_fix(lgf_batch *b, double *const *links, double alpha, double eps, const lgf_options *opt,
                         double *theta, double *F, int *iters, int *status);

/* JSON description of the groups, the tuned FFT plans and the replay counts of the last lgf_batch_fix. */
lgf_status lgf_batch_describe(const lgf_batch *b, char *buf, int len);

/* ---- Measurement without allocation. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory when they need Delta, theta and F -- a framework whose
 * pool owns all device memory and rejects or starves other allocations, a loop that must not stall on
 * cudaMalloc (which may synchronize the device), or an out-of-memory handler that has nothing left to
 * allocate. It needs no context: every input and output is the caller's, and the only scratch (per-block
 * partial sums of the reduction and a counter, 1 MiB) is a fixed array inside the library's device
 * image. The call allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   links     device pointer of the current device, the links layout above, 16-byte aligned
 *   delta     device pointer of the current device to V*9 complex doubles (site-field layout), 16-byte
 *             aligned, that receives the gauge-fixing violation Delta(x) of every site; or NULL
 *   theta_F   device pointer of the current device to 2 doubles, 8-byte aligned: the gauge-fixing
 *             residual theta (the lattice average of Tr Delta Delta^+ / 3) and the functional F (the
 *             average of Re Tr U_mu(x) / 3 over sites and directions, i.e. at g = 1)
 *   stream    cudaStream_t to issue on (NULL = the legacy default stream); the call does not wait:
 *             the outputs are complete when the stream reaches that point
 * Limits: V = Nx*Ny*Nz*Nt <= 16777216 (2^24, e.g. 64^4); extents as for lgf_create. Larger lattices,
 * host pointers, pointers of another GPU, misaligned pointers or bad extents return LGF_EINVAL with a
 * message from lgf_last_error(NULL).
 * The first call on a device looks up the device address of the scratch array (once per device, with
 * that device current); make that first call before any stream capture. Under CUDA's lazy module
 * loading, that first call (or the first launch) is also when the device commits memory for the 1 MiB
 * array, so it can fail with LGF_ECUDA if the device is full at that moment: make the first call, as a
 * warm-up, while device memory is still available. All calls on a device share the scratch array, which
 * keeps the last call's contents (the counter is cleared by each call): calls that overlap on the GPU
 * race and give wrong results, so order them on one stream. */
lgf_status lgf_delta_noalloc(const double *links, int Nx, int Ny, int Nz, int Nt, double *delta, double *theta_F,
                             void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LGF_H */
