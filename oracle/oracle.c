/*
 * oracle.c -- plain FP64 CPU oracle for Fourier-accelerated steepest-descent Landau gauge fixing
 * of SU(3) lattice gauge fields (Cardoso, Silva, Oliveira, Bicudo, "GPU implementation of a Landau
 * gauge fixing algorithm", Lattice 2012; Eqs. 1-5 and Algorithm 1).
 *
 * TEST INFRASTRUCTURE. This file is the checker, not the product. Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it. It shares no code, header, table or helper
 * with the CUDA path, and the CUDA path never calls it.
 *
 * It is written to be read against the paper, not to be fast: every step is the textbook definition,
 * in the order Algorithm 1 states it, in double precision. OpenMP only distributes independent sites
 * or FFT pencils over threads; every global sum is taken over fixed chunks in a fixed order, so the
 * results do not depend on the thread count.
 *
 * Conventions
 *   dims n[4] = {Nx, Ny, Nz, Nt}, V = Nx*Ny*Nz*Nt, site s = x + Nx*(y + Ny*(z + Nz*t)), periodic.
 *   direction mu in {0,1,2,3} = {x,y,z,t}.
 *   links U: complex doubles (re,im interleaved), index ((mu*V + s)*3 + i)*3 + j  (row i, column j),
 *            i.e. the array [mu][t][z][y][x][3][3].
 *   site fields (Delta, g): ((s*3 + i)*3 + j).
 *   N_c = 3.
 *
 * Readings of the paper used here (the paper leaves these open):
 *   p^2(k) = sum_mu 4 sin^2(pi k_mu / N_mu), the eigenvalues of the lattice -d^2 with a = 1.
 *   p^2_max = sum_mu 4 sin^2(pi floor(N_mu/2) / N_mu), the largest of them.
 *   the k = 0 mode, where p^2_max/p^2 diverges, is multiplied by 0 (sum_x Delta(x) = 0 exactly).
 *   "normalize" = divide by V once after the backward transform.
 *   reunitarization = Gram-Schmidt on rows 1 and 2, row 3 = conj(row1 x row2).
 *   the iteration count is the number of gauge updates applied; the loop runs while theta >= eps.
 *
 * parity pins: see tests/test_oracle_*.py. All functions below are pinned (none is "parity unpinned").
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define NC 3
#define CHUNK 4096 /* fixed summation chunk: results independent of the thread count */

static long volume(const int n[4]) { return (long)n[0] * n[1] * n[2] * n[3]; }

static void coords(const int n[4], long s, int c[4]) {
  for (int mu = 0; mu < 4; ++mu) {
    c[mu] = (int)(s % n[mu]);
    s /= n[mu];
  }
}

static long index_of(const int n[4], const int c[4]) {
  return c[0] + (long)n[0] * (c[1] + (long)n[1] * (c[2] + (long)n[2] * c[3]));
}

/* s + step * mu-hat on the periodic lattice (step = +1 or -1) */
static long shift(const int n[4], long s, int mu, int step) {
  int c[4];
  coords(n, s, c);
  c[mu] = (c[mu] + step + n[mu]) % n[mu];
  return index_of(n, c);
}

static const cplx *link_c(const cplx *U, long V, int mu, long s) { return U + ((long)mu * V + s) * 9; }
static cplx *link(cplx *U, long V, int mu, long s) { return U + ((long)mu * V + s) * 9; }

/* ---- 3x3 complex matrix helpers (row-major) ---- */
static void mat_mul(const cplx *a, const cplx *b, cplx *c) { /* c = a b */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += a[3 * i + k] * b[3 * k + j];
      c[3 * i + j] = acc;
    }
}
static void mat_mul_adj(const cplx *a, const cplx *b, cplx *c) { /* c = a b^dagger */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += a[3 * i + k] * conj(b[3 * j + k]);
      c[3 * i + j] = acc;
    }
}

/* Fixed-order sum of per-chunk partial sums (chunks of CHUNK consecutive items). */
static double ordered_sum(const double *partial, long nchunks) {
  double acc = 0.0;
  for (long c = 0; c < nchunks; ++c) acc += partial[c];
  return acc;
}

/* =========================================================================================== */
/* Eq. 3 and Eq. 5: Delta(x) = sum_nu [ U_nu(x - nu) - U_nu(x) - h.c. - trace ].              */
/* The anti-Hermitian part of the sum is taken first and the trace/3 removed once (linear).    */
/* =========================================================================================== */
void orc_delta(const int n[4], const double *U_, double *Delta_) {
  const cplx *U = (const cplx *)U_;
  cplx *Delta = (cplx *)Delta_;
  const long V = volume(n);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    cplx M[9] = {0};
    for (int nu = 0; nu < 4; ++nu) {
      const long sb = shift(n, s, nu, -1);
      const cplx *back = link_c(U, V, nu, sb); /* U_nu(x - nu) */
      const cplx *here = link_c(U, V, nu, s);  /* U_nu(x)      */
      cplx A[9];
      for (int e = 0; e < 9; ++e) A[e] = back[e] - here[e]; /* Delta_{-nu} U_nu(x), Eq. 3 */
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] += A[3 * i + j] - conj(A[3 * j + i]); /* minus h.c. */
    }
    const cplx tr = (M[0] + M[4] + M[8]) / 3.0;
    cplx *D = Delta + s * 9;
    for (int e = 0; e < 9; ++e) D[e] = M[e];
    D[0] -= tr;
    D[4] -= tr;
    D[8] -= tr; /* minus trace */
  }
}

/* Eq. 4: theta = 1/(N_c V) sum_x Tr[Delta(x) Delta^dagger(x)]. */
double orc_theta(const int n[4], const double *Delta_) {
  const cplx *Delta = (const cplx *)Delta_;
  const long V = volume(n);
  const long nchunks = (V + CHUNK - 1) / CHUNK;
  double *partial = (double *)malloc(sizeof(double) * nchunks);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nchunks; ++c) {
    double acc = 0.0;
    const long end = (c + 1) * CHUNK < V ? (c + 1) * CHUNK : V;
    for (long s = c * CHUNK; s < end; ++s) {
      const cplx *D = Delta + s * 9;
      /* Tr[D D^dagger] = sum_ij D_ij conj(D_ij) */
      for (int e = 0; e < 9; ++e) acc += creal(D[e] * conj(D[e]));
    }
    partial[c] = acc;
  }
  const double theta = ordered_sum(partial, nchunks) / (NC * (double)V);
  free(partial);
  return theta;
}

/* Eq. 1: F_U[g] = 1/(4 N_c V) sum_x sum_mu Re Tr[g(x) U_mu(x) g^dagger(x + mu)].
 * With g == NULL the identity transformation is used (Algorithm 1 reports F on the current links). */
double orc_functional(const int n[4], const double *U_, const double *g_) {
  const cplx *U = (const cplx *)U_;
  const cplx *g = (const cplx *)g_;
  const long V = volume(n);
  const long nchunks = (V + CHUNK - 1) / CHUNK;
  double *partial = (double *)malloc(sizeof(double) * nchunks);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nchunks; ++c) {
    double acc = 0.0;
    const long end = (c + 1) * CHUNK < V ? (c + 1) * CHUNK : V;
    for (long s = c * CHUNK; s < end; ++s)
      for (int mu = 0; mu < 4; ++mu) {
        const cplx *u = link_c(U, V, mu, s);
        if (g) {
          cplx t[9], w[9];
          mat_mul(g + s * 9, u, t);                        /* g(x) U_mu(x)            */
          mat_mul_adj(t, g + shift(n, s, mu, +1) * 9, w); /* ... g^dagger(x + mu)    */
          acc += creal(w[0] + w[4] + w[8]);
        } else {
          acc += creal(u[0] + u[4] + u[8]);
        }
      }
    partial[c] = acc;
  }
  const double F = ordered_sum(partial, nchunks) / (4.0 * NC * (double)V);
  free(partial);
  return F;
}

/* =========================================================================================== */
/* The FFT (F-hat of Eq. 2): a recursive mixed-radix Cooley-Tukey transform, decimation in     */
/* time on the smallest prime factor, with twiddles taken directly from cos/sin.               */
/*   out[k] = sum_j in[j] exp(sign * 2 pi i j k / N)                                           */
/* =========================================================================================== */
static int smallest_factor(int N) {
  for (int p = 2; p * p <= N; ++p)
    if (N % p == 0) return p;
  return N;
}

static cplx root_of_unity(long num, long N, int sign) {
  /* exp(sign * 2 pi i num / N), with num reduced mod N first */
  const long r = ((num % N) + N) % N;
  const double ang = 2.0 * M_PI * (double)r / (double)N;
  return cos(ang) + (double)sign * I * sin(ang);
}

/* in: N values at stride istride; out: N contiguous values; work: N scratch values */
static void dft_recursive(int N, const cplx *in, long istride, cplx *out, cplx *work, int sign) {
  if (N == 1) {
    out[0] = in[0];
    return;
  }
  const int p = smallest_factor(N);
  const int m = N / p;
  /* sub-transforms of the p decimated sequences in[j1 + p*j2], written to work[j1*m + k2] */
  for (int j1 = 0; j1 < p; ++j1) dft_recursive(m, in + j1 * istride, istride * p, work + j1 * m, out, sign);
  /* combine: X[k2 + m*k1] = sum_j1 exp(sign 2 pi i j1 (k2 + m k1) / N) * sub_j1[k2] */
  for (int k1 = 0; k1 < p; ++k1)
    for (int k2 = 0; k2 < m; ++k2) {
      const int k = k2 + m * k1;
      cplx acc = 0;
      for (int j1 = 0; j1 < p; ++j1) acc += root_of_unity((long)j1 * k, N, sign) * work[j1 * m + k2];
      out[k] = acc;
    }
}

/* In-place 1D transform of N values at stride `stride`. */
void orc_fft1d(int N, double *data_, long stride, int sign) {
  cplx *data = (cplx *)data_;
  cplx *tmp = (cplx *)malloc(sizeof(cplx) * 3 * N);
  cplx *in = tmp, *out = tmp + N, *work = tmp + 2 * N;
  for (int j = 0; j < N; ++j) in[j] = data[j * stride];
  dft_recursive(N, in, 1, out, work, sign);
  for (int k = 0; k < N; ++k) data[k * stride] = out[k];
  free(tmp);
}

/* 4D transform of one complex field f[s] as four successive 1D transforms (one per axis). */
void orc_fft4d(const int n[4], double *f_, int sign) {
  cplx *f = (cplx *)f_;
  const long V = volume(n);
  long stride = 1;
  for (int mu = 0; mu < 4; ++mu) {
    const int N = n[mu];
    const long npencils = V / N;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < npencils; ++p) {
      /* pencil p: all indices except the mu-th; lower part below `stride`, upper part above */
      const long lo = p % stride, hi = p / stride;
      const long base = lo + hi * stride * N;
      orc_fft1d(N, (double *)(f + base), stride, sign);
    }
    stride *= N;
  }
}

/* p^2(k) = sum_mu 4 sin^2(pi k_mu / N_mu): eigenvalues of the lattice -d^2 (a = 1). */
double orc_p2(const int n[4], const int k[4]) {
  double p2 = 0.0;
  for (int mu = 0; mu < 4; ++mu) {
    const double sn = sin(M_PI * (double)k[mu] / (double)n[mu]);
    p2 += 4.0 * sn * sn;
  }
  return p2;
}

double orc_p2max(const int n[4]) {
  int kmax[4];
  for (int mu = 0; mu < 4; ++mu) kmax[mu] = n[mu] / 2;
  return orc_p2(n, kmax);
}

/* =========================================================================================== */
/* Algorithm 1, "for all elements of Delta(x)": FFT forward, apply p^2_max/p^2, FFT backward,  */
/* normalize (1/V). Each of the 9 matrix elements is transformed as a separate scalar field.   */
/* =========================================================================================== */
void orc_fourier_filter(const int n[4], const double *Delta_, double *Dt_) {
  const cplx *Delta = (const cplx *)Delta_;
  cplx *Dt = (cplx *)Dt_;
  const long V = volume(n);
  const double p2max = orc_p2max(n);
  cplx *field = (cplx *)malloc(sizeof(cplx) * V);
  for (int e = 0; e < 9; ++e) {
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; ++s) field[s] = Delta[s * 9 + e];
    orc_fft4d(n, (double *)field, -1); /* apply FFT forward */
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; ++s) { /* apply p^2_max / p^2 (mode k stored at index k) */
      int k[4];
      coords(n, s, k);
      const double p2 = orc_p2(n, k);
      field[s] *= (p2 == 0.0) ? 0.0 : p2max / p2;
    }
    orc_fft4d(n, (double *)field, +1); /* apply FFT backward */
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; ++s) Dt[s * 9 + e] = field[s] / (double)V; /* normalize */
  }
  free(field);
}

/* Projection to SU(3) (paper: reunitarization): Gram-Schmidt on rows 1 and 2, then
 * row 3 = conj(row1 x row2), which makes det = +1. */
void orc_reunitarize(double *m_) {
  cplx *m = (cplx *)m_;
  cplx *r0 = m, *r1 = m + 3, *r2 = m + 6;
  double nrm = 0.0;
  for (int j = 0; j < 3; ++j) nrm += creal(r0[j] * conj(r0[j]));
  nrm = 1.0 / sqrt(nrm);
  for (int j = 0; j < 3; ++j) r0[j] *= nrm;
  cplx proj = 0; /* <r0, r1> = sum_j conj(r0_j) r1_j */
  for (int j = 0; j < 3; ++j) proj += conj(r0[j]) * r1[j];
  for (int j = 0; j < 3; ++j) r1[j] -= proj * r0[j];
  nrm = 0.0;
  for (int j = 0; j < 3; ++j) nrm += creal(r1[j] * conj(r1[j]));
  nrm = 1.0 / sqrt(nrm);
  for (int j = 0; j < 3; ++j) r1[j] *= nrm;
  r2[0] = conj(r0[1] * r1[2] - r0[2] * r1[1]);
  r2[1] = conj(r0[2] * r1[0] - r0[0] * r1[2]);
  r2[2] = conj(r0[0] * r1[1] - r0[1] * r1[0]);
}

/* Eq. 2 with the exponential expanded to first order in alpha, then reunitarized:
 * g(x) = SU(3)-projection of [ 1 + (alpha/2) Delta-tilde(x) ]. */
void orc_gauge_field(const int n[4], const double *Dt_, double alpha, double *g_) {
  const cplx *Dt = (const cplx *)Dt_;
  cplx *g = (cplx *)g_;
  const long V = volume(n);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    cplx *m = g + s * 9;
    for (int e = 0; e < 9; ++e) m[e] = 0.5 * alpha * Dt[s * 9 + e];
    m[0] += 1.0;
    m[4] += 1.0;
    m[8] += 1.0;
    orc_reunitarize((double *)m);
  }
}

/* Algorithm 1: U_mu(x) -> g(x) U_mu(x) g^dagger(x + mu) for all x and mu, with g fixed for the
 * whole sweep (each new link depends only on its own old value). */
void orc_gauge_transform(const int n[4], double *U_, const double *g_) {
  cplx *U = (cplx *)U_;
  const cplx *g = (const cplx *)g_;
  const long V = volume(n);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s)
    for (int mu = 0; mu < 4; ++mu) {
      cplx *u = link(U, V, mu, s);
      cplx t[9];
      mat_mul(g + s * 9, u, t);
      mat_mul_adj(t, g + shift(n, s, mu, +1) * 9, u);
    }
}

/* =========================================================================================== */
/* Algorithm 1, the whole loop.                                                                 */
/*   history (optional, length hist_len): hist[2*k] = theta, hist[2*k+1] = F after k updates.   */
/*   returns the number of updates applied; theta_out/F_out get the final values.               */
/* =========================================================================================== */
int orc_fix(const int n[4], double *U, double alpha, double eps, int max_iter, double *hist, int hist_len,
            double *theta_out, double *F_out) {
  const long V = volume(n);
  double *Delta = (double *)malloc(sizeof(cplx) * 9 * V);
  double *Dt = (double *)malloc(sizeof(cplx) * 9 * V);
  double *g = (double *)malloc(sizeof(cplx) * 9 * V);
  /* calculate Delta(x), F_g[U] and theta */
  orc_delta(n, U, Delta);
  double theta = orc_theta(n, Delta);
  double F = orc_functional(n, U, NULL);
  int iters = 0;
  if (hist && hist_len > 0) {
    hist[0] = theta;
    hist[1] = F;
  }
  while (theta >= eps && iters < max_iter) {
    orc_fourier_filter(n, Delta, Dt);    /* FFT forward, p^2_max/p^2, FFT backward, normalize */
    orc_gauge_field(n, Dt, alpha, g);    /* obtain g(x) and reunitarize                       */
    orc_gauge_transform(n, U, g);        /* U_mu(x) -> g(x) U_mu(x) g^dagger(x + mu)          */
    orc_delta(n, U, Delta);              /* calculate Delta(x), F_g[U] and theta              */
    theta = orc_theta(n, Delta);
    F = orc_functional(n, U, NULL);
    ++iters;
    if (hist && iters < hist_len) {
      hist[2 * iters] = theta;
      hist[2 * iters + 1] = F;
    }
  }
  free(Delta);
  free(Dt);
  free(g);
  if (theta_out) *theta_out = theta;
  if (F_out) *F_out = F;
  return iters;
}

/* =========================================================================================== */
/* Gauge-invariant observables, used to check that the fixing leaves the physics unchanged.    */
/* =========================================================================================== */

/* Average planar R x T Wilson loop: (1/3) Re Tr of the ordered product around the rectangle,
 * averaged over all sites and the 12 ordered planes (mu != nu). R = T = 1 is the plaquette. */
double orc_wilson_loop(const int n[4], const double *U_, int R, int T) {
  const cplx *U = (const cplx *)U_;
  const long V = volume(n);
  const long nchunks = (V + CHUNK - 1) / CHUNK;
  double *partial = (double *)malloc(sizeof(double) * nchunks);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nchunks; ++c) {
    double acc = 0.0;
    const long end = (c + 1) * CHUNK < V ? (c + 1) * CHUNK : V;
    for (long s0 = c * CHUNK; s0 < end; ++s0)
      for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu) {
          if (mu == nu) continue;
          cplx P[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, t[9];
          long s = s0;
          for (int r = 0; r < R; ++r) { /* R steps along +mu */
            mat_mul(P, link_c(U, V, mu, s), t);
            memcpy(P, t, sizeof t);
            s = shift(n, s, mu, +1);
          }
          for (int q = 0; q < T; ++q) { /* T steps along +nu */
            mat_mul(P, link_c(U, V, nu, s), t);
            memcpy(P, t, sizeof t);
            s = shift(n, s, nu, +1);
          }
          for (int r = 0; r < R; ++r) { /* R steps along -mu: U_mu(x - mu)^dagger */
            s = shift(n, s, mu, -1);
            mat_mul_adj(P, link_c(U, V, mu, s), t);
            memcpy(P, t, sizeof t);
          }
          for (int q = 0; q < T; ++q) { /* T steps along -nu */
            s = shift(n, s, nu, -1);
            mat_mul_adj(P, link_c(U, V, nu, s), t);
            memcpy(P, t, sizeof t);
          }
          acc += creal(P[0] + P[4] + P[8]) / 3.0;
        }
    partial[c] = acc;
  }
  const double w = ordered_sum(partial, nchunks) / (12.0 * (double)V);
  free(partial);
  return w;
}

/* Largest deviation from SU(3) over all links: max of ||U U^dagger - 1||_max and |det U - 1|. */
double orc_unitarity_violation(const int n[4], const double *U_, long nlinks) {
  const cplx *U = (const cplx *)U_;
  (void)n;
  double worst = 0.0;
#pragma omp parallel for schedule(static) reduction(max : worst)
  for (long l = 0; l < nlinks; ++l) {
    const cplx *u = U + l * 9;
    cplx p[9];
    mat_mul_adj(u, u, p);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const double d = cabs(p[3 * i + j] - (i == j ? 1.0 : 0.0));
        if (d > worst) worst = d;
      }
    const cplx det = u[0] * (u[4] * u[8] - u[5] * u[7]) - u[1] * (u[3] * u[8] - u[5] * u[6]) +
                     u[2] * (u[3] * u[7] - u[4] * u[6]);
    const double dd = cabs(det - 1.0);
    if (dd > worst) worst = dd;
  }
  return worst;
}
