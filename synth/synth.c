/*
 * synth.c -- seeded synthetic SU(3) gauge configurations for tests and benchmarks.
 *
 * A configuration is  U_mu(x) = h(x) exp(i eps A_mu(x)) h^dagger(x + mu),
 *   A_mu(x) = sum_a A^a_mu(x) lambda^a / (2 sqrt 2),  A^a ~ N(0,1)  (lambda^a: Gell-Mann matrices),
 *   h(x) Haar-random on SU(3)  (or near the identity, or the identity, see h_mode).
 * eps = 0 gives a pure-gauge field whose Landau-gauge functional maximum is F = 1 (at g = h^dagger).
 *
 * This module only draws inputs. It holds nothing of the gauge-fixing method itself: no Delta, no
 * Fourier transform, no filter, no update. Both the CPU oracle and the GPU library consume the bytes
 * it writes; neither calls into it.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC11), a counter-based generator, so every link and site draws from its own counter and
 * the output does not depend on the number of threads. Normals by the Box-Muller transform.
 *
 * Layout of the output: complex doubles (re, im interleaved), [mu][t][z][y][x][3][3].
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef double complex cplx;

/* ---------------- Philox4x32-10 ---------------- */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
  const uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void synth_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c[0], &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c[2], &hi1, &lo1);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
  }
  memcpy(out, c, sizeof c);
}

/* A stream of standard normals for one (seed, site, slot) triple. */
typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  double buf[4];
  int avail;
} normal_stream;

static void ns_init(normal_stream *ns, uint64_t seed, uint64_t site, uint32_t slot) {
  ns->key[0] = (uint32_t)seed;
  ns->key[1] = (uint32_t)(seed >> 32);
  ns->ctr[0] = 0; /* draw counter */
  ns->ctr[1] = slot;
  ns->ctr[2] = (uint32_t)site;
  ns->ctr[3] = (uint32_t)(site >> 32);
  ns->avail = 0;
}

static double ns_next(normal_stream *ns) {
  if (ns->avail == 0) {
    uint32_t r[4];
    synth_philox4x32_10(ns->ctr, ns->key, r);
    ns->ctr[0]++;
    for (int p = 0; p < 2; ++p) {
      /* uniforms in (0, 1) */
      const double u1 = ((double)r[2 * p] + 0.5) * (1.0 / 4294967296.0);
      const double u2 = ((double)r[2 * p + 1] + 0.5) * (1.0 / 4294967296.0);
      const double rad = sqrt(-2.0 * log(u1));
      ns->buf[2 * p] = rad * cos(2.0 * M_PI * u2);
      ns->buf[2 * p + 1] = rad * sin(2.0 * M_PI * u2);
    }
    ns->avail = 4;
  }
  return ns->buf[--ns->avail];
}

/* ---------------- small SU(3) helpers ---------------- */
static void mm(const cplx *a, const cplx *b, cplx *c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += a[3 * i + k] * b[3 * k + j];
      c[3 * i + j] = acc;
    }
}

/* Haar measure on SU(3): two rows of i.i.d. complex Gaussians, orthonormalised (the QR of a complex
 * Ginibre matrix is Haar on U(3)); the third row conj(r0 x r1) fixes the determinant to 1, which
 * pushes Haar(U(3)) forward to Haar(SU(3)). */
static void haar_su3(normal_stream *ns, cplx *h) {
  cplx r[6];
  for (int e = 0; e < 6; ++e) {
    const double re = ns_next(ns), im = ns_next(ns);
    r[e] = re + I * im;
  }
  double n0 = 0;
  for (int j = 0; j < 3; ++j) n0 += creal(r[j]) * creal(r[j]) + cimag(r[j]) * cimag(r[j]);
  n0 = sqrt(n0);
  for (int j = 0; j < 3; ++j) r[j] /= n0;
  cplx ip = 0;
  for (int j = 0; j < 3; ++j) ip += conj(r[j]) * r[3 + j];
  for (int j = 0; j < 3; ++j) r[3 + j] -= ip * r[j];
  double n1 = 0;
  for (int j = 0; j < 3; ++j) n1 += creal(r[3 + j]) * creal(r[3 + j]) + cimag(r[3 + j]) * cimag(r[3 + j]);
  n1 = sqrt(n1);
  for (int j = 0; j < 3; ++j) r[3 + j] /= n1;
  for (int e = 0; e < 6; ++e) h[e] = r[e];
  h[6] = conj(r[1] * r[5] - r[2] * r[4]);
  h[7] = conj(r[2] * r[3] - r[0] * r[5]);
  h[8] = conj(r[0] * r[4] - r[1] * r[3]);
}

/* H = sum_a c^a lambda^a (Hermitian, traceless), from the 8 Gell-Mann matrices. */
static void gell_mann_combination(const double c[8], cplx *H) {
  const double s3 = 1.0 / sqrt(3.0);
  H[0] = c[2] + s3 * c[7];
  H[4] = -c[2] + s3 * c[7];
  H[8] = -2.0 * s3 * c[7];
  H[1] = c[0] - I * c[1];
  H[3] = c[0] + I * c[1];
  H[2] = c[3] - I * c[4];
  H[6] = c[3] + I * c[4];
  H[5] = c[5] - I * c[6];
  H[7] = c[5] + I * c[6];
}

/* exp(i H) for Hermitian H by scaling and squaring of a degree-16 Taylor polynomial. */
static void exp_i_hermitian(const cplx *H, cplx *E) {
  double nrm = 0;
  for (int e = 0; e < 9; ++e) nrm += creal(H[e] * conj(H[e]));
  nrm = sqrt(nrm);
  int sq = 0;
  while (nrm > 0.125) {
    nrm *= 0.5;
    ++sq;
  }
  const double scale = ldexp(1.0, -sq);
  cplx X[9];
  for (int e = 0; e < 9; ++e) X[e] = I * H[e] * scale;
  /* Horner: E = 1 + X (1 + X/2 (1 + X/3 (... ))) */
  cplx P[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, T[9];
  for (int k = 16; k >= 1; --k) {
    mm(X, P, T);
    for (int e = 0; e < 9; ++e) P[e] = T[e] / (double)k;
    P[0] += 1;
    P[4] += 1;
    P[8] += 1;
  }
  for (int s = 0; s < sq; ++s) {
    mm(P, P, T);
    memcpy(P, T, sizeof T);
  }
  memcpy(E, P, sizeof P);
}

static long vol(const int n[4]) { return (long)n[0] * n[1] * n[2] * n[3]; }

static long fwd(const int n[4], long s, int mu) {
  int c[4];
  long r = s;
  for (int m = 0; m < 4; ++m) {
    c[m] = (int)(r % n[m]);
    r /= n[m];
  }
  c[mu] = (c[mu] + 1) % n[mu];
  return c[0] + (long)n[0] * (c[1] + (long)n[1] * (c[2] + (long)n[2] * c[3]));
}

enum { H_HAAR = 0, H_NEAR_IDENTITY = 1, H_IDENTITY = 2 };

/* The gauge rotation h(x) at site s. */
static void gauge_rotation(uint64_t seed, long s, int h_mode, double h_scale, cplx *h) {
  normal_stream ns;
  ns_init(&ns, seed, (uint64_t)s, 4u /* slot 4: h */);
  if (h_mode == H_HAAR) {
    haar_su3(&ns, h);
  } else if (h_mode == H_NEAR_IDENTITY) {
    double c[8];
    for (int a = 0; a < 8; ++a) c[a] = h_scale * ns_next(&ns) / (2.0 * sqrt(2.0));
    cplx H[9];
    gell_mann_combination(c, H);
    exp_i_hermitian(H, h);
  } else {
    for (int e = 0; e < 9; ++e) h[e] = (e % 4 == 0) ? 1 : 0;
  }
}

/*
 * Fill U (4*V*9 complex doubles) with the configuration above.
 *   seed       key of the generator
 *   eps        strength of the non-pure-gauge part (0: pure gauge)
 *   h_mode     0: Haar h(x); 1: h(x) = exp(i h_scale sum_a c^a lambda^a/(2 sqrt 2)), c^a ~ N(0,1); 2: h = 1
 *   algebra_norm  the factor multiplying lambda^a in A (1/(2 sqrt 2) for the default ensembles)
 */
void synth_config(const int n[4], uint64_t seed, double eps, int h_mode, double h_scale, double algebra_norm,
                  double *U_) {
  cplx *U = (cplx *)U_;
  const long V = vol(n);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    cplx hx[9];
    gauge_rotation(seed, s, h_mode, h_scale, hx);
    for (int mu = 0; mu < 4; ++mu) {
      cplx hy[9];
      gauge_rotation(seed, fwd(n, s, mu), h_mode, h_scale, hy);
      normal_stream ns;
      ns_init(&ns, seed, (uint64_t)s, (uint32_t)mu /* slots 0..3: A_mu */);
      double c[8];
      for (int a = 0; a < 8; ++a) c[a] = eps * algebra_norm * ns_next(&ns);
      cplx H[9], E[9], T[9];
      gell_mann_combination(c, H);
      exp_i_hermitian(H, E);
      mm(hx, E, T); /* h(x) exp(i eps A) */
      cplx *u = U + ((long)mu * V + s) * 9;
      for (int i = 0; i < 3; ++i) /* ... h^dagger(x + mu) */
        for (int j = 0; j < 3; ++j) {
          cplx acc = 0;
          for (int k = 0; k < 3; ++k) acc += T[3 * i + k] * conj(hy[3 * j + k]);
          u[3 * i + j] = acc;
        }
    }
  }
}

/* A global (x-independent) gauge rotation h applied to every link: U -> h U h^dagger. */
void synth_global_rotation(const int n[4], uint64_t seed, double *U_) {
  cplx *U = (cplx *)U_;
  const long V = vol(n);
  cplx h[9];
  normal_stream ns;
  ns_init(&ns, seed, 0xFFFFFFFFFFull, 7u);
  haar_su3(&ns, h);
#pragma omp parallel for schedule(static)
  for (long l = 0; l < 4 * V; ++l) {
    cplx *u = U + l * 9, T[9];
    mm(h, u, T);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        cplx acc = 0;
        for (int k = 0; k < 3; ++k) acc += T[3 * i + k] * conj(h[3 * j + k]);
        u[3 * i + j] = acc;
      }
  }
}

/* Standard normals for an arbitrary (seed, stream) pair: the Lie-algebra field omega of the
 * differentiable functional is drawn from here. out[i] for i in [0, count). */
void synth_normals(uint64_t seed, uint32_t stream, long count, double scale, double *out) {
  const long nblk = (count + 7) / 8;
#pragma omp parallel for schedule(static)
  for (long b = 0; b < nblk; ++b) {
    normal_stream ns;
    ns_init(&ns, seed, (uint64_t)b, 16u + stream);
    for (long i = b * 8; i < (b + 1) * 8 && i < count; ++i) out[i] = scale * ns_next(&ns);
  }
}
