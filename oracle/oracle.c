/*
 * oracle.c -- plain, slow CPU reference for the 1-D complex DFT (Eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference legs, never by the product library.
 * Written from the paper's definitions (Eq. 1; the radix-2 split of
 * Eqs. 4-6 in Sec. 2.2) and the published SplitMix64 generator.  It is
 * deliberately unblocked and unfused so that it can be checked by eye.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (oracle/build.py).
 * -ffp-contract=off keeps every product and sum separately rounded, which the
 * compensated summations below rely on.
 *
 * ORACLE_MUTANT=k (compile-time, default 0) plants one known mistake so that
 * tests/test_oracle_mutants.py can prove the pins catch it.  The shipped
 * build always has ORACLE_MUTANT=0.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

int oracle_version(void) { return 1; }
int oracle_mutant(void) { return ORACLE_MUTANT; }

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

static int ilog2_i64(int64_t n) {
  int e = 0;
  while (((int64_t)1 << e) < n) e++;
  return e;
}

/* ------------------------------------------------------------------------ */
/* Twiddle factors: exp(sign*2*pi*i*m/N) by exact octant reduction.          */
/*                                                                            */
/* angle = 2*pi*m/N = (pi/4) * (8m/N).  With a = 8m = o*N + r (0 <= r < N),  */
/* octant o in 0..7: for even o the angle is (o/2)*(pi/2) + phi with          */
/* phi = (pi/4)*r/N; for odd o it is ((o+1)/2)*(pi/2) - phi' with             */
/* phi' = (pi/4)*(N-r)/N.  Both phi, phi' lie in [0, pi/4].  Quadrant q turns */
/* (cos psi, sin psi) by q quarter turns.                                     */
/* ------------------------------------------------------------------------ */

static void quarter_turn(int q, long double c, long double s, long double* oc,
                         long double* os) {
  switch (q & 3) {
    case 0: *oc = c; *os = s; break;
    case 1: *oc = -s; *os = c; break;
    case 2: *oc = -c; *os = -s; break;
    default:
#if ORACLE_MUTANT == 14
      *oc = -s; *os = -c; break; /* MUTANT: wrong fourth quadrant */
#else
      *oc = s; *os = -c; break;
#endif
  }
}

void oracle_twiddle(int64_t m, int64_t N, int sign, double* re, double* im) {
  /* pi/4 to 64+ bits; long double holds it to its own precision. */
  static const long double PI_4 = 0.785398163397448309615660845819875721L;
  m %= N;
  if (m < 0) m += N;
  /* 8m < 8N: N is at most 2^40 here, so no overflow. */
  int64_t a = 8 * m;
  int64_t o = a / N;
  int64_t r = a - o * N;
  long double psi;
  int q;
  if ((o & 1) == 0) {
    q = (int)(o / 2);
    psi = PI_4 * ((long double)r / (long double)N);
  } else {
    q = (int)((o + 1) / 2);
    psi = -PI_4 * ((long double)(N - r) / (long double)N);
  }
  long double c = cosl(psi), s = sinl(psi), oc, os;
#if ORACLE_MUTANT == 4
  { long double t = c; c = s; s = t; } /* MUTANT: re/im of the twiddle swapped */
#endif
  quarter_turn(q, c, s, &oc, &os);
#if ORACLE_MUTANT == 1
  sign = -sign; /* MUTANT: twiddle sign flipped */
#endif
  *re = (double)oc;
  *im = (double)(sign < 0 ? -os : os);
}

/* Same reduction in double precision, for the large tables of the radix-2
 * FFT and the sampled mode (N/2 long-double sin/cos would be too slow on
 * hosts whose long double is software quad precision). */
static void twiddle_d(int64_t m, int64_t N, int sign, double* re, double* im) {
  static const double PI_4 = 0.78539816339744830961566084581987572;
  m %= N;
  if (m < 0) m += N;
  int64_t a = 8 * m;
  int64_t o = a / N;
  int64_t r = a - o * N;
  double psi;
  int q;
  if ((o & 1) == 0) {
    q = (int)(o / 2);
    psi = PI_4 * ((double)r / (double)N);
  } else {
    q = (int)((o + 1) / 2);
    psi = -PI_4 * ((double)(N - r) / (double)N);
  }
  double c = cos(psi), s = sin(psi), oc, os;
#if ORACLE_MUTANT == 13
  if (o == 3) { double t = c; c = s; s = t; } /* MUTANT: one octant mis-reduced */
#endif
  switch (q & 3) {
    case 0: oc = c; os = s; break;
    case 1: oc = -s; os = c; break;
    case 2: oc = -c; os = -s; break;
    default: oc = s; os = -c; break;
  }
  *re = oc;
  *im = sign < 0 ? -os : os;
}

/* ------------------------------------------------------------------------ */
/* Neumaier compensated accumulator (Neumaier 1974).                         */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v))
    a->c += (a->s - t) + v;
  else
    a->c += (v - t) + a->s;
  a->s = t;
}
static double nsum_get(const nsum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Eq. 1 by direct summation.                                               */
/* ------------------------------------------------------------------------ */
int oracle_dft_naive(const double* x, double* X, int64_t N, int sign) {
  if (!x || !X || N < 1 || (sign != 1 && sign != -1)) return -1;
  double* w = (double*)malloc(sizeof(double) * 2 * (size_t)N);
  if (!w) return -2;
  for (int64_t m = 0; m < N; m++) oracle_twiddle(m, N, sign, &w[2 * m], &w[2 * m + 1]);
  int64_t nlast = N;
#if ORACLE_MUTANT == 2
  nlast = N - 1; /* MUTANT: last term of the sum dropped */
#endif
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; k++) {
    nsum re = {0.0, 0.0}, im = {0.0, 0.0};
    for (int64_t n = 0; n < nlast; n++) {
      /* exact phase index (n*k) mod N; n, k < N <= 2^31 for this routine */
      int64_t m = (int64_t)(((unsigned __int128)n * (unsigned __int128)k) % (unsigned __int128)N);
#if ORACLE_MUTANT == 3
      m = (m + 1) % N; /* MUTANT: phase index off by one */
#endif
      double xr = x[2 * n], xi = x[2 * n + 1];
      double wr = w[2 * m], wi = w[2 * m + 1];
      nsum_add(&re, xr * wr);
      nsum_add(&re, -(xi * wi));
      nsum_add(&im, xr * wi);
      nsum_add(&im, xi * wr);
    }
    X[2 * k] = nsum_get(&re);
    X[2 * k + 1] = nsum_get(&im);
  }
  free(w);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Radix-2 Cooley-Tukey, Sec. 2.2 (Eqs. 4-6).                               */
/* ------------------------------------------------------------------------ */
static uint64_t bit_reverse(uint64_t v, int bits) {
  uint64_t r = 0;
  for (int b = 0; b < bits; b++) {
    r = (r << 1) | (v & 1);
    v >>= 1;
  }
  return r;
}

int oracle_fft_radix2(double* x, int64_t N, int sign) {
  if (!x || !is_pow2(N) || (sign != 1 && sign != -1)) return -1;
  if (N == 1) return 0;
  const int e = ilog2_i64(N);

  /* Even/odd split applied recursively = inputs in bit-reversed order. */
#if ORACLE_MUTANT != 6 /* MUTANT 6: reordering skipped */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) {
    int64_t j = (int64_t)bit_reverse((uint64_t)i, e);
    if (i < j) {
      double tr = x[2 * i], ti = x[2 * i + 1];
      x[2 * i] = x[2 * j];
      x[2 * i + 1] = x[2 * j + 1];
      x[2 * j] = tr;
      x[2 * j + 1] = ti;
    }
  }
#endif

  /* T[t] = exp(sign*2*pi*i*t/N), t < N/2, each evaluated directly. */
  const int64_t H = N / 2;
  double* T = (double*)malloc(sizeof(double) * 2 * (size_t)H);
  if (!T) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < H; t++) twiddle_d(t, N, sign, &T[2 * t], &T[2 * t + 1]);

  /* Levels L = 2, 4, ..., N.  Block b of length L holds E (first half) and
   * O (second half); w = exp(sign*2*pi*i*j/L) = T[j*(N/L)]. */
  for (int64_t L = 2; L <= N; L *= 2) {
    const int64_t half = L / 2, step = N / L;
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < H; f++) {
      int64_t b = (f / half) * L, j = f % half;
#if ORACLE_MUTANT == 7
      int64_t t = j; /* MUTANT: twiddle stride forgotten */
#else
      int64_t t = j * step;
#endif
      double wr = T[2 * t], wi = T[2 * t + 1];
      double* u = &x[2 * (b + j)];
      double* v = &x[2 * (b + j + half)];
      double vr = v[0] * wr - v[1] * wi;
      double vi = v[0] * wi + v[1] * wr;
      double ur = u[0], ui = u[1];
      u[0] = ur + vr;
      u[1] = ui + vi;
#if ORACLE_MUTANT == 5
      v[0] = ur + vr; /* MUTANT: lower butterfly output with the wrong sign */
      v[1] = ui + vi;
#else
      v[0] = ur - vr;
      v[1] = ui - vi;
#endif
    }
  }
  free(T);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood 2014), counter form.                      */
/* ------------------------------------------------------------------------ */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t oracle_splitmix64(uint64_t seed, uint64_t i) {
#if ORACLE_MUTANT == 9
  return mix64(seed + i * 0x9E3779B97F4A7C15ull); /* MUTANT: counter offset lost */
#else
  return mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
#endif
}

static double uniform_pm1(uint64_t seed, uint64_t i) {
#if ORACLE_MUTANT == 8
  double u = (double)(oracle_splitmix64(seed, i) >> 12) * 0x1.0p-53; /* MUTANT: wrong bits */
#else
  double u = (double)(oracle_splitmix64(seed, i) >> 11) * 0x1.0p-53;
#endif
  return 2.0 * u - 1.0;
}

void oracle_gen_uniform(uint64_t seed, int64_t n0, int64_t count, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; i++) {
    uint64_t n = (uint64_t)(n0 + i);
    out[2 * i] = uniform_pm1(seed, 2 * n);
    out[2 * i + 1] = uniform_pm1(seed, 2 * n + 1);
  }
}

/* ------------------------------------------------------------------------ */
/* Sampled bins: Eq. 1 at a few k, input regenerated or given.              */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t N;
  int B;        /* low-table bits */
  double* lo;   /* exp(sign*2*pi*i*t/N), t < 2^B */
  double* hi;   /* exp(sign*2*pi*i*(t*2^B)/N), t < N/2^B */
} two_level;

static int two_level_init(two_level* tl, int64_t N, int sign) {
  int e = ilog2_i64(N);
  tl->N = N;
  tl->B = (e + 1) / 2;
  int64_t nlo = (int64_t)1 << tl->B, nhi = ((N - 1) >> tl->B) + 1; /* hi index of m <= N-1 */
  tl->lo = (double*)malloc(sizeof(double) * 2 * (size_t)nlo);
  tl->hi = (double*)malloc(sizeof(double) * 2 * (size_t)nhi);
  if (!tl->lo || !tl->hi) {
    free(tl->lo);
    free(tl->hi);
    return -2;
  }
  for (int64_t t = 0; t < nlo; t++) twiddle_d(t, N, sign, &tl->lo[2 * t], &tl->lo[2 * t + 1]);
  for (int64_t t = 0; t < nhi; t++)
    twiddle_d(t << tl->B, N, sign, &tl->hi[2 * t], &tl->hi[2 * t + 1]);
#if ORACLE_MUTANT == 10
  for (int64_t t = 0; t < nhi; t++) tl->hi[2 * t + 1] = -tl->hi[2 * t + 1]; /* MUTANT: conj */
#endif
  return 0;
}

static void two_level_free(two_level* tl) {
  free(tl->lo);
  free(tl->hi);
}

/* w = exp(sign*2*pi*i*m/N) for m < N as hi[m >> B] * lo[m & (2^B-1)] */
static void two_level_get(const two_level* tl, uint64_t m, double* wr, double* wi) {
  const double* a = &tl->hi[2 * (m >> tl->B)];
  const double* b = &tl->lo[2 * (m & (((uint64_t)1 << tl->B) - 1))];
#if ORACLE_MUTANT == 11
  *wr = a[0]; *wi = a[1]; (void)b; /* MUTANT: low factor dropped */
#else
  *wr = a[0] * b[0] - a[1] * b[1];
  *wi = a[0] * b[1] + a[1] * b[0];
#endif
}

#define BIN_BLOCK 4096

/* Shared body: x_at(n, &re, &im) yields input n. */
static int dft_bins_impl(const double* xarr, uint64_t seed, int64_t N, int sign,
                         const int64_t* ks, int64_t nk, double* X) {
  if (N < 1 || (sign != 1 && sign != -1) || nk < 0 || (nk > 0 && (!ks || !X))) return -1;
  if (nk == 0) return 0;
  two_level tl;
  if (two_level_init(&tl, N, sign)) return -2;
  const uint64_t UN = (uint64_t)N;
  int nth = oracle_threads();
  /* per-thread, per-bin compensated totals */
  nsum* acc = (nsum*)calloc((size_t)nth * (size_t)nk * 2, sizeof(nsum));
  if (!acc) {
    two_level_free(&tl);
    return -2;
  }
  int64_t nblocks = (N + BIN_BLOCK - 1) / BIN_BLOCK;
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    nsum* my = &acc[(size_t)tid * (size_t)nk * 2];
    double* blk = (double*)malloc(sizeof(double) * 2 * BIN_BLOCK);
    double* part = (double*)malloc(sizeof(double) * 2 * (size_t)nk);
#pragma omp for schedule(static)
    for (int64_t bI = 0; bI < nblocks; bI++) {
      int64_t n0 = bI * BIN_BLOCK;
      int64_t cnt = (n0 + BIN_BLOCK <= N) ? BIN_BLOCK : N - n0;
      const double* xb;
      if (xarr) {
        xb = &xarr[2 * n0];
      } else {
        for (int64_t i = 0; i < cnt; i++) {
          uint64_t n = (uint64_t)(n0 + i);
          blk[2 * i] = uniform_pm1(seed, 2 * n);
          blk[2 * i + 1] = uniform_pm1(seed, 2 * n + 1);
        }
        xb = blk;
      }
      for (int64_t j = 0; j < nk; j++) {
        const uint64_t k = (uint64_t)(((ks[j] % N) + N) % N);
        /* exact phase m = (n*k) mod N: 128-bit product at the block start,
         * then one addition of k (mod N) per term */
        uint64_t m = (uint64_t)(((unsigned __int128)(uint64_t)n0 * k) % UN);
        double sr = 0.0, si = 0.0;
        for (int64_t i = 0; i < cnt; i++, m = (m + k >= UN) ? m + k - UN : m + k) {
          double wr, wi;
          two_level_get(&tl, m, &wr, &wi);
          double xr = xb[2 * i], xi = xb[2 * i + 1];
          sr += xr * wr - xi * wi;
          si += xr * wi + xi * wr;
        }
        part[2 * j] = sr;
        part[2 * j + 1] = si;
      }
      for (int64_t j = 0; j < nk; j++) {
        nsum_add(&my[2 * j], part[2 * j]);
        nsum_add(&my[2 * j + 1], part[2 * j + 1]);
      }
    }
    free(blk);
    free(part);
  }
  for (int64_t j = 0; j < nk; j++) {
    nsum re = {0.0, 0.0}, im = {0.0, 0.0};
    for (int t = 0; t < nth; t++) {
      const nsum* a = &acc[((size_t)t * (size_t)nk + (size_t)j) * 2];
      nsum_add(&re, a[0].s);
      nsum_add(&re, a[0].c);
      nsum_add(&im, a[1].s);
      nsum_add(&im, a[1].c);
    }
    X[2 * j] = nsum_get(&re);
    X[2 * j + 1] = nsum_get(&im);
  }
  free(acc);
  two_level_free(&tl);
  return 0;
}

int oracle_dft_bins_uniform(uint64_t seed, int64_t N, int sign, const int64_t* ks, int64_t nk,
                            double* X) {
  return dft_bins_impl(NULL, seed, N, sign, ks, nk, X);
}

int oracle_dft_bins(const double* x, int64_t N, int sign, const int64_t* ks, int64_t nk,
                    double* X) {
  if (!x) return -1;
  return dft_bins_impl(x, 0, N, sign, ks, nk, X);
}
