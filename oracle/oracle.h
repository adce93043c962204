/*
 * oracle.h -- plain, slow, CPU reference for the one-dimensional complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this library.
 * It shares no code, header, table or constant with the CUDA library and
 * neither side includes or links the other.
 *
 * Everything is IEEE binary64 ("double"); complex arrays are interleaved
 * (re, im) pairs, element n at x[2n], x[2n+1].  The transform computed by
 * every routine is the DFT of Eq. 1 of the paper (Sec. 1),
 *
 *     X[k] = sum_{n=0}^{N-1} x[n] * exp(sign * 2*pi*i * n*k / N),
 *
 * with sign = -1 the forward transform printed in Eq. 1 and sign = +1 the
 * unnormalised conjugate-sign transform (no 1/N factor anywhere).
 *
 * Pins: every function here is checked in tests/test_oracle_pins.py against
 * closed forms, brute force in multiple precision, numpy's FFT and
 * invariants; tests/test_oracle_mutants.py rebuilds this file with planted
 * mistakes (ORACLE_MUTANT=k) and checks that each one fails a pin.
 */
#ifndef EFFT_ORACLE_H
#define EFFT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Version of this oracle's arithmetic (bumped when the arithmetic changes). */
int oracle_version(void);

/* Active planted mistake (0 = none); see ORACLE_MUTANT in oracle.c. */
int oracle_mutant(void);

/*
 * exp(sign*2*pi*i*m/N) in long double with exact octant reduction of the
 * integer phase m mod N, rounded to double.  The angle that reaches cosl/sinl
 * never exceeds pi/4.  Follows the twiddle factor of Eq. 4 (Sec. 2.2).
 */
void oracle_twiddle(int64_t m, int64_t N, int sign, double* re, double* im);

/*
 * Direct O(N^2) evaluation of Eq. 1 (Sec. 1): X = DFT(x).  x and X are
 * 2*N doubles, must not alias.  Phase index (n*k) mod N is exact integer
 * arithmetic; the N twiddles come from oracle_twiddle(); the sum over n is
 * Neumaier-compensated.  Any N >= 1.  Returns 0, or -1 on a bad argument.
 */
int oracle_dft_naive(const double* x, double* X, int64_t N, int sign);

/*
 * Iterative radix-2 Cooley-Tukey FFT in place (Sec. 2.2): bit-reversal
 * reordering, then log2 N levels of the butterfly pair of Eqs. 5-6,
 * F_k = E_k + w*O_k and F_{k+L/2} = E_k - w*O_k with w = exp(sign*2*pi*i*k/L).
 * The N/2 twiddles are evaluated one by one (octant-reduced double sin/cos,
 * no recurrence).  N must be a power of two >= 1.  OpenMP-parallel.
 * Returns 0, or -1 on a bad argument, -2 if the table cannot be allocated.
 */
int oracle_fft_radix2(double* x, int64_t N, int sign);

/*
 * Seeded input generator (the oracle's own copy; the device generator is a
 * separate implementation of the same published definition).  SplitMix64
 * (Steele, Lea & Flood, OOPSLA 2014): output i of the stream seeded with s is
 * mix64(s + (i+1)*0x9E3779B97F4A7C15).  Element n, part c (0 = re, 1 = im)
 * takes output i = 2n + c; its top 53 bits give u in [0,1) and the value is
 * 2u - 1 in [-1, 1), exact in double.  Writes elements n0 .. n0+count-1.
 */
void oracle_gen_uniform(uint64_t seed, int64_t n0, int64_t count, double* out);

/* Raw SplitMix64 output i of the stream seeded with s (for known-answer pins). */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t i);

/*
 * Sampled mode: X[k] of Eq. 1 for the nk frequencies ks[], where x is the
 * uniform input of oracle_gen_uniform(seed, 0, N) regenerated on the fly, so
 * no N-element array is ever held.  Any N >= 1.  Phase (n*k) mod N is exact
 * in integers; exp(sign*2*pi*i*m/N) = hi-table * lo-table (two levels,
 * double); partial sums over blocks of 4096 terms are combined with Neumaier
 * compensation.  Returns 0 or -1 / -2 as above.
 */
int oracle_dft_bins_uniform(uint64_t seed, int64_t N, int sign,
                            const int64_t* ks, int64_t nk, double* X);

/*
 * Same as oracle_dft_bins_uniform but for an explicit input array x (2*N
 * doubles): the direct sum of Eq. 1 at the listed bins only.
 */
int oracle_dft_bins(const double* x, int64_t N, int sign,
                    const int64_t* ks, int64_t nk, double* X);

/* Threads the OpenMP routines use (omp_get_max_threads()). */
int oracle_threads(void);

#ifdef __cplusplus
}
#endif
#endif
