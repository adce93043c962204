/*
 * efft_inputs.h -- seeded synthetic inputs and norm reductions on the device.
 *
 * A separate library (libefft_inputs.so) from the transform: it holds no DFT
 * arithmetic.  It exists so that tests and the benchmark can create inputs of
 * 2^30..2^33 elements directly in HBM and reduce them there.
 *
 * The generator is SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) in counter
 * form: output i of the stream seeded with s is
 *     mix64(s + (i+1) * 0x9E3779B97F4A7C15),
 *     mix64(z) = z ^= z>>30, z *= 0xBF58476D1CE4E5B9, z ^= z>>27,
 *                z *= 0x94D049BB133111EB, z ^= z>>31.
 * Element n, part c (0 = re, 1 = im) uses output i = 2n + c; its top 53 bits
 * give u in [0, 1).  The CPU oracle carries its own implementation of the
 * same definition; tests check the two bit for bit.
 *
 * All pointers marked "dev" are device memory the caller owns; all calls are
 * asynchronous on `stream` (a cudaStream_t, NULL = default stream) except
 * where stated.  Return: 0 on success, otherwise a CUDA error code.
 */
#ifndef EFFT_INPUTS_H
#define EFFT_INPUTS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* x[n] = (2u_{2n} - 1) + i(2u_{2n+1} - 1), n = n0 .. n0+count-1, written to
 * dev[0 .. count).  dtype 1 = complex128 (exact), 0 = complex64 (the same
 * values rounded to binary32). */
int efft_gen_uniform(void* dev, uint64_t count, int dtype, uint64_t seed, uint64_t n0, void* stream);

/* Gaussian(0, 1) re and im by Box-Muller on (u_{2n}, u_{2n+1}):
 * r = sqrt(-2 ln(1 - u_{2n})), theta = 2*pi*u_{2n+1},
 * x[n] = r cos(theta) + i r sin(theta), evaluated in FP64 on the device. */
int efft_gen_gaussian(void* dev, uint64_t count, int dtype, uint64_t seed, uint64_t n0, void* stream);

/* x[n] += sum_j a_j * exp(+2*pi*i * f_j * n / N) for n < N (the whole array),
 * phase (f_j * n) mod N exact in integers, sincospi in FP64.
 * freqs, amps (re, im pairs) are HOST arrays of ntones entries (<= 256). */
int efft_add_tones(void* dev, uint64_t N, int dtype, const int64_t* freqs, const double* amps,
                   int ntones, void* stream);

/* Synchronous FP64 reductions over complex arrays of `count` elements:
 * out[0] = sum |scale*a[n] - b[n]|^2, out[1] = sum |b[n]|^2.  b may be NULL
 * (then out[0] = sum |scale*a|^2, out[1] = 0).  out is a HOST array of 2. */
int efft_diff_norms(const void* a, const void* b, uint64_t count, int dtype, double scale,
                    double* out, void* stream);

/* Page-locked host memory for benchmark buffers (cudaHostAlloc /
 * cudaFreeHost); *ptr receives the address.  Synchronous. */
int efft_host_alloc(void** ptr, uint64_t bytes);
int efft_host_free(void* ptr);

#ifdef __cplusplus
}
#endif
#endif
