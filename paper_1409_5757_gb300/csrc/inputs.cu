// inputs.cu -- seeded device inputs and FP64 norm reductions (include/efft_inputs.h).
//
// Test and benchmark harness only: no DFT arithmetic lives here.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "../../include/efft_inputs.h"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double unit53(uint64_t seed, uint64_t i) {
  return (double)(mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53;
}

__global__ void k_uniform(void* dev, uint64_t count, int dtype, uint64_t seed, uint64_t n0) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t n = n0 + i;
    double re = 2.0 * unit53(seed, 2 * n) - 1.0;
    double im = 2.0 * unit53(seed, 2 * n + 1) - 1.0;
    if (dtype == 1) reinterpret_cast<double2*>(dev)[i] = make_double2(re, im);
    else reinterpret_cast<float2*>(dev)[i] = make_float2(__double2float_rn(re), __double2float_rn(im));
  }
}

__global__ void k_gaussian(void* dev, uint64_t count, int dtype, uint64_t seed, uint64_t n0) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t n = n0 + i;
    double u1 = unit53(seed, 2 * n), u2 = unit53(seed, 2 * n + 1);
    double r = sqrt(-2.0 * log(1.0 - u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    double re = r * c, im = r * s;
    if (dtype == 1) reinterpret_cast<double2*>(dev)[i] = make_double2(re, im);
    else reinterpret_cast<float2*>(dev)[i] = make_float2(__double2float_rn(re), __double2float_rn(im));
  }
}

struct Tones {
  int n;
  long long f[256];
  double ar[256], ai[256];
};

__global__ void k_tones(void* dev, uint64_t N, int dtype, const Tones* __restrict__ t) {
  const int nt = t->n;
  for (uint64_t n = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += (uint64_t)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < nt; ++j) {
      uint64_t m = ((uint64_t)t->f[j] * n) & (N - 1);  // exact phase (N | 2^64)
      double s, c;
      sincospi(2.0 * ((double)m / (double)N), &s, &c);
      re += t->ar[j] * c - t->ai[j] * s;
      im += t->ar[j] * s + t->ai[j] * c;
    }
    if (dtype == 1) {
      double2 v = reinterpret_cast<double2*>(dev)[n];
      reinterpret_cast<double2*>(dev)[n] = make_double2(v.x + re, v.y + im);
    } else {
      float2 v = reinterpret_cast<float2*>(dev)[n];
      reinterpret_cast<float2*>(dev)[n] = make_float2(__double2float_rn((double)v.x + re),
                                                      __double2float_rn((double)v.y + im));
    }
  }
}

__global__ void k_norms(const void* a, const void* b, uint64_t count, int dtype, double scale, double* out) {
  double s0 = 0.0, s1 = 0.0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    double ar, ai, br = 0.0, bi = 0.0;
    if (dtype == 1) {
      double2 v = reinterpret_cast<const double2*>(a)[i];
      ar = v.x; ai = v.y;
      if (b) { double2 w = reinterpret_cast<const double2*>(b)[i]; br = w.x; bi = w.y; }
    } else {
      float2 v = reinterpret_cast<const float2*>(a)[i];
      ar = v.x; ai = v.y;
      if (b) { float2 w = reinterpret_cast<const float2*>(b)[i]; br = w.x; bi = w.y; }
    }
    double dr = scale * ar - br, di = scale * ai - bi;
    s0 += dr * dr + di * di;
    s1 += br * br + bi * bi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, o);
    s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
  }
  __shared__ double w0[32], w1[32];
  if ((threadIdx.x & 31) == 0) { w0[threadIdx.x >> 5] = s0; w1[threadIdx.x >> 5] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t0 += w0[w]; t1 += w1[w]; }
    out[2 * blockIdx.x] = t0;
    out[2 * blockIdx.x + 1] = t1;
  }
}

unsigned grid_for(uint64_t count) {
  uint64_t g = (count + 255) / 256;
  if (g > 152ull * 16) g = 152ull * 16;
  if (g == 0) g = 1;
  return (unsigned)g;
}

}  // namespace

extern "C" {

int efft_gen_uniform(void* dev, uint64_t count, int dtype, uint64_t seed, uint64_t n0, void* stream) {
  if (count == 0) return 0;
  k_uniform<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(dev, count, dtype, seed, n0);
  return (int)cudaGetLastError();
}

int efft_gen_gaussian(void* dev, uint64_t count, int dtype, uint64_t seed, uint64_t n0, void* stream) {
  if (count == 0) return 0;
  k_gaussian<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(dev, count, dtype, seed, n0);
  return (int)cudaGetLastError();
}

int efft_add_tones(void* dev, uint64_t N, int dtype, const int64_t* freqs, const double* amps, int ntones,
                   void* stream) {
  if (ntones < 0 || ntones > 256 || (N & (N - 1)) != 0) return (int)cudaErrorInvalidValue;
  if (ntones == 0 || N == 0) return 0;
  Tones h;
  std::memset(&h, 0, sizeof(h));
  h.n = ntones;
  for (int j = 0; j < ntones; ++j) {
    h.f[j] = (long long)freqs[j];
    h.ar[j] = amps[2 * j];
    h.ai[j] = amps[2 * j + 1];
  }
  cudaStream_t st = (cudaStream_t)stream;
  Tones* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(Tones));
  if (e != cudaSuccess) return (int)e;
  e = cudaMemcpyAsync(d, &h, sizeof(Tones), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_tones<<<grid_for(N), 256, 0, st>>>(dev, N, dtype, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  return (int)e;
}

int efft_diff_norms(const void* a, const void* b, uint64_t count, int dtype, double scale, double* out,
                    void* stream) {
  out[0] = out[1] = 0.0;
  if (count == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned g = grid_for(count);
  double* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(double) * 2 * g);
  if (e != cudaSuccess) return (int)e;
  k_norms<<<g, 256, 0, st>>>(a, b, count, dtype, scale, d);
  e = cudaGetLastError();
  double* h = new double[2 * g];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(double) * 2 * g, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    for (unsigned i = 0; i < g; ++i) { out[0] += h[2 * i]; out[1] += h[2 * i + 1]; }
  }
  delete[] h;
  cudaFree(d);
  return (int)e;
}

int efft_host_alloc(void** ptr, uint64_t bytes) {
  if (!ptr) return (int)cudaErrorInvalidValue;
  return (int)cudaHostAlloc(ptr, bytes, cudaHostAllocDefault);
}

int efft_host_free(void* ptr) { return (int)cudaFreeHost(ptr); }

}  // extern "C"
