/*
 * efft.h -- C ABI of the GB300 (sm_103a) in-place 1-D complex DFT library.
 *
 * What it computes (the paper's problem statement, Eq. 1 of Sec. 1):
 *
 *     X[k] = sum_{n=0}^{N-1} x[n] * exp(sign * 2*pi*i * n*k / N),  0 <= k < N,
 *
 * in place, unnormalised.  sign = -1 is the forward transform printed in
 * Eq. 1; sign = +1 is the conjugate-sign transform (the adjoint; applying it
 * after the forward transform and dividing by N recovers x).
 *
 * How (the paper's three stages, Sec. 2.3, restated for one GPU): N = 2^e is
 * split into radices R_0 * R_1 * ... * R_{p-1}; each pass runs a batch of
 * strided size-R_j sub-FFTs in shared memory (the "processing" of bins,
 * Sec. 3.3) with the twiddle factors of Eq. 4 fused into its epilogue (the
 * "reassembly", Sec. 3.4), writing back to the slots it read (the in-place
 * principle of Sec. 3.4, Fig. 4-5).  The digit-reversed result is put in
 * natural order by a tiled in-place transpose (the "scattering" of
 * Sec. 3.2, Listings 5-6, moved to the end).
 *
 * Data layout: interleaved complex, element n at byte offset n*S with
 * S = 16 (EFFT_C128: two IEEE binary64, re then im; torch.complex128) or
 * S = 8 (EFFT_C64: two binary32; torch.complex64).
 *
 * Threading: apart from its profiling records, a plan is immutable after
 * creation and may be shared by host threads; executes of one plan must be
 * stream-ordered (they share the plan's 16-byte device state word), and two
 * executes that touch the same buffer concurrently race.
 * All entry points return an efft_status code; none aborts the process.
 */
#ifndef EFFT_H
#define EFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EFFT_VERSION 1

/* Element types.  Interleaved (re, im). */
enum efft_dtype {
  EFFT_C64 = 0,  /* 2 x float32, 8 bytes per element  */
  EFFT_C128 = 1  /* 2 x float64, 16 bytes per element */
};

/* Status codes returned by every entry point. */
enum efft_status {
  EFFT_OK = 0,
  EFFT_ERR_INVALID_SIZE = 1,   /* N is not 2^e with 0 <= e <= EFFT_MAX_LOG2N   */
  EFFT_ERR_INVALID_DTYPE = 2,  /* dtype is not EFFT_C64 / EFFT_C128             */
  EFFT_ERR_INVALID_SIGN = 3,   /* sign is not -1 or +1                          */
  EFFT_ERR_INVALID_PTR = 4,    /* NULL, or not device memory of this device     */
  EFFT_ERR_MISALIGNED = 5,     /* data pointer not aligned to the element size  */
  EFFT_ERR_ALLOC = 6,          /* device or host allocation failed              */
  EFFT_ERR_LAUNCH = 7,         /* a kernel launch or async copy was rejected    */
  EFFT_ERR_TIMEOUT = 8,        /* reserved: a bounded device wait expired       */
  EFFT_ERR_UNSUPPORTED = 9,    /* valid request this build does not implement   */
  EFFT_ERR_INVALID_PLAN = 10,  /* NULL, destroyed or foreign plan handle        */
  EFFT_ERR_CUDA = 11,          /* CUDA runtime error (no device, bad context)   */
  EFFT_ERR_INVALID_FLAGS = 12  /* unknown bits in flags                         */
};

/* Largest supported log2 N (2^33 complex128 = 128 GiB). */
#define EFFT_MAX_LOG2N 33

/*
 * Plan flags.
 *  EFFT_FLAG_DIGIT_REVERSED_OUT: skip the final in-place transpose.  Output
 *    position P = sum_j q_j * s_j (s_j = R_{j+1} * ... * R_{p-1}, 0 <= q_j <
 *    R_j) then holds X[q_0 + R_0*q_1 + R_0*R_1*q_2 + ...]; the radices are
 *    reported by efft_plan_radices().
 */
#define EFFT_FLAG_DIGIT_REVERSED_OUT 0x1u
/*  EFFT_FLAG_NORMALIZE: multiply the output by 1/N (exact: N is a power of
 *    two).  Not part of Eq. 1, which is unnormalised; with sign = +1 it gives
 *    the inverse DFT, so forward then normalised inverse returns x. */
#define EFFT_FLAG_NORMALIZE 0x2u
#define EFFT_FLAG_ALL 0x3u

typedef struct efft_plan_s* efft_plan_t;

/*
 * Create a plan for N-point transforms of the given dtype and sign on the
 * CUDA device current on the calling thread.  This is the one-time set-up of
 * the paper's Sec. 3.1 (Listing 3): it chooses the radices, allocates the
 * plan's device tables (O(sqrt N) twiddle factors, generated on the device in
 * FP64, plus a few bytes of per-plan state) and synchronises.
 *  out    [out] receives the handle (set to NULL on failure).
 *  n      transform length, a power of two, 1 <= n <= 2^EFFT_MAX_LOG2N.
 *  dtype  EFFT_C64 or EFFT_C128.
 *  sign   -1 (forward, Eq. 1) or +1 (conjugate sign).
 *  flags  bitwise OR of EFFT_FLAG_*.
 * Errors: INVALID_SIZE / INVALID_DTYPE / INVALID_SIGN / INVALID_FLAGS are
 * detected before any CUDA call; ALLOC or CUDA if device set-up fails.
 * Ownership: the caller destroys the plan with efft_plan_destroy().
 */
int efft_plan_create(efft_plan_t* out, uint64_t n, int dtype, int sign, uint32_t flags);

/*
 * Enqueue one in-place transform of the n elements at `data` on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Asynchronous: returns
 * after enqueueing; the result is ready when the stream reaches that point.
 *  data   device pointer (cudaMalloc / torch CUDA tensor storage) on the
 *         plan's device, aligned to the element size, n*S bytes, owned by
 *         the caller.  Its contents are replaced by X.
 * The plan's device state is used by the launched kernels: executes of one
 * plan must be ordered (same stream, or events), or they race on that state.
 * Errors: INVALID_PLAN, INVALID_PTR, MISALIGNED before any launch; LAUNCH if
 * CUDA rejects a launch (the buffer may then be partly transformed).
 * Non-finite inputs (Inf/NaN) give NaN in every output; subnormal complex128
 * inputs are treated as zero.
 */
int efft_execute(efft_plan_t plan, void* data, void* stream);

/*
 * Convenience form for host-resident data: copies n elements from
 * `host_data` to the device buffer `dev_data` (n*S bytes, caller-owned),
 * transforms it in place and copies the result back to `host_data`, all
 * enqueued on `stream`, then synchronises the stream.  Pinned host memory
 * gives the full copy bandwidth.
 * Errors: as efft_execute, plus INVALID_PTR for a NULL host pointer and CUDA
 * if a copy or the synchronisation fails.
 */
int efft_execute_host(efft_plan_t plan, void* host_data, void* dev_data, void* stream);

/*
 * Stream `count` host arrays through the device with the copies overlapped
 * with the transforms.  Array i is copied from host_in[i] into device buffer
 * dev_bufs[i % nbufs], the plans[0 .. nplans) are applied to it in order, in
 * place, and the result is copied to host_out[i].  Copies in, transforms and
 * copies out run on three streams (the transforms on `stream`), so array i+1
 * is copied in and array i-1 copied out while array i is transformed; a
 * buffer is reused only after the copy-out of its previous array finished.
 * With nbufs >= 3 the copies in both directions also overlap each other.
 * Synchronous: returns when every result is in host memory.
 *  plans      nplans >= 1 live plans with the same n and dtype.
 *  host_in    count host pointers (pinned memory gives the full copy rate).
 *  host_out   count host pointers; host_out[i] may equal host_in[i] but must
 *             not overlap any host_in[j], j != i.  Several host_in entries may
 *             share memory, and so may several host_out entries (the copies
 *             out are issued in order on one stream).
 *  dev_bufs   nbufs >= 1 device buffers of n*S bytes on the plans' device.
 * Errors: INVALID_PLAN, INVALID_PTR, MISALIGNED, INVALID_SIZE (plans of
 * different n or dtype, count < 0, nplans or nbufs < 1), LAUNCH, CUDA.
 */
int efft_execute_host_stream(const efft_plan_t* plans, int nplans, void* const* host_in,
                             void* const* host_out, int count, void* const* dev_bufs, int nbufs,
                             void* stream);

/* Destroy a plan and free its device tables.  NULL is accepted (no-op).
 * Errors: INVALID_PLAN for a handle that is not a live plan. */
int efft_plan_destroy(efft_plan_t plan);

/* Static, human-readable text for a status code (never NULL). */
const char* efft_strerror(int status);

/* Library version (EFFT_VERSION of the build). */
int efft_version(void);

/*
 * Plan introspection.
 *  efft_plan_radices: writes log2 of R_0..R_{p-1} to log2_radices (room for
 *    at most `cap` entries) and p to *npasses.
 *  efft_plan_info: *hbm_passes = number of full read+write sweeps of the
 *    array one execute makes (sub-FFT passes + transpose; the range scan of
 *    a complex128 execute, which only reads, counts as 0.5); *table_bytes =
 *    device bytes the plan owns.
 */
int efft_plan_radices(efft_plan_t plan, int* log2_radices, int cap, int* npasses);
int efft_plan_info(efft_plan_t plan, double* hbm_passes, uint64_t* table_bytes);

/*
 * Per-kernel timing with CUDA events recorded on the execute's own stream
 * around every launch (measurement support; no effect on results).
 *  efft_plan_profile(plan, 1) starts recording for subsequent executes and
 *    clears earlier records; efft_plan_profile(plan, 0) stops recording.
 *  efft_plan_profile_read synchronises on the recorded events and writes, per
 *    launch slot s < cap, total milliseconds ms[s] and launch count count[s];
 *    *nslots receives EFFT_PROFILE_SLOTS.  Slots: 0 range scan (complex128),
 *    1 + j pass j (j < 4), 5 digit swap, 6 direct-sum kernel (N <= 8).
 *    Records are consumed by the read.
 * Profiling mutates the plan: do not profile a plan that other host threads
 * execute concurrently.
 */
#define EFFT_PROFILE_SLOTS 7
int efft_plan_profile(efft_plan_t plan, int enable);
int efft_plan_profile_read(efft_plan_t plan, double* ms, int* count, int cap, int* nslots);

/*
 * One transform that allocates nothing (the paper has no counterpart; this
 * is for callers that cannot call cudaMalloc: a framework whose pooled
 * allocator owns all device memory, or a pipeline that cannot afford
 * cudaMalloc's implicit device-wide synchronisation).
 *
 * Computes what a plan created with (n, dtype, sign, flags) and efft_execute
 * compute, with the same kernels, on the `data` buffer (the caller's device
 * memory, as for efft_execute) on `stream`.  Instead of plan-owned memory it
 * uses one file-scope device array of the library holding the twiddle
 * tables (2048 + 2 * 4096 complex entries) and a 16-byte state word,
 * 160 KiB plus 256 bytes, that every GPU which loads the library keeps until
 * the process exits.  No cudaMalloc, cudaFree or allocating library call is
 * made.
 *  n      a power of two, 1 <= n <= 2^EFFT_NOALLOC_MAX_LOG2N; larger n is
 *         rejected with EFFT_ERR_INVALID_SIZE (use a plan instead).
 * Set-up: the first call on a device (with that device current) looks up
 * the array's device address and enqueues the table generation; make that
 * first call before any stream capture.  The tables are regenerated, on the
 * call's stream, whenever n differs from the previous call on the device.
 * Every call shares the array, which keeps the last call's contents; the
 * state word is cleared by each call before use.  Calls whose work overlaps
 * on the GPU (different streams without ordering) race on the array and give
 * undefined results: order them.
 * Errors: as efft_plan_create (argument checks) and efft_execute (buffer
 * checks, LAUNCH).
 */
#define EFFT_NOALLOC_MAX_LOG2N 24
int efft_execute_noalloc(void* data, uint64_t n, int dtype, int sign, uint32_t flags, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* EFFT_H */
