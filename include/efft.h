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
 * creation and may be shared by host threads.  Executes of one plan on
 * different buffers may run concurrently on unordered streams: each execute
 * has a 16-byte device state word of its own (see efft_execute).  Two
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
  EFFT_ERR_INVALID_SIZE = 1,   /* N is not M * 2^e (M odd <= 15), or too large  */
  EFFT_ERR_INVALID_DTYPE = 2,  /* dtype is not EFFT_C64 / EFFT_C128             */
  EFFT_ERR_INVALID_SIGN = 3,   /* sign is not -1 or +1                          */
  EFFT_ERR_INVALID_PTR = 4,    /* NULL, or not device memory of this device     */
  EFFT_ERR_MISALIGNED = 5,     /* data pointer not aligned to the element size  */
  EFFT_ERR_ALLOC = 6,          /* device or host allocation failed              */
  EFFT_ERR_LAUNCH = 7,         /* a kernel launch or async copy was rejected    */
  EFFT_ERR_TIMEOUT = 8,        /* reserved: a bounded device wait expired       */
  EFFT_ERR_UNSUPPORTED = 9,    /* valid request the library does not implement  */
  EFFT_ERR_INVALID_PLAN = 10,  /* NULL, destroyed or foreign plan handle        */
  EFFT_ERR_CUDA = 11,          /* CUDA runtime error (no device, bad context)   */
  EFFT_ERR_INVALID_FLAGS = 12  /* unknown bits in flags                         */
};

/* Largest supported log2 N (2^33 complex128 = 128 GiB). */
#define EFFT_MAX_LOG2N 33
/* Supported lengths: N = M * 2^e with M odd, 1 <= M <= EFFT_MAX_ODD (the
 * paper's size set N = M * 2^s, Sec. 2.1), 1 <= N <= 2^EFFT_MAX_LOG2N. */
#define EFFT_MAX_ODD 15

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
/*  EFFT_FLAG_AUTOTUNE: choose the radix schedule by measurement instead of
 *    the built-in table (the GPU counterpart of the paper's scan over the
 *    split depth s and the worker count, Sec. 5.2, Figs. 6-7).  A schedule
 *    cached for (device, n, dtype) by an earlier tuning is reused; otherwise,
 *    if n*S <= EFFT_AUTOTUNE_MAX_BYTES, efft_plan_create allocates a
 *    temporary n*S-byte buffer and runs efft_plan_autotune on it.  Larger n
 *    keep the table's schedule unless efft_plan_autotune is called with a
 *    caller buffer.  Results are unchanged up to rounding. */
#define EFFT_FLAG_AUTOTUNE 0x4u
#define EFFT_FLAG_ALL 0x7u
#define EFFT_AUTOTUNE_MAX_BYTES (1ull << 31)

typedef struct efft_plan_s* efft_plan_t;

/*
 * Create a plan for N-point transforms of the given dtype and sign on the
 * CUDA device current on the calling thread.  This is the one-time set-up of
 * the paper's Sec. 3.1 (Listing 3): it chooses the radices, allocates the
 * plan's device tables (O(sqrt N) twiddle factors, generated on the device in
 * FP64, plus a few bytes of per-plan state) and synchronises.
 *  out    [out] receives the handle (set to NULL on failure).
 *  n      transform length N = M * 2^e (M odd, M <= EFFT_MAX_ODD),
 *         1 <= n <= 2^EFFT_MAX_LOG2N.  For M > 1 the schedule is one
 *         mixed-radix pass (N up to 2048 points) or three passes
 *         (2^a, M*2^b, 2^a): palindromic, so the final digit reversal is the
 *         same in-place swap; efft_plan_radices then reports the
 *         power-of-two part of each radix (M belongs to the middle or only
 *         pass, whose extent is N / 4^a) and efft_plan_schedule the whole
 *         radices.  EFFT_FLAG_NORMALIZE is rejected for M > 1
 *         (EFFT_ERR_UNSUPPORTED: 1/N is not exact in binary floating point);
 *         explicit schedules, the autotuner and the no-allocation entry
 *         point take powers of two.
 *  dtype  EFFT_C64 or EFFT_C128.
 *  sign   -1 (forward, Eq. 1) or +1 (conjugate sign).
 *  flags  bitwise OR of EFFT_FLAG_*.
 * Errors: INVALID_SIZE / INVALID_DTYPE / INVALID_SIGN / INVALID_FLAGS /
 * UNSUPPORTED are detected before any CUDA call; ALLOC or CUDA if device
 * set-up fails.
 * Ownership: the caller destroys the plan with efft_plan_destroy().
 */
int efft_plan_create(efft_plan_t* out, uint64_t n, int dtype, int sign, uint32_t flags);

/*
 * Enqueue one in-place transform of the n elements at `data` on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Asynchronous: returns
 * after enqueueing; the result is ready when the stream reaches that point.
 * This is the paper's EFFT_Transform::RunTransform() (Sec. 4, Listings 12-13),
 * in place on a caller buffer instead of out of place on plan-owned arrays.
 *  data   device pointer (cudaMalloc / torch CUDA tensor storage) on the
 *         plan's device, aligned to the element size, n*S bytes, owned by
 *         the caller.  Its contents are replaced by X.
 * Device state: a complex128 execute records the largest binary64 exponent
 * of its input in a 16-byte state word that its later launches read.  The
 * plan keeps a ring of 16 such words; an execute takes the next one and its
 * launches first wait (on the device, through an event) for the execute that
 * used that word before, so executes on different buffers never share a
 * word while they run.  An execute enqueued while `stream` is being captured
 * into a CUDA graph instead gets a word from the stream-ordered allocator,
 * allocated and freed inside the graph (each launch of the graph has its own).
 * Errors: INVALID_PLAN, INVALID_PTR, MISALIGNED before any launch; LAUNCH if
 * CUDA rejects a launch (the buffer may then be partly transformed); CUDA if
 * the stream's capture state cannot be read or the capture was invalidated;
 * ALLOC if the graph allocation of a captured execute fails.
 * Special values: non-finite inputs (Inf/NaN) give NaN in every output.
 * complex128 data are scaled by a power of two so that the largest input
 * magnitude lies in [1, 2) and carried as pairs of binary32 numbers.  So an
 * input component whose binary64 exponent is more than 126 below the
 * largest input exponent is treated as zero (this includes every subnormal
 * input), and one whose exponent is more than 74 below it keeps 24 of its
 * 53 significand bits; either change is below 2^-74 of the largest input,
 * far under the transform's rounding error.  This is not binary64
 * behaviour.  Outputs whose magnitude falls below the smallest normal
 * binary64 number are flushed to zero.
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
 * is copied in and array i-1 copied out while array i is transformed.  The
 * copies go in 1 GiB pieces; a piece of a buffer is refilled once the copy
 * out of the buffer's previous array has read that piece, so even with one
 * buffer the copy out of array i and the copy in of array i+nbufs overlap
 * (the link's two directions), and with nbufs >= 3 the copies in both
 * directions also overlap the transforms.
 * Synchronous: returns when every result is in host memory.
 *  plans      nplans >= 1 live plans with the same n and dtype.
 *  host_in    count host pointers (pinned memory gives the full copy rate).
 *  host_out   count host pointers; host_out[i] may equal host_in[i] but must
 *             not overlap any host_in[j], j != i, except that with nbufs = 1
 *             host_in[j] (j > i) may equal host_out[i] (each piece is then
 *             copied in after the same piece was copied out).  Several
 *             host_in entries may share memory, and so may several host_out
 *             entries (the copies out are issued in order on one stream).
 *  dev_bufs   nbufs >= 1 device buffers of n*S bytes on the plans' device.
 * Errors: INVALID_PLAN, INVALID_PTR, MISALIGNED, INVALID_SIZE (plans of
 * different n or dtype, count < 0, nplans or nbufs < 1), LAUNCH, CUDA.
 */
int efft_execute_host_stream(const efft_plan_t* plans, int nplans, void* const* host_in,
                             void* const* host_out, int count, void* const* dev_bufs, int nbufs,
                             void* stream);

/*
 * Create a plan with an explicit radix schedule (log2 R_0 .. log2 R_{p-1});
 * otherwise as efft_plan_create.  Accepted schedules:
 *  p = 0 for n <= 8 (direct sums);
 *  p = 1 with log2 R_0 = log2 n in [4, 11];
 *  p = 2 or 3 with every log2 R_j in [4, 11], sum log2 n, and R_0 = R_{p-1}
 *    (symmetric: the digit reversal is then an involution, done in place).
 * For n = M * 2^e with M > 1 odd (Sec. 2.1's size set):
 *  p = 1 with log2 R_0 = e and n <= 2048 (one CTA tile);
 *  p = 3 given as (a, b, a), a >= 1, 2a + b = e: the passes 2^a, M * 2^b,
 *    2^a, each at most 2048 points.
 * Any other schedule: EFFT_ERR_UNSUPPORTED (before any CUDA call).
 * EFFT_FLAG_AUTOTUNE is rejected here (EFFT_ERR_INVALID_FLAGS).
 */
int efft_plan_create_with_radices(efft_plan_t* out, uint64_t n, int dtype, int sign, uint32_t flags,
                                  const int* log2_radices, int npasses);

/*
 * Measure the plan's schedules and kernel variants and switch the plan to
 * the fastest (the GPU counterpart of the paper's scan over the split depth s
 * and the worker count, Sec. 5.2, Figs. 6-7); the choice is cached for
 * (device, n, dtype) and used by later plans created with
 * EFFT_FLAG_AUTOTUNE.  Candidates, in order:
 *  - n a power of two: every accepted schedule (above) with the built-in
 *    variant rules; then, for the fastest schedule, each kernel variant
 *    switched the other way where it changes the passes (kept when faster):
 *    the tile width of the strided first pass (complex64: also of the 2^11
 *    middle pass) doubled or not, the digit swap folded into the middle pass
 *    or not, the persistent prefetching pass kernels or not (these two
 *    complex128 only), the TMA-fed first and 2^11 middle passes or not
 *    (complex64 only);
 *  - n = M * 2^e, M > 1: every outer radix 2^a of the (2^a, M * 2^b, 2^a)
 *    schedule that efft_plan_create accepts, and one pass when n <= 2048;
 *    then, for the fastest, the first pass's tile width switched the other
 *    way where that changes the passes (kept when faster).
 * Each candidate is run on `scratch` (n*S bytes of the caller's device
 * memory on the plan's device; its contents are overwritten) on `stream`,
 * twice untimed and then a few times between CUDA events; its time is the
 * median.  Synchronous.  No execute of the plan may be in flight, and the
 * plan must not be used by another host thread meanwhile.
 *  cand_log2r  [out, may be NULL] room for cap*4 ints: candidate c's
 *              log2 radices at [4c, 4c+4), unused entries 0 (for M > 1 the
 *              power-of-two part of each radix).
 *  cand_ms     [out, may be NULL] room for cap doubles: candidate c's time.
 *  ncand       [out, may be NULL] number of candidates (may exceed cap).
 * For n <= 8 there is nothing to tune (*ncand = 1, the direct-sum kernel).
 * Errors: INVALID_PLAN, INVALID_PTR, MISALIGNED, LAUNCH, CUDA.
 */
int efft_plan_autotune(efft_plan_t plan, void* scratch, void* stream, int* cand_log2r, double* cand_ms,
                       int cap, int* ncand);

/* One candidate measured by efft_plan_autotune_candidates. */
typedef struct efft_candidate {
  int npasses;          /* p (0: the direct-sum kernel)                         */
  uint64_t radices[4];  /* R_0 .. R_{p-1} (whole: M included for N = M * 2^e)   */
  int wide;             /* 1: the wide strided tiles (see efft_plan_autotune)   */
  int fused_swap;       /* 1: digit swap folded into the middle pass            */
  int persistent;       /* 1: persistent prefetching pass kernels               */
  int tma;              /* 1: complex64 wide first and 2^11 middle passes fed   */
                        /*    by TMA copies                                     */
  double ms;            /* median time of one execute (milliseconds)            */
} efft_candidate;

/* efft_plan_autotune with the full record of every candidate:
 *  out    [out, may be NULL] room for cap records, in measuring order.
 *  ncand  [out, may be NULL] number of candidates (may exceed cap).
 * The plan ends on the fastest; efft_plan_autotune's other rules apply.
 * Errors: as efft_plan_autotune. */
int efft_plan_autotune_candidates(efft_plan_t plan, void* scratch, void* stream, efft_candidate* out, int cap,
                                  int* ncand);

/* The kernel variant a plan runs (each 0 or 1; see efft_candidate).  Any
 * pointer may be NULL.  Errors: INVALID_PLAN. */
int efft_plan_variant(efft_plan_t plan, int* wide, int* fused_swap, int* persistent, int* tma);

/* Switch a plan's kernel variant, keeping its schedule (e.g. to pin a choice
 * an earlier efft_plan_autotune_candidates measured).  Each knob: -1 the
 * built-in rule (by size), 0 off, 1 on wherever the pass shapes allow it
 * (efft_plan_variant reports what took effect).  Results are unchanged up to
 * rounding.  No execute of the plan may be in flight.
 * A real-data plan switches its complex plan.
 * Errors: INVALID_PLAN; INVALID_FLAGS for a knob outside -1..1;
 * UNSUPPORTED for a plan of N = M * 2^e (M > 1) with a knob other than
 * `wide` set (there `wide` is the tile width of the first pass when it runs
 * on the power-of-two kernels: 2^10 or 2^11 rows for complex128, 2^10 for
 * complex64). */
int efft_plan_set_variant(efft_plan_t plan, int wide, int fused_swap, int persistent, int tma);

/*
 * Synchronise `stream`, then report whether a kernel of one of the plan's
 * earlier executes gave up a bounded device wait: EFFT_ERR_TIMEOUT if so
 * (that execute's output is incomplete; the record is cleared), else EFFT_OK.
 * The only device waits in the library are those of the complex64 passes
 * fed by TMA copies (the `tma` variant: the wide first pass and the wide
 * 2^11 middle pass), which wait on an mbarrier in shared memory for their
 * copies and, when those do not complete within about 2^24 polls, record the
 * timeout in the execute's state word and return.
 * Errors: INVALID_PLAN, CUDA.
 */
int efft_execute_check(efft_plan_t plan, void* stream);

/* Destroy a plan and free its device tables, after waiting for the
 * executes still using its state words.  The paper's ~EFFT_Transform()
 * (Sec. 4, Listings 12-13); the caller's data buffers are not touched.  NULL is
 * accepted (no-op).
 * Errors: INVALID_PLAN for a handle that is not a live plan. */
int efft_plan_destroy(efft_plan_t plan);

/* Static, human-readable text for a status code (never NULL).  The paper has
 * no counterpart (its C++ interface reports no errors). */
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

/*
 * The schedule efft_plan_create chooses for (n, dtype) without the
 * autotuner, computed on the host with no CUDA call (no device needed):
 * the radices R_0..R_{p-1} (whole integers: for N = M * 2^e the middle or
 * only radix carries M) to radices (room for at most `cap` entries) and p to
 * *npasses; p = 0 for N <= 8 (one direct-sum kernel) and N = 1.
 * Errors: INVALID_PTR (npasses NULL), INVALID_SIZE, INVALID_DTYPE.
 */
int efft_plan_schedule(uint64_t n, int dtype, uint64_t* radices, int cap, int* npasses);
int efft_plan_info(efft_plan_t plan, double* hbm_passes, uint64_t* table_bytes);

/*
 * Per-kernel timing with CUDA events recorded on the execute's own stream
 * around every launch (measurement support; no effect on results).
 *  efft_plan_profile(plan, 1) starts recording for subsequent executes and
 *    clears earlier records; efft_plan_profile(plan, 0) stops recording.
 *  efft_plan_profile_read synchronises on the recorded events and writes, per
 *    launch slot s < cap, total milliseconds ms[s] and launch count count[s];
 *    *nslots receives EFFT_PROFILE_SLOTS.  Slots: 0 range scan (complex128),
 *    1 + j pass j (j < 4), 5 digit swap, 6 direct-sum kernel (N <= 8),
 *    7 mirrored-pair kernel of a real-data plan.
 *    Records are consumed by the read.
 * Profiling mutates the plan: do not profile a plan that other host threads
 * execute concurrently.
 */
#define EFFT_PROFILE_SLOTS 8
int efft_plan_profile(efft_plan_t plan, int enable);
int efft_plan_profile_read(efft_plan_t plan, double* ms, int* count, int cap, int* nslots);

/*
 * Real-data transforms: the paper's real-input form (Sec. 2.1, the packed
 * "perm" layout of Eq. 3) with its in-place pairing of mirrored elements
 * (Sec. 3.4).  The N reals are viewed as N/2 complex values
 * z[m] = x[2m] + i x[2m+1]; a complex plan of N/2 points transforms them and
 * one more in-place sweep combines each mirrored pair (k, N/2 - k), so that
 * a real transform costs about half a complex one of the same N.
 *  direction  EFFT_REAL_FORWARD: x[0..N) real in place -> the perm layout
 *               {R_0, R_{N/2}, R_1, I_1, ..., R_{N/2-1}, I_{N/2-1}} of
 *               F[k] = R_k + i I_k = sum_n x[n] exp(-2*pi*i*n*k/N), 0 <= k <= N/2
 *               (F[k] for k > N/2 is conj(F[N-k]));
 *             EFFT_REAL_INVERSE: a perm array in place ->
 *               x[n] = sum_{k<N} F[k] exp(+2*pi*i*n*k/N) over the Hermitian
 *               spectrum (F[N-k] = conj F[k]), a real result: N times the
 *               original data, or the original data with EFFT_FLAG_NORMALIZE.
 *  precision  EFFT_C64: float32 reals (4 bytes each); EFFT_C128: float64.
 *  n          number of reals, even, with n/2 a supported complex size
 *             (n = M * 2^e, M odd <= EFFT_MAX_ODD, e >= 1,
 *             2 <= n <= 2^(EFFT_MAX_LOG2N+1)).
 *  flags      EFFT_FLAG_NORMALIZE (multiply by 1/N; powers of two only, as
 *             for complex plans), EFFT_FLAG_AUTOTUNE (for the complex plan);
 *             EFFT_FLAG_DIGIT_REVERSED_OUT is rejected.
 * The plan is executed with efft_execute / efft_execute_host /
 * efft_execute_host_stream like a complex plan (data: n reals, aligned to
 * two reals); efft_plan_radices reports the complex plan's radices and
 * efft_plan_autotune tunes it; batches take complex plans only.
 * Errors: as efft_plan_create (INVALID_SIZE for n < 2, odd n or n/2 not a
 * supported size; UNSUPPORTED for EFFT_FLAG_NORMALIZE with M > 1),
 * INVALID_SIGN for another direction, INVALID_FLAGS.
 */
#define EFFT_REAL_FORWARD (-1)
#define EFFT_REAL_INVERSE (+1)
int efft_plan_create_real(efft_plan_t* out, uint64_t n, int precision, int direction, uint32_t flags);

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

/*
 * Batches: `count` independent in-place transforms of mixed sizes run by
 * one CUDA graph launch.  The paper's many sub-FFTs of one
 * split (Sec. 3.3), whose order is left to the Cilk scheduler, become one
 * user-level batch whose order is fixed once, at creation.
 *
 * efft_batch_create: transform i has sizes[i] points (a supported length
 *   of efft_plan_create: M * 2^e, M odd <= EFFT_MAX_ODD, at most
 *   2^EFFT_MAX_LOG2N); all share dtype, sign and flags
 *   (EFFT_FLAG_AUTOTUNE applies per distinct size).  Transforms of equal
 *   size share one plan and run in the same kernel launches (one grid row
 *   per transform); distinct sizes run as parallel branches of one CUDA
 *   graph that is captured here and replayed by every execute.  Allocates
 *   the plans' tables, a device array of `count` pointers, 16 bytes of
 *   device state per transform and pinned host staging for
 *   EFFT_BATCH_INFLIGHT * count pointers, then synchronises.
 *   Errors: INVALID_SIZE (count < 1, a bad size, more than 65535 transforms
 *   of one size), INVALID_PTR (sizes NULL), the plan errors, ALLOC, CUDA.
 * efft_batch_execute: data is a HOST array of `count` device pointers;
 *   data[i] is transform i's buffer with the rules of efft_execute.  The
 *   pointers are copied to pinned staging, then to the device on `stream`
 *   ahead of the graph launch, so `data` may be reused on return.
 *   Asynchronous.  Executes of one batch must be stream-ordered (they share
 *   the device pointer array and state); at most EFFT_BATCH_INFLIGHT of them
 *   are outstanding: the next one first waits on the host for the oldest.
 *   Errors: INVALID_PLAN (not a live batch), INVALID_PTR, MISALIGNED, LAUNCH.
 * efft_batch_execute_host_stream: host data through a chain of nbatches
 *   batches of the same sizes (in the same order, one device), applied in
 *   chain order (e.g. a forward batch, then an inverse one): transform i is
 *   copied from host_in[i] to the device buffer dev[i] (the rules of
 *   efft_execute; no two overlapping), transformed by every batch of the
 *   chain, and copied to host_out[i] (host_out[i] may equal host_in[i]).
 *   The transforms go group by group (largest size first) in chunks of
 *   about 256 MiB; the copies in, the launches and the copies out run on
 *   three streams ordered by events (the launches on `stream`), so the
 *   copies of one chunk overlap the transforms of the previous ones.  The
 *   host arrays should be pinned (cudaHostAlloc) for the copies to overlap.
 *   Synchronous: returns when every result is in host memory.  The graph
 *   is not used (the launches of each chunk are enqueued directly).
 *   Errors: INVALID_PLAN (a batch not live), INVALID_SIZE (nbatches < 1 or
 *   batches of different sizes, dtype or device), INVALID_PTR / MISALIGNED
 *   (host or device pointers), LAUNCH, CUDA.
 * efft_batch_info: *ngroups = number of distinct sizes; *kernels = kernel
 *   nodes in the graph (kernel launches per execute).  Either may be NULL.
 * efft_batch_destroy: waits for the batch's outstanding executes, then
 *   frees everything.  NULL is a no-op; INVALID_PLAN for a foreign handle.
 */
#define EFFT_BATCH_INFLIGHT 4
typedef struct efft_batch_s* efft_batch_t;
int efft_batch_create(efft_batch_t* out, const uint64_t* sizes, int count, int dtype, int sign,
                      uint32_t flags);
int efft_batch_execute(efft_batch_t batch, void* const* data, void* stream);
int efft_batch_execute_host_stream(const efft_batch_t* batches, int nbatches, void* const* host_in,
                                   void* const* host_out, void* const* dev, void* stream);
int efft_batch_info(efft_batch_t batch, int* ngroups, int* kernels);
int efft_batch_destroy(efft_batch_t batch);

#ifdef __cplusplus
}
#endif
#endif /* EFFT_H */
