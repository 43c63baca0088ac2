/*
 * bplg.h -- C ABI of the GB300 batched parallel-prefix library.
 *
 * The library computes three families of batched parallel-prefix operations
 * (Section III of "Performance Tuning for GPU-Embedded Systems: Machine-
 * Learning-based and Analytical Model-driven Tuning Methodologies", Dieguez
 * and Amor, 2023) with hand-written sm_103a CUDA kernels, and the two tuning
 * methodologies of Section IV that choose their performance parameters:
 *
 *   scan     inclusive sum scan, int32 (wrap-around) and float32
 *   FFT      complex Stockham FFT of power-of-two length, radix 2/4/8/16
 *   tridiag  cyclic reduction + parallel cyclic reduction (CR/PCR) hybrid,
 *            and the same solver wrapped in float64-residual refinement
 *   tuning   analytical guideline (Section IV-A), Bayesian optimisation with a
 *            Gaussian-process cost model (Section IV-B), exhaustive search and
 *            the Phi metric (Section VI)
 *
 * Conventions for every entry point
 *   - Return value: BPLG_OK (0) or a negative BPLG_ERR_* code; the message of
 *     the last error on the calling thread is returned by bplg_last_error().
 *   - Memory: the caller owns every buffer and every stream.  "device" buffers
 *     are CUDA global memory of the current device; "host" buffers are CPU
 *     memory.  Compute entry points never allocate on their hot path; the
 *     first FFT call on a device allocates the shared twiddle table (256 KB)
 *     once, synchronously, so it must not be the first call inside a stream
 *     capture.  The library keeps such per-device state (tables, scratch,
 *     kernel attributes) for the life of the process: do not use it on a
 *     device after cudaDeviceReset of that device.
 *   - Grid: a call whose batch would need more than 2^31 - 1 blocks under its
 *     plan (problems per block) returns BPLG_ERR_UNSUPPORTED_SIZE before
 *     anything is enqueued.
 *   - Layout: batched data is row-major [batch][n], problem after problem,
 *     with no padding between problems.  Device pointers must be 16-byte
 *     aligned.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Compute entry points are asynchronous on it; argument
 *     errors are reported before anything is enqueued.
 *   - Plans: a NULL plan means "the plan bplg_query_plan returns" (with
 *     online tuning on, a candidate of the online search instead; see
 *     bplg_set_online_tuning).  A non-NULL plan is validated against the size
 *     and the device; an unusable plan returns BPLG_ERR_INVALID_PLAN without
 *     launching.
 */
#ifndef BPLG_H
#define BPLG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ error codes */
#define BPLG_OK 0
#define BPLG_ERR_INVALID_ARG (-1)      /* null pointer, n/batch out of range, misaligned pointer */
#define BPLG_ERR_UNSUPPORTED_SIZE (-2) /* n not a power of two or above the kernel's maximum */
#define BPLG_ERR_INVALID_PLAN (-3)     /* plan does not fit the size or the device limits */
#define BPLG_ERR_CUDA (-4)             /* a CUDA runtime call failed; see bplg_last_error() */
#define BPLG_ERR_TIMEOUT (-5)          /* a tuning candidate exceeded its wall-clock limit */
#define BPLG_ERR_DEVICE_FLAG (-6)      /* a kernel reported a device-side failure */
#define BPLG_ERR_NO_DEVICE (-7)        /* no CUDA device is visible */

/* ----------------------------------------------------------------- enums */
typedef enum { BPLG_I32 = 0, BPLG_F32 = 1 } bplg_dtype;

typedef enum {
    BPLG_OP_SCAN = 0,            /* Section III, scan primitive */
    BPLG_OP_FFT = 1,             /* Section III, Stockham FFT */
    BPLG_OP_TRIDIAG = 2,         /* Section III, tridiagonal solver (CR/PCR hybrid) */
    BPLG_OP_TRIDIAG_REFINED = 3, /* the solver inside float64-residual refinement */
    BPLG_OP_FFT_TC = 4,          /* FFT whose radix-16 stages run on tensor cores */
    BPLG_OP_TRIDIAG_WM = 5       /* Section III, tridiagonal solver of Wang and Mou (divide and conquer) */
} bplg_op;

typedef enum { BPLG_PATTERN_KS = 0, BPLG_PATTERN_LF = 1 } bplg_scan_pattern;
typedef enum {
    BPLG_TUNE_ANALYTIC = 0,   /* Section IV-A guideline, as the paper states it (Maxwell-era thresholds) */
    BPLG_TUNE_LEARNED = 1,    /* Section IV-B Bayesian optimisation over timed candidates */
    BPLG_TUNE_EXHAUSTIVE = 2, /* every valid plan timed (Section VI's reference) */
    BPLG_TUNE_MODEL = 3       /* Section IV-A premises restated as a GB300 cost model; no evaluation */
} bplg_tune_method;
typedef enum { BPLG_TC_BF16 = 0, BPLG_TC_F16 = 1 } bplg_tc_precision;

/* --------------------------------------------------------------- the plan
 * The performance parameters B of Section IV-B ("Table I"): the (S, P, L)
 * tuple of Section IV-A plus the radix, the shuffle switch and the layout
 * knobs.  A plain value: copy it, store it, compare it with memcmp.
 *
 *   P       elements per thread.  For the FFT P equals the radix r.
 *   L       threads per block = spb * (n / P).
 *   spb     problems (signals or systems) per block.
 *   S       shared-memory elements per block (derived, reported).
 *   radix   FFT radix r in {2,4,8,16}; Wang-Mou tridiag: runs merged per
 *           stage, r in {2,4,8} (r <= n / P unless n = P); 2 for scan and
 *           the CR/PCR tridiag.
 *   shuffle tridiag: the PCR phase runs in one warp with shuffles (cr_switch
 *           <= 32); Wang-Mou: merge stages whose groups fit in a warp
 *           exchange by shuffles (else every stage goes through shared
 *           memory); scan: always 1 (warp-shuffle prefix stages).
 *   pattern scan: prefix circuit of the shuffle stages, BPLG_PATTERN_KS or
 *           BPLG_PATTERN_LF (Fig. 1(f) / 1(d)).
 *   smem_layout FFT: 0 interleaved complex, 1 real and imaginary parts
 *           exchanged in turn through one float buffer (Section V-C).
 *           Tridiag: 0 all CR levels in place in shared memory, 1 one
 *           shared-memory array per CR level (stride-free), 2 the first
 *           log2 P CR levels in registers, the rest in shared memory.
 *           Refined tridiag: 0-3: shared-memory solver, bit 0 coefficients
 *           also cached as float64, bit 1 one array per CR level; 4 every
 *           equation in registers (register-level CR), 5 the same with the
 *           coefficients held as float64 registers and their float32
 *           copies in shared memory (P <= 8), 6 the same with the float32
 *           coefficients in shared memory only (fewer registers per thread),
 *           7 as 6 with the float32 solves done by the Wang-Mou divide and
 *           conquer (radix 2; shuffle 1, smem_pad 0, cr_switch 32).
 *   smem_pad 1: pad shared-memory rows against bank conflicts.
 *   io      FFT: 0 registers <-> global memory directly, 1 staged through
 *           shared memory with 16-byte accesses, 2 persistent blocks fed by
 *           a ring of bulk asynchronous copies (TMA).  Tridiag: 0 one tile
 *           per block, 1 persistent blocks fed by bulk asynchronous copies.
 *   cr_switch tridiag: system size m at which cyclic reduction hands over to
 *           parallel cyclic reduction (1 = pure CR, n = pure PCR).
 *   n1_log  FFT with n > 16384, computed in two kernels (the multi-kernel
 *           transform of Section V-C for signals that do not fit one
 *           block): n = N1 N2 with N1 = 2^n1_log.  The first kernel runs the
 *           N1-point transforms of the columns of the N1 x N2 row-major
 *           signal, spb adjacent columns per block, and multiplies by
 *           exp(dir 2 pi i k1 n2 / n); the second runs the N2-point
 *           transforms of the rows, row_spb rows per block, and writes the
 *           result in natural order.  Both use radix 16 (P = radix = 16,
 *           padded interleaved exchanges, io 0) and L = spb * N1 / 16.
 *           0 for every other plan.
 *   row_spb FFT with n > 16384: rows per block of the second kernel
 *           (spb and row_spb are powers of two up to 64, with 32 to 1024
 *           threads and at most 227 KB of shared memory per block).
 *   reserved 0.
 */
typedef struct {
    int32_t op;
    int32_t n;
    int32_t P;
    int32_t L;
    int32_t spb;
    int32_t S;
    int32_t radix;
    int32_t shuffle;
    int32_t pattern;
    int32_t smem_layout;
    int32_t smem_pad;
    int32_t io;
    int32_t cr_switch;
    int32_t n1_log;
    int32_t row_spb;
    int32_t reserved;
} bplg_plan;

/* -------------------------------------------------------- compute calls */

/* Batched inclusive sum scan (Section III, "Scan Operator"): for every
 * problem s, out[s][i] = in[s][0] + ... + in[s][i].
 *   dtype  BPLG_I32 (two's-complement wrap-around, bit-exact) or BPLG_F32.
 *   in,out device, [batch][n] of dtype; in == out (in place) is allowed.
 *   n      1 <= n <= 32768; batch >= 1.  A power of two runs its own plan;
 *          any other n runs the plan of the next power of two n' (plan->n ==
 *          n', or plan NULL), the rows read as if padded with zeros to n'
 *          (element-wise accesses; rows stay n apart, nothing past n is
 *          written).
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, INVALID_PLAN, CUDA. */
int bplg_scan_batched(int32_t dtype, const void *in, void *out, int64_t n, int64_t batch,
                      const bplg_plan *plan, void *stream);

/* Batched complex FFT by the Stockham self-sorting algorithm (Section III,
 * "Fast Fourier Transform", Fig. 1(c)): X[k] = sum_j x[j] exp(dir*2*pi*i*j*k/n)
 * with dir = -1 (forward) or +1 (inverse, unnormalised), natural order.
 *   in,out device, [batch][n] complex64 as interleaved (re, im) float pairs;
 *          in == out is allowed.
 *   n      2 <= n <= 2^24 (at most 2^23 when n is not a power of two);
 *          batch >= 1.  Above 16384 points the transform runs as two kernels
 *          (see n1_log in the plan) through a scratch buffer of n * batch
 *          complex values that the library allocates on first use per device
 *          and stream and grows when needed (a growth waits for the stream);
 *          in may equal out.
 *          A length n = 2^a 3^b 5^c up to 12288 that is not a power of two
 *          (and no plan) runs a mixed-radix Stockham kernel compiled for
 *          that length: stages of radix 2, 3, 4, 5, 6, 8, 9, 10, 12, 15 or
 *          16, the block's signals in shared memory, the stage twiddles
 *          from a per-n table W_n^e made on the first call with that n
 *          (float64 on the host, rounded to float32, uploaded
 *          synchronously).
 *          Any other length that is not a power of two runs Bluestein's
 *          chirp identity: X_k = h_k sum_j (x_j h_j) conj(h_{k-j}) with
 *          h_m = exp(dir pi i m^2 / n), a cyclic convolution of length
 *          M = next power of two >= 2n - 1.  With no plan and 32 <= M <=
 *          8192 it is one fused kernel; otherwise (or with a plan, which
 *          must be made for M) two M-point FFTs and three elementwise
 *          kernels through a scratch of M * batch complex values per device
 *          and stream.  The chirp and the transformed chirp are per-(n, dir)
 *          tables made like the mixed-radix table.
 * Twiddles W_M^k are generated once per device in float64 and rounded to
 * float32.  Errors: INVALID_ARG, UNSUPPORTED_SIZE, INVALID_PLAN, CUDA. */
int bplg_fft_batched(const void *in, void *out, int64_t n, int64_t batch, int32_t dir,
                     const bplg_plan *plan, void *stream);

/* The same FFT with its DFT stages run on tensor cores as real contractions
 * on 16-bit operands split into hi and lo parts, x = xh + xl and
 * F = Fh + Fl, summing xh Fh + xh Fl + xl Fh in float32.
 *   io 0 (n >= 1024): every radix-16 stage; each 16-point DFT is a 32 x 32
 *        contraction issued as tcgen05.mma with the accumulator in tensor
 *        memory; a mixed-radix first stage (log2 n not a multiple of 4)
 *        runs on the CUDA cores.
 *   io 1: the same stages in the legacy mma.sync m16n8k16 form.
 *   io 2 (n = 4096: P 16, spb 2; n = 16384: P 32, spb 1; 512 threads):
 *        two passes of 64-point DFTs (the 64 x 64 four-step form; 16384
 *        points after a radix-4 stage on the CUDA cores), each pass one
 *        chain of K = 128 products with the 128 x 128 DFT matrix held in
 *        tensor memory, in a persistent kernel that loads the next tile
 *        while the current one runs.
 * Twiddles are applied in float32 from the float64-generated table.  Not in
 * the paper (whose FFT is float32 on CUDA cores, Section III); the error
 * against the float64 oracle is reported per size.
 *   precision BPLG_TC_BF16 or BPLG_TC_F16 (FP16 scales each stage by 1/4,
 *             exactly, and undoes it at the end).
 *   n        power of two, 512 <= n <= 16384; in, out as bplg_fft_batched.
 *   plan     op BPLG_OP_FFT_TC (radix 16; P, spb, io as above), or NULL
 *            (the GB300 cost model's choice).
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, INVALID_PLAN, CUDA. */
int bplg_fft_tc_batched(const void *in, void *out, int64_t n, int64_t batch, int32_t dir,
                        int32_t precision, const bplg_plan *plan, void *stream);

/* The FFT of bplg_fft_batched for callers that cannot allocate device
 * memory while they run -- code under an allocator that owns the whole
 * device, fixed real-time memory budgets, code that must not trigger the
 * device synchronisation an allocation can cause.  The paper has no
 * counterpart: this is a property of the library, not of the method.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine: its twiddle
 * table is a file-scope device array of 64 KB that every GPU loading the
 * library holds until the process exits, so it accepts only n <= 4096 (larger
 * n returns BPLG_ERR_UNSUPPORTED_SIZE with a message).  On success nothing is
 * allocated; on failure the error message string may be.
 *   in,out  device, [batch][n] complex64 interleaved; in == out is allowed.
 *   dir     -1 forward, +1 inverse (unnormalised).
 *   plan    a valid FFT plan with io 0 or 1, or NULL for a fixed default
 *           (radix min(16, n), at least 128 threads per block).  A plan whose
 *           shared memory exceeds the device's per-block limit returns
 *           BPLG_ERR_INVALID_PLAN.
 * Set-up: the table's values are a static initializer of the array (made at
 * build time in float64 and rounded once to float32), so they are in place
 * as soon as the library's code is loaded on a device; nothing is launched
 * or waited for.  The first call on each device, with that device current,
 * looks up the array's device address (cudaGetSymbolAddress), which can load
 * the library's code on that device; make that first call before any stream
 * capture.  All calls share the array, which is only ever read, so nothing in
 * it has to start at zero and calls that overlap each other on the GPU read
 * it concurrently without harm.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, INVALID_PLAN, CUDA. */
int bplg_fft_batched_noalloc(const void *in, void *out, int64_t n, int64_t batch, int32_t dir,
                             const bplg_plan *plan, void *stream);

/* Batched tridiagonal solve (Section III, "Tridiagonal system solvers"):
 * a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i for every system.  The plan's op
 * picks the solver:
 *   BPLG_OP_TRIDIAG (and plan NULL): cyclic reduction down to
 *           plan->cr_switch equations, parallel cyclic reduction on those,
 *           and CR back substitution; all in float32.
 *   BPLG_OP_TRIDIAG_WM: the divide-and-conquer method of Wang and Mou (the
 *           WM pattern of Fig. 1(e)): each thread solves its P equations for
 *           their two outer neighbours (one Thomas sweep, three right-hand
 *           sides), then merge stages of radix plan->radix join adjacent
 *           runs until one run covers the system; float32.
 *   a,b,c,d device, float32 [batch][n] each (structure of arrays);
 *           a[s][0] and c[s][n-1] are never read.
 *   x       device, float32 [batch][n]; may alias d.
 *   n       2 <= n <= 8192; batch >= 1.  Any n that is not a power of two
 *           runs the Wang-Mou solver with the plan of the next power of two
 *           n' (a BPLG_OP_TRIDIAG_WM plan with plan->n == n', or NULL): the
 *           system is padded with identity rows (a = c = 0, b = 1, d = 0),
 *           c[s][n-1] is taken as 0, rows stay n apart and nothing past n is
 *           read or written (element-wise accesses).
 * No pivoting: the systems must be safe for elimination without pivoting
 * (e.g. strictly diagonally dominant).  Pivots are inverted with the fast
 * float32 reciprocal (__fdividef(1, x)), which gives 0 for |x| > 2^126, so
 * every pivot's magnitude must stay below 2^126 (systems scaled by 2^100
 * and 2^-100 are tested).  Errors: as for the scan. */
int bplg_tridiag_batched(const float *a, const float *b, const float *c, const float *d, float *x,
                         int64_t n, int64_t batch, const bplg_plan *plan, void *stream);

/* The same solver inside iterative refinement: x0 = solve32(d); then
 * r = d - A x_k in float64 from the stored float32 coefficients, a float32
 * solve of the power-of-two-scaled residual, and x_{k+1} = x_k + e in
 * float64.  A system stops when the correction just applied has
 * max|e| <= tol * max|x0|, or, before another solve, when its residual
 * bounds the error: for strictly diagonally dominant rows
 * max|r| / min_i(|b_i| - |a_i| - |c_i|) <= tol * max|x0|; and after at most
 * max_iter corrections.  The stopping tests are evaluated in float32 on
 * the float32 maxima with a 1e-5 relative safety margin, against tol rounded
 * toward zero; a test whose right-hand side falls below 2^-100 never stops a
 * system (it then runs max_iter corrections).  The residual's float32 copy
 * for the correction solve flushes magnitudes below 2^-126 to zero.
 *   x       device, float64 [batch][n] (must not alias the inputs).
 *   iters   device int32 [batch] (corrections applied per system) or NULL.
 *   n       power of two, 2 <= n <= 4096.
 *   max_iter 0..64; tol >= 0.
 * Errors: as for bplg_tridiag_batched. */
int bplg_tridiag_refined(const float *a, const float *b, const float *c, const float *d, double *x,
                         int64_t n, int64_t batch, int32_t max_iter, double tol, int32_t *iters,
                         const bplg_plan *plan, void *stream);

/* ------------------------------------------------ uneven-size batches */

/* One problem of an uneven batch (the uniform batches of Section IV-A
 * generalised to mixed operations and sizes); every problem has its own
 * device buffers, 16-byte aligned, laid out as in the batched calls. */
typedef struct {
    int32_t op;        /* BPLG_OP_SCAN, BPLG_OP_FFT or BPLG_OP_TRIDIAG */
    int32_t n;         /* power of two, 32 <= n <= 8192 */
    int32_t dtype;     /* scan: BPLG_I32 or BPLG_F32 */
    int32_t dir;       /* FFT: -1 forward, +1 inverse (unnormalised) */
    const void *in[4]; /* scan, FFT: in[0]; tridiag: a, b, c, d (float32) */
    void *out;         /* scan, FFT: output (may equal in[0]); tridiag: x (may alias d) */
} bplg_item;

typedef struct bplg_uneven_batch *bplg_uneven_handle;

/* Prepare an uneven batch on the current device: validate the items, group
 * them by (operation, size) into units (largest first), copy the descriptors
 * to library-owned device memory, and capture into a CUDA graph one counter
 * reset plus three persistent kernels (scan, radix-16 Stockham FFT, and the
 * Wang-Mou tridiagonal solver) that pull units from an atomic counter each.  The item buffers must stay valid while the
 * handle is used.  Synchronous; allocates.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, CUDA. */
int bplg_uneven_create(const bplg_item *items, int64_t count, bplg_uneven_handle *out);

/* Run every problem of the batch: one graph launch on `stream`.  Launches of
 * the same handle share its work counters, so they must not overlap on the
 * GPU (launches on one stream never do).  Errors: INVALID_ARG, CUDA. */
int bplg_uneven_launch(bplg_uneven_handle h, void *stream);

/* Units per operation (scan, FFT, tridiag) of a prepared batch. */
int bplg_uneven_units(bplg_uneven_handle h, int32_t *units_scan_fft_tridiag);

/* Release the handle (graph and device descriptors).  Call after its last
 * launch has completed. */
int bplg_uneven_destroy(bplg_uneven_handle h);

/* ------------------------------------------------------------- tuning */

/* Per-SM limits that bound occupancy (Section IV-A: W^max, B^max, registers
 * and shared memory). */
typedef struct {
    int32_t max_warps_per_sm;
    int32_t max_blocks_per_sm;
    int32_t regs_per_sm;
    int32_t reg_alloc_unit;
    int32_t warp_alloc_granularity;
    int32_t max_regs_per_thread;
    int32_t smem_per_sm;
    int32_t smem_alloc_unit;
    int32_t max_smem_per_block;
    int32_t smem_reserved_per_block;
    int32_t max_threads_per_block;
    int32_t num_sms;
} bplg_arch;

/* Fill *out with the limits of device `device` (cudaGetDeviceProperties).
 * Errors: NO_DEVICE, CUDA, INVALID_ARG. */
int bplg_arch_query(int32_t device, bplg_arch *out);

/* Fill *out with a built-in preset: 0 = GM20B (Jetson TX1, Section II),
 * 1 = GB300.  Errors: INVALID_ARG. */
int bplg_arch_preset(int32_t which, bplg_arch *out);

/* Occupancy of one block shape (Section IV-A): active warps W_SM and active
 * blocks B_a per SM; both 0 when the shape cannot launch.  Host only. */
int bplg_occupancy(const bplg_arch *arch, int32_t warps_per_block, int32_t regs_per_thread,
                   int32_t smem_per_block, int32_t *w_sm, int32_t *b_a);

/* One configuration as the analytical guideline sees it. */
typedef struct {
    int32_t S, P, L, regs, smem, radix, shuffle, reserved;
} bplg_candidate;

/* The analytical guideline of Section IV-A (the four bullets, with the
 * shuffle premise (i) and the radix bullet) applied to an explicit candidate
 * list; *chosen is the index of the picked candidate, or -1 if none can
 * launch.  Host only.  Errors: INVALID_ARG. */
int bplg_guideline_select(const bplg_arch *arch, const bplg_candidate *cands, int32_t count,
                          int32_t radix_tunable, int32_t *chosen);

/* Phi(a, C) = |C| / sum_i 1/e_i (Section VI).  Returns 0 for an empty list
 * or any e_i <= 0. */
double bplg_phi(const double *efficiencies, int32_t count);

/* All valid plans for (op, dtype, n) on the current device, in the library's
 * canonical order (written up to `capacity`; *count gets the total).
 * Validity uses the device limits and each kernel's register count from
 * cudaFuncGetAttributes.  Errors: INVALID_ARG, UNSUPPORTED_SIZE, CUDA. */
int bplg_enumerate_plans(int32_t op, int32_t dtype, int64_t n, bplg_plan *out, int32_t capacity,
                         int32_t *count);

/* Resources of one plan on the current device: registers per thread, dynamic
 * + static shared memory per block, threads per block.
 * Errors: INVALID_PLAN, CUDA. */
int bplg_plan_resources(const bplg_plan *plan, int32_t dtype, int32_t *regs, int32_t *smem,
                        int32_t *threads);

/* Cost of one candidate in milliseconds for a caller-supplied objective;
 * return a negative value or INFINITY for an invalid candidate. */
typedef double (*bplg_cost_fn)(const bplg_plan *plan, void *user);

typedef struct {
    int32_t method;        /* bplg_tune_method used */
    int32_t space_size;    /* valid plans in the search space */
    int32_t evaluations;   /* candidate evaluations performed */
    int32_t invalid;       /* evaluations that returned an invalid cost */
    double chosen_ms;      /* cost of the returned plan (NaN if never evaluated) */
    double best_seen_ms;   /* best cost among the evaluated candidates */
} bplg_tune_report;

/* The tuning problem of Section IV-B: argmin over the plans x_B of f(a_j, x_B)
 * with a_j = (op, dtype, n, batch), where f is the median time of timed
 * launches on the current device on library-owned buffers of that shape.
 *   ANALYTIC    the guideline of Section IV-A on the device limits, as the
 *               paper states it (its occupancy thresholds were set for a
 *               Maxwell SM); no GPU evaluation.
 *   MODEL       the premises of Section IV-A (coalescing, occupancy, ILP and
 *               radix, kernel count) restated as a cost estimate for this GPU:
 *               per plan, from the kernel's real register and shared-memory
 *               counts and the device's SM count, clock and HBM bandwidth,
 *               the soft maximum of the HBM time, the latency time (Little's
 *               law: resident blocks each living one HBM round trip plus its
 *               own transfer and compute), the issue time (instructions per
 *               element of the op's algorithm), the load/store-unit time (128-
 *               byte lines per warp-wide access), the block-launch time and,
 *               for the refined solve, the FP64-pipe time; the plan with the
 *               least estimate wins.  No GPU evaluation.
 *   LEARNED     Bayesian optimisation: a seeded space-filling initial
 *               design, a Gaussian-process surrogate (Matern-5/2 on the
 *               encoded knobs, on log time), expected improvement, stop after
 *               a window of 8 evaluations without improvement (environment
 *               variable BPLG_BO_WINDOW = 1..64 overrides it; 5 is the
 *               paper's) or at `budget` evaluations (0 = 40).
 *   EXHAUSTIVE  every valid plan is timed.
 * The result is stored in the per-process plan cache that bplg_query_plan
 * reads.  Synchronous.  Errors: INVALID_ARG, UNSUPPORTED_SIZE, CUDA, NO_DEVICE. */
int bplg_tune_plan(int32_t op, int32_t dtype, int64_t n, int64_t batch, int32_t method,
                   int32_t budget, uint64_t seed, bplg_plan *out, bplg_tune_report *report);

/* The same search over an explicit plan list with a caller objective (host
 * only; used to test the search strategies without a GPU).  `arch` and
 * `regs` (per-plan register counts, may be NULL = 32) and `smem` feed the
 * analytical methods; MODEL takes the problem size from plans[0].n, a batch
 * of 2^24 / n problems and the preset GB300 clock (2.07 GHz) and HBM rate
 * (8.18 TB/s nominal).  Errors: INVALID_ARG. */
int bplg_tune_plans_cost(const bplg_plan *plans, int32_t count, const int32_t *regs,
                         const int32_t *smem, const bplg_arch *arch, int32_t method, int32_t budget,
                         uint64_t seed, bplg_cost_fn cost, void *user, int32_t *chosen,
                         bplg_tune_report *report);

/* The plan for (op, dtype, n, batch) without any GPU evaluation ("online"
 * tuning, Section IV): the plan cached by an earlier bplg_tune_plan, else the
 * plan of the GB300 cost model (BPLG_TUNE_MODEL) on the current device.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, CUDA, NO_DEVICE. */
int bplg_query_plan(int32_t op, int32_t dtype, int64_t n, int64_t batch, bplg_plan *out);

/* Online tuning: the learned search of Section IV-B spread over the
 * library's own calls (the paper tunes once, up front; this amortises the
 * evaluations over repeated calls).  With it on, a compute call that passes
 * no plan and finds no tuned plan in the cache runs the next candidate of a
 * search kept per (device, op, dtype, n, batch class), timed by two CUDA
 * events recorded around its launch on the caller's stream.  A later call
 * of the same shape reads that time without waiting; while a measurement is
 * still in flight, or after the search has finished, calls run the best plan
 * seen so far.  When the search stops (its stopping window or `budget`
 * evaluations), the best plan enters the plan cache, where bplg_query_plan
 * and every later call find it.  Results are exact throughout (every
 * candidate is a valid plan); only speed varies while the search runs.
 *   enable  1 on, 0 off (the searches in progress are kept).
 *   budget  evaluations per shape (0 = 40); seed: the search's seed.
 * Errors: INVALID_ARG. */
int bplg_set_online_tuning(int32_t enable, int32_t budget, uint64_t seed);

/* Progress of the online search for one shape: evaluations so far, whether
 * it has finished, and its best plan so far (zeroed when none).
 * Errors: INVALID_ARG, CUDA. */
int bplg_online_status(int32_t op, int32_t dtype, int64_t n, int64_t batch, int32_t *evaluations,
                       int32_t *finished, bplg_plan *best);

/* Median time in milliseconds of `reps` launches of `plan` (after two
 * warm-up launches) on library-owned buffers of shape (dtype, n, batch),
 * each launch bracketed by CUDA events: the objective f(a_j, x_B) the tuners
 * minimise.  Allocates and frees its buffers; synchronous.
 * Errors: INVALID_ARG, INVALID_PLAN, CUDA. */
int bplg_time_plan(const bplg_plan *plan, int32_t dtype, int64_t n, int64_t batch, int32_t reps,
                   double *median_ms);

/* Validate `plan` for (op, dtype, n) on the current device.
 * Returns BPLG_OK or BPLG_ERR_INVALID_PLAN (reason in bplg_last_error()). */
int bplg_check_plan(const bplg_plan *plan, int32_t dtype, int64_t n);

/* Device-side status of the current device: *flag receives 0, or the
 * nonzero code a pipelined kernel recorded when one of its bounded waits on
 * an asynchronous copy ran out (it then returned early, leaving its outputs
 * incomplete).  reset != 0 clears the word.  Synchronous.
 * Errors: INVALID_ARG, CUDA, NO_DEVICE. */
int bplg_device_status(int32_t *flag, int32_t reset);

/* Message of the last error on the calling thread ("" if none). */
const char *bplg_last_error(void);

/* ABI version (major * 100 + minor). */
int32_t bplg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BPLG_H */
