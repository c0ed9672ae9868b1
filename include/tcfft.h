/*
 * tcfft -- batched 1D and 2D complex-to-complex FP16 FFTs on GB300 (sm_103a)
 * tensor cores.  C ABI of the library libtcfft.so.
 *
 * Method: arXiv 2104.11471 ("tcFFT: Accelerating Half-Precision FFT through
 * Tensor Cores").  Every radix-16 merging process of the Cooley-Tukey
 * recursion, Eq. (dft_mm) of Sec. 2.1, X_out = F_16 . (T (.) X_in), runs as a
 * dense matrix multiply on the 5th-generation tensor cores; radix 2/4/8 steps
 * run on CUDA cores (Sec. 3.1); the plan / execution-function split follows
 * Sec. 3.1 ("Architecture", Fig. 1).
 *
 * Conventions shared by every call:
 *  - Transform: forward, X[k] = sum_n x[n] exp(-2 pi i n k / N), sign -,
 *    no normalisation (Eq. dft_def, Sec. 2.1), unless the plan flags ask for
 *    the inverse and/or 1/N scaling.  Output in natural order.
 *  - Data: interleaved complex FP16 (re, im), 4 bytes per point.  1D
 *    transform b starts at element b*n; 2D data is [batch][nx][ny], row-major
 *    with ny contiguous (the tcfftPlan2D statement in Sec. 3.1).
 *  - Split precision (TCFFT_FP16_SPLIT): one buffer holding two planes laid
 *    out like the plain data, plane 0 = hi, plane 1 = lo; the value is
 *    hi + lo * 2^-11.  A caller with plain FP16 input passes lo = 0.
 *  - TCFFT_FP32: interleaved FP32 complex (re, im), 8 bytes per point, in the
 *    same element order as the plain data.
 *  - Device pointers must be 16-byte aligned.  in == out (in place) is
 *    allowed; otherwise in is never written.
 *  - Sizes: n, nx, ny powers of two with 16 <= n <= 2^27 (1D; 2^24 in a
 *    ragged plan) and 16 <= nx, ny <= 8192 (2D, nx != ny allowed); batch >= 1.
 *    Anything else returns TCFFT_ERR_INVALID_SIZE.
 *  - Errors: every call returns a status code and never aborts.  tcfft_exec
 *    is asynchronous on the given stream; a device-side failure (a bounded
 *    wait that expired) is recorded in a plan-owned status word read by
 *    tcfft_plan_last_error after the stream has been synchronised.
 *  - Threading: a plan owns scratch memory; do not run two tcfft_exec calls
 *    on one plan concurrently.  Create one plan per stream.
 */
#ifndef TCFFT_H_
#define TCFFT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tcfft_plan_s* tcfft_plan;

typedef enum {
  TCFFT_OK = 0,
  TCFFT_ERR_INVALID_SIZE = 1,     /* unsupported n, nx, ny or batch */
  TCFFT_ERR_INVALID_VALUE = 2,    /* null or misaligned pointer, bad enum */
  TCFFT_ERR_ALLOC = 3,            /* device or host allocation failed */
  TCFFT_ERR_LAUNCH = 4,           /* kernel launch failed */
  TCFFT_ERR_TIMEOUT = 5,          /* a device-side bounded wait expired */
  TCFFT_ERR_UNSUPPORTED = 6,      /* no sm_103a device, or feature not built */
  TCFFT_ERR_NOT_IMPLEMENTED = 7,
  TCFFT_ERR_CUDA = 8              /* other CUDA runtime error */
} tcfft_status;

typedef enum {
  TCFFT_FP16 = 0,       /* FP16 storage and operands, FP32 accumulation */
  TCFFT_FP16_SPLIT = 1, /* hi + 2^-11 lo pairs, three MMA products per stage */
  TCFFT_FP32 = 2        /* interleaved FP32 complex in and out (8 B per point):
                           each value is split into hi + 2^-11 lo FP16 on load,
                           the stages run as TCFFT_FP16_SPLIT (FP16 operands,
                           three products, FP32 accumulation) and the FP32
                           accumulator is stored as is.  About 22 significant
                           bits; input values and intermediates must stay
                           within FP16 range (|x| < 65504, as in the other
                           precisions) */
} tcfft_precision;

/* Plan flags (tcfft_plan_*_ex, tcfft_plan_many): */
#define TCFFT_PLAN_AUTOTUNE 1u /* time candidate CTA geometries per pass at plan
                                  time (points per CTA, 128 or 256 threads,
                                  prefetching or synchronous loads; ragged
                                  groups: points only); picks are cached in
                                  TCFFT_TUNE_CACHE (default
                                  $HOME/.cache/tcfft_tune.txt) */
#define TCFFT_PLAN_GRAPH 2u    /* tcfft_exec replays one instantiated CUDA graph
                                  per (in, out) pair (captured on first use) */
#define TCFFT_PLAN_INVERSE 4u  /* inverse transform: sign +, X[k] = sum_n x[n]
                                  exp(+2 pi i n k / N), unnormalised */
#define TCFFT_PLAN_SCALE 8u    /* multiply the results by 1/N (N = points of one
                                  transform); with TCFFT_PLAN_INVERSE the exact
                                  inverse of the forward transform */
#define TCFFT_PLAN_SHARE_SM 16u /* use at most half of each SM's CTA slots, so
                                  that kernels on other (higher-priority)
                                  streams find room while this plan runs
                                  (serving: large jobs beside small ones) */
#define TCFFT_PLAN_FUSED_2D 32u /* square 2D transforms up to 512 x 512 (256 x
                                  256 split; ragged groups too): rows and
                                  columns in one launch, a cluster of up to 16
                                  CTAs per matrix exchanging the row results
                                  through distributed shared memory, one HBM
                                  read and one write per matrix (Sec. 3.1, 2D
                                  FFT).  Off by default: on GB300 the stage
                                  kernels are bound by on-chip work, not HBM,
                                  and the two-pass plan is faster; with
                                  TCFFT_PLAN_AUTOTUNE the faster of the two is
                                  timed and kept */
#define TCFFT_PLAN_PERSISTENT 64u /* tcfft_plan_many, plain FP16: every pass of
                                  every shape group in ONE persistent launch
                                  that claims (pass, chunk) items from a device
                                  work queue; a pass starts on a chunk once the
                                  previous pass of its group has completed (a
                                  device counter, bounded wait: a wait that
                                  runs out reports TCFFT_ERR_TIMEOUT through
                                  tcfft_plan_last_error and skips the rest).
                                  Other precisions ignore it */

/* Plan a batch of `batch` 1D transforms of length n (the paper's
 * tcfftPlan1D(plan, nx, batch), Sec. 3.1).  Allocates device twiddle tables
 * and, for n > 16384, a workspace of batch*n*4 bytes (x2 for
 * split); n > 2^24 runs three passes of at most 1024 points each.  On
 * success *plan owns them until tcfft_destroy.  Not timed by benchmarks. */
tcfft_status tcfft_plan_1d(tcfft_plan* plan, int64_t n, int64_t batch);

/* Plan a batch of 2D transforms of nx x ny points, row-major, ny contiguous
 * (the paper's tcfftPlan2D(plan, nx, ny, batch), Sec. 3.1). */
tcfft_status tcfft_plan_2d(tcfft_plan* plan, int64_t nx, int64_t ny, int64_t batch);

/* As above with an explicit precision and TCFFT_PLAN_* flags. */
tcfft_status tcfft_plan_1d_ex(tcfft_plan* plan, int64_t n, int64_t batch,
                              tcfft_precision precision, unsigned flags);
tcfft_status tcfft_plan_2d_ex(tcfft_plan* plan, int64_t nx, int64_t ny, int64_t batch,
                              tcfft_precision precision, unsigned flags);

/* Ragged batch (many transforms of mixed shapes in one exec): transform i
 * is 1D of length n0[i] when n1 is NULL or n1[i] == 0, else 2D
 * n0[i] x n1[i] (row-major, n1[i] contiguous).  The transforms are packed in
 * one buffer in the given order: transform i starts at element offset
 * sum_{j<i} size_j (x planes for split precision, each plane holding all
 * transforms).  Sizes follow the 1D / 2D rules above, except that 2D first
 * dimensions are limited to 4096 (2048 split).  Transforms of one shape
 * form a group; each group runs as one batched pass sequence reading and
 * writing through a device table of transform offsets; with
 * TCFFT_PLAN_GRAPH the groups are independent branches of one graph launch.
 * count >= 1. */
tcfft_status tcfft_plan_many(tcfft_plan* plan, int64_t count, const int64_t* n0, const int64_t* n1,
                             tcfft_precision precision, unsigned flags);

/* The execution function (Sec. 3.1, Fig. 1): runs the plan's merging
 * kernels in turn on `stream` (a cudaStream_t; NULL = legacy default
 * stream).  in/out: device buffers of tcfft_io_bytes(plan) bytes each,
 * 16-byte aligned; may be equal.  Asynchronous: returns once the kernels
 * are enqueued. */
tcfft_status tcfft_exec(tcfft_plan plan, const void* in, void* out, void* stream);

/* As tcfft_exec on the first `batch` transforms only (1 <= batch <= the
 * planned batch): in/out hold `batch` transforms (split: two planes of
 * `batch` transforms each).  Lets a resident plan serve requests of any
 * smaller batch.  Not for ragged plans (TCFFT_ERR_UNSUPPORTED). */
tcfft_status tcfft_exec_batch(tcfft_plan plan, const void* in, void* out, int64_t batch, void* stream);

/* End-to-end variant for host buffers: copies host_in to a plan-owned
 * device buffer, runs the plan, copies the result to host_out, and returns
 * once the result is in host_out.  host_in and host_out hold
 * tcfft_io_bytes(plan) bytes each (pinned memory gives full copy bandwidth
 * and the overlap below).  Batches of one plane (TCFFT_FP16, TCFFT_FP32) of
 * at least 2^22 points run as up to 8 slices of whole transforms whose
 * uploads, transforms (on `stream`) and downloads overlap, on two streams
 * the plan owns; other plans copy, run and copy back on `stream`.  The
 * result equals tcfft_exec's bit for bit.  The device buffers and streams
 * are allocated on the first call. */
tcfft_status tcfft_exec_host(tcfft_plan plan, const void* host_in, void* host_out, void* stream);

/* Frees everything the plan owns (no counterpart in the paper: plan
 * lifetime is library plumbing).  NULL is accepted. */
tcfft_status tcfft_destroy(tcfft_plan plan);

/* Reads and clears the plan's device status word (synchronises the device
 * first).  TCFFT_OK when no kernel reported an error.  No counterpart in the
 * paper: it reports the bounded device-side waits and launch checks of this
 * library. */
tcfft_status tcfft_plan_last_error(tcfft_plan plan);

/* Bytes of one input (== output) buffer of the plan (no counterpart in the
 * paper; follows from the plan's sizes and precision). */
size_t tcfft_io_bytes(tcfft_plan plan);

/* Device memory the plan holds besides the caller's buffers (workspace,
 * tables, host-path staging); for admission control (no counterpart in the
 * paper). */
size_t tcfft_workspace_bytes(tcfft_plan plan);

/* Number of kernel launches one tcfft_exec issues (no counterpart in the
 * paper; the launches are the merging passes of Sec. 3.1). */
int tcfft_plan_num_launches(tcfft_plan plan);

/* Writes a JSON description of the plan's kernel launches (length, layout
 * mode, transforms per CTA, tiles, TMEM columns, shared memory, grid) into
 * buf (at most len bytes, NUL-terminated; no counterpart in the paper).  Returns the length the full
 * description needs, including the NUL; 0 for a NULL plan. */
size_t tcfft_plan_describe(tcfft_plan plan, char* buf, size_t len);

/* Allocation-free batched 1D transform (no counterpart in the paper).
 * For callers that cannot allocate device memory when they need a
 * transform: processes that reserved their whole device-memory budget up
 * front (a caching allocator or a serving process with a fixed pool), where
 * an allocation by the library would fail or take memory promised
 * elsewhere, and loops that must not pay for cudaMalloc / cudaFree, which
 * may synchronise the device.  Computes the same forward transform as a
 * plan made by tcfft_plan_1d(n, batch) and run by tcfft_exec, with the
 * workspace between its two passes, its twiddle tables and its status word
 * in fixed-size device arrays of the library (held by every GPU that loads
 * it until the process exits); it allocates nothing.
 *   n      power of two, 2^15 <= n <= 2^24 (the two-pass lengths)
 *   batch  >= 1 with n * batch <= 2^24 points (64 MiB workspace); larger
 *          requests return TCFFT_ERR_INVALID_SIZE
 *   in/out device buffers of n * batch interleaved FP16 complex values,
 *          16-byte aligned (in == out allowed); plain FP16 only
 *   stream cudaStream_t (NULL = legacy default stream); asynchronous.
 * The first call on a device fills the tables and synchronises that device;
 * make that first call before recording work on any stream.  Every call
 * shares the one workspace: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.  Nothing
 * needs clearing between calls (each call overwrites the workspace region
 * it reads).  Device-side wait timeouts of these kernels are not reported. */
tcfft_status tcfft_exec_1d_noalloc(int64_t n, int64_t batch, const void* in, void* out, void* stream);

/* Failure-path self-test (no counterpart in the paper): runs one kernel
 * that waits, with the library's bounded device-side wait, on a barrier
 * that nothing ever completes, and returns what the kernel reports --
 * TCFFT_ERR_TIMEOUT once limit_cycles (SM clock cycles, <= 4e9) have
 * passed.  The kernel exits normally; the context stays usable.
 * Synchronises the device. */
tcfft_status tcfft_selftest_wait_timeout(long long limit_cycles);

/* Failure-path self-test of the persistent executor (TCFFT_PLAN_PERSISTENT;
 * no counterpart in the paper): builds a persistent plan of one two-pass
 * transform of 2^16 points, withholds the first pass's queue items, runs the
 * launch with dependency waits limited to limit_cycles (SM clock cycles,
 * <= 4e9) and returns what the plan reports -- TCFFT_ERR_TIMEOUT when the
 * bounded wait ran out and the launch skipped the orphaned items.  The
 * kernel exits normally; the context stays usable.  Allocates and frees its
 * own buffers; synchronises the device. */
tcfft_status tcfft_selftest_queue_timeout(long long limit_cycles);

/* Human-readable name of a status code (static string; no counterpart in
 * the paper). */
const char* tcfft_status_string(tcfft_status status);

#ifdef __cplusplus
}
#endif

#endif /* TCFFT_H_ */
