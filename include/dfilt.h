/*
 * dfilt.h -- C ABI of libdfilt.so: batched direct-form IIR filters and their
 * closed-form gradients on one NVIDIA GB300 (sm_103a).
 *
 * The operation (paper: "Accelerating Automatic Differentiation of Direct Form
 * Digital Filters", Eq. rtf, Sec. 2): for every channel i of a batch,
 *
 *     y[n] = sum_{k=0..N} b_k x[n-k] - sum_{k=1..M} a_k y[n-k]
 *
 * with a_0 = 1 implicit, b zero-padded to order M (Sec. 2 pads the shorter
 * polynomial) and an initial state zi[0..M) in the transposed direct form II
 * convention (the form Sec. 2 names for SciPy/MATLAB): zi is the TDF-II state at
 * n = 0, equivalently zi[k] is added to the all-pole input at time k.
 *
 * The backward (Sec. 3.1, Eqs. dLdz, dLdx, dLdvBA; boundary condition App. A) is
 * the same recursion run in reversed time.  With u the reverse-time adjoint
 *     u[n] = gy[n] - sum_{k=1..M} a_k u[n+k],  u[n >= T] = 0,
 * the library returns
 *     grad_x[n]  = sum_{k=0..N} b_k u[n+k]
 *     grad_b[k]  = sum_n u[n] x[n-k]       (k = 0..N)
 *     grad_a[k]  = -sum_n u[n] y[n-k]      (k = 1..M)
 *     grad_zi[k] = u[k]                    (k = 0..M-1)
 *
 * Conventions shared by every entry point:
 *   - All array pointers are DEVICE pointers into caller-owned, contiguous,
 *     row-major fp32 memory (the ragged metadata arrays are int64/int32, also on
 *     the device).  The library never allocates or frees memory: outputs, the
 *     `saved` buffer and the workspace `ws` are sized with dfilt_workspace_size*
 *     and allocated by the caller.
 *   - Calls are asynchronous and ordered on `stream` (a cudaStream_t passed as
 *     void*; NULL = legacy default stream).  Argument errors are detected on the
 *     host and returned synchronously, before anything is launched.  A wait that
 *     ran out inside a kernel is recorded in a device status word that
 *     dfilt_sync_status() returns (and clears).
 *   - Shapes: 1 <= M <= 64, 0 <= N <= M, B >= 0, T >= 0.  Larger M returns
 *     DFILT_ERR_UNSUPPORTED; N > M returns DFILT_ERR_INVALID_ARG.
 *   - The library is not thread-safe with respect to concurrent calls that share
 *     a workspace or saved buffer.
 */
#ifndef DFILT_H
#define DFILT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DFILT_OK = 0,
    DFILT_ERR_INVALID_ARG = 1,   /* bad shape, NULL where required, misaligned buffer */
    DFILT_ERR_UNSUPPORTED = 2,   /* M > 64, unsupported option or device */
    DFILT_ERR_CUDA = 3,          /* a CUDA runtime call failed (launch, copy) */
    DFILT_ERR_TIMEOUT = 4,       /* a bounded device-side wait ran out */
    DFILT_ERR_NUMERIC = 5,       /* non-finite output (dfilt_set_numeric_check) */
    DFILT_ERR_WORKSPACE = 6,     /* ws_bytes smaller than dfilt_workspace_size asks */
    DFILT_ERR_BOUNDS = 7         /* debug build: a device-side index check failed */
} dfilt_status;

typedef enum {
    DFILT_ALGO_AUTO = 0,         /* library choice (chunked where supported) */
    DFILT_ALGO_SEQUENTIAL = 1,   /* one thread per channel, serial recursion */
    DFILT_ALGO_CHUNKED = 2       /* chunked scan: Toeplitz products on the tensor cores */
} dfilt_algo;

typedef enum {
    DFILT_PREC_FP32 = 0,         /* sequential kernel arithmetic (CUDA cores) */
    DFILT_PREC_TF32 = 1,         /* chunked: one TF32 product per Toeplitz tile */
    DFILT_PREC_TF32X3 = 3        /* chunked: split TF32 (hi*hi + hi*lo + lo*hi), FP32-class */
} dfilt_precision;

typedef struct {
    int algo;        /* dfilt_algo */
    int precision;   /* dfilt_precision; ignored by the sequential algorithm */
    int chunk_len;   /* chunk length L of the chunked algorithm; 0 = default (64) */
    int fp64_scan;   /* high-precision chunk-state scan (a serial scan in double-word
                        FP32 arithmetic, about 44 bits: FP64-class accuracy without
                        GB300's narrow FP64 pipe): -1 auto (orders above 2),
                        0 off (FP32 two-level scan, orders <= 16), 1 on */
    int path;        /* chunked algorithm, orders above 8 (state buckets 16..64) with the
                        high-precision scan: DFILT_PATH_AUTO, DFILT_PATH_FUSED or
                        DFILT_PATH_DECOUPLED (below); lower orders always run fused */
    int span_tiles;  /* decoupled path: 8192-sample tiles per scan span (a power of two,
                        1..4096) -- a channel longer than one span is scanned by several
                        CTAs joined by a look-back; 0 = automatic (tuning table, else a
                        rule on the batch shape) */
} dfilt_opts;

typedef enum {
    DFILT_PATH_AUTO = 0,         /* decoupled where a `saved` buffer is given, else fused */
    DFILT_PATH_FUSED = 1,        /* one persistent kernel per call: tiles of a channel in
                                    order on one SM, the chunk-state scan inside it */
    DFILT_PATH_DECOUPLED = 2     /* separate launches: E pass (chunk end states, CUDA
                                    cores), chunk-state scan over spans of channels on many
                                    SMs (bounded look-back), tensor-core output passes;
                                    needs `saved` */
} dfilt_path;

/* Library version (major*10000 + minor*100 + patch). */
int dfilt_version(void);

/* Human-readable name of a status code (static string, never NULL). */
const char *dfilt_status_string(dfilt_status s);

/*
 * Fill *opts with the defaults: AUTO algorithm, TF32X3, default chunk length,
 * automatic scan precision.  opts must not be NULL.
 */
dfilt_status dfilt_default_opts(dfilt_opts *opts);

/*
 * Byte sizes the caller must provide for a fixed-shape batch x[B,T]:
 *   fwd_ws     -- workspace of dfilt_forward
 *   saved      -- buffer dfilt_forward fills for dfilt_backward (chunk-boundary
 *                 states and the backward's per-channel coefficient tables; 0 for
 *                 the sequential algorithm, which re-reads y)
 *   bwd_ws     -- workspace of dfilt_backward
 * opts may be NULL (defaults).  Output pointers may be NULL (not wanted).
 */
dfilt_status dfilt_workspace_size(int64_t B, int64_t T, int N, int M, const dfilt_opts *opts,
                                  size_t *fwd_ws, size_t *saved, size_t *bwd_ws);

/*
 * Forward filter of a fixed-shape batch (Eq. rtf, TDF-II initial state).
 *   x   [B,T]      input signal
 *   b   [B,N+1]    numerator b_0..b_N per channel
 *   a   [B,M]      denominator a_1..a_M per channel (a_0 = 1 implicit)
 *   zi  [B,M]      initial TDF-II state; NULL = zero
 *   y   [B,T]      output (must not alias any input)
 *   saved          NULL, or at least `saved` bytes from dfilt_workspace_size: filled
 *                  with what dfilt_backward needs to recompute y per chunk and the
 *                  backward's coefficient tables (so the backward skips its setup)
 *   ws, ws_bytes   workspace of at least `fwd_ws` bytes (may be NULL when 0)
 * Returns DFILT_OK once all work is enqueued on `stream`.
 */
dfilt_status dfilt_forward(const float *x, const float *b, const float *a, const float *zi,
                           float *y, void *saved, void *ws, size_t ws_bytes,
                           int64_t B, int64_t T, int N, int M, const dfilt_opts *opts,
                           void *stream);

/*
 * Backward (closed-form adjoint of Sec. 3.1) of a fixed-shape batch.
 *   gy  [B,T]      upstream gradient dL/dy
 *   x   [B,T]      the forward's input
 *   y   [B,T]      the forward's output; may be NULL only for the chunked algorithm
 *                  when `saved` holds the forward's chunk states (y is then
 *                  recomputed per chunk)
 *   b, a, zi       the forward's coefficients and initial state
 *   saved          the forward's saved buffer, or NULL when y is given
 *   gx  [B,T], gb [B,N+1], ga [B,M], gzi [B,M]   gradients; each may be NULL (not
 *                  wanted)
 *   ws, ws_bytes   workspace of at least `bwd_ws` bytes
 * With `saved`, b and a must be the forward's (the tables in `saved` were formed
 * from them) and opts must select the same algorithm, chunk length, scan precision,
 * path and span length as the forward that filled `saved`.  The call may be repeated
 * with the same `saved`.  Passing y together with `saved` saves the decoupled path a
 * recomputation of y (the single-kernel path recomputes it either way).
 */
dfilt_status dfilt_backward(const float *gy, const float *x, const float *y,
                            const float *b, const float *a, const float *zi, const void *saved,
                            float *gx, float *gb, float *ga, float *gzi,
                            void *ws, size_t ws_bytes,
                            int64_t B, int64_t T, int N, int M, const dfilt_opts *opts,
                            void *stream);

/*
 * Ragged batch: channel i owns samples [offsets[i], offsets[i+1]) of the packed
 * signals (x, y, gy, gx of `total` floats), has orders Ms[i] (1..Mmax) and
 * Ns[i] (0..Ms[i]), and coefficient rows b[i*(Nmax+1) ..], a[i*Mmax ..],
 * zi[i*Mmax ..], zero-padded past its own order.  offsets (int64[B+1]), Ms, Ns
 * (int32[B]) are device arrays; offsets must be non-decreasing with offsets[0] = 0
 * and offsets[B] = total (checked on the device; a violation is reported through
 * dfilt_sync_status as DFILT_ERR_INVALID_ARG).
 * Workspace sizes depend only on (B, total, Nmax, Mmax).
 */
dfilt_status dfilt_workspace_size_ragged(int64_t B, int64_t total, int Nmax, int Mmax,
                                         const dfilt_opts *opts, size_t *fwd_ws, size_t *saved,
                                         size_t *bwd_ws);

dfilt_status dfilt_forward_ragged(const float *x, const int64_t *offsets, const int *Ms,
                                  const int *Ns, const float *b, const float *a, const float *zi,
                                  float *y, void *saved, void *ws, size_t ws_bytes,
                                  int64_t B, int64_t total, int Nmax, int Mmax,
                                  const dfilt_opts *opts, void *stream);

dfilt_status dfilt_backward_ragged(const float *gy, const float *x, const float *y,
                                   const int64_t *offsets, const int *Ms, const int *Ns,
                                   const float *b, const float *a, const float *zi,
                                   const void *saved, float *gx, float *gb, float *ga, float *gzi,
                                   void *ws, size_t ws_bytes, int64_t B, int64_t total,
                                   int Nmax, int Mmax, const dfilt_opts *opts, void *stream);

/*
 * Synchronise `stream` and return (then clear) the device status word: DFILT_OK,
 * DFILT_ERR_TIMEOUT (a bounded wait ran out; outputs of that call are undefined),
 * DFILT_ERR_INVALID_ARG (ragged metadata failed its device-side check), or
 * DFILT_ERR_CUDA if the synchronisation itself failed.
 */
dfilt_status dfilt_sync_status(void *stream);

/*
 * Kernel timing (a measurement aid; the paper has no counterpart).
 * dfilt_kernel_timing(1) makes every later forward/backward call record a pair of
 * CUDA events on its stream around its main kernel (not the coefficient setup), up
 * to 4096 pending pairs; dfilt_kernel_timing(0) stops recording.  Either call
 * discards pairs not yet read.  dfilt_kernel_timing_read waits for the recorded
 * pairs, returns the summed durations (milliseconds) and the number of calls per
 * direction (each output pointer may be NULL), and discards them.  Recording must
 * be off while a stream is being captured into a CUDA graph.
 */
dfilt_status dfilt_kernel_timing(int enable);
dfilt_status dfilt_kernel_timing_read(double *fwd_ms, int *fwd_calls, double *bwd_ms,
                                      int *bwd_calls);
/*
 * The same records split by class (each array of 8 entries, not NULL; read and discarded
 * like dfilt_kernel_timing_read): 0 the forward calls and 1 the backward calls as above;
 * within them, for the chunked algorithm, 2 the chunk-state scans, 3 the E passes
 * (zero-state chunk end states), 4 the output passes (y), 5 the adjoint output passes
 * (grad_x and the coefficient-gradient sums), 6 the span transitions, 7 the
 * single-kernel path's main kernels.  A class records one pair per state bucket and call.
 */
dfilt_status dfilt_kernel_timing_read_classes(double *ms, int *calls);

/* Number of kernels the library has launched in this process (a measurement aid). */
dfilt_status dfilt_launch_count(int64_t *n);

/*
 * Tuning table of the decoupled path (the paper has no counterpart; the launch shape is
 * this library's choice), per state bucket (2, 4, 8, 16, 32 or 64; orders up to the
 * bucket, above the previous one): span_tiles, the 8192-sample tiles per scan span (a
 * power of two up to 4096), and chains_per_sm, the chunk-state scan's CTAs per SM (at
 * most 32); 0 restores the built-in rule.  Calls whose opts give span_tiles use that
 * instead.  Process-wide; a call made while another thread changes the table sees
 * either setting.  The package's tuner (paper_2511_14390_gb300.tune) measures candidates
 * and installs the best.
 */
dfilt_status dfilt_tuning_set(int state_bucket, int span_tiles, int chains_per_sm);
dfilt_status dfilt_tuning_get(int state_bucket, int *span_tiles, int *chains_per_sm);

/*
 * Optional output check (off by default).  With enable != 0, every later forward /
 * backward call (dfilt_forward*, dfilt_backward*) also scans its outputs on `stream`
 * for non-finite values and records DFILT_ERR_NUMERIC in the device status word
 * (read by dfilt_sync_status) if it finds one.  Costs one extra read of the outputs.
 * Applies to calls made after it on any thread of the process.
 */
dfilt_status dfilt_set_numeric_check(int enable);

/*
 * Debug build (libdfilt_debug.so, compiled with -DDFILT_DEBUG; the paper has no
 * counterpart).  Its decoupled-path kernels (orders 3..64: E, scan, tile, lag and
 * correction passes) check every sample range and chunk-state slot range they derive
 * from the channel metadata and the work plan against the buffers before touching
 * them; a range that fails is skipped (no access) and DFILT_ERR_BOUNDS is recorded in
 * the device status word (read by dfilt_sync_status).  Nothing traps.  The release
 * library compiles the checks out.
 *
 * dfilt_debug_build: 1 in the debug library, 0 in the release library.
 * dfilt_debug_set_limit: makes the debug checks treat every signal as at most
 *   `samples` long (<= 0: no limit, the default), so that a test can make them fail
 *   on valid buffers: later calls skip the tiles and spans past the limit and report
 *   DFILT_ERR_BOUNDS, and their outputs there are undefined.  Process-wide, applies to
 *   calls made after it.  The release library returns DFILT_ERR_UNSUPPORTED.
 */
int dfilt_debug_build(void);
dfilt_status dfilt_debug_set_limit(int64_t samples);

/*
 * Test hook for the bounded device-side waits (no waits are unbounded).
 *   iters > 0   cap every wait at `iters` polls
 *   iters == 0  restore the default cap
 *   iters < 0   timeout drill: cap at -iters polls and make each tensor-core kernel
 *               additionally wait on a barrier that nothing ever signals, so the
 *               timeout path (status word, drain of in-flight work, tensor-memory
 *               release) runs deterministically without faulting or hanging the GPU.
 * Applies to calls made after it on any thread of the process.
 */
dfilt_status dfilt_set_wait_limit(int64_t iters);

/*
 * Forward filter that allocates nothing and takes no workspace (the paper has no
 * counterpart; this is a deployment convenience).  For callers that must not
 * allocate device memory while they run -- a real-time audio callback, where
 * cudaMalloc/cudaFree can synchronise the device and stall for an unbounded time, or
 * a host program without a device allocator to obtain a workspace from.
 *   Arguments as dfilt_forward without `saved`, `ws` and `ws_bytes`; computes the
 *   same y with the chunked algorithm (opts->algo must be AUTO or CHUNKED).
 *   Scratch: a fixed 4 MiB device array inside this library (per GPU that loads it,
 *   held until the process exits) instead of a caller workspace.  A batch whose
 *   per-channel tables need more -- dfilt_workspace_size's fwd_ws for the same batch
 *   and opts with path = DFILT_PATH_FUSED above 4 MiB -- is rejected with
 *   DFILT_ERR_WORKSPACE before anything is launched.  With the automatic scan
 *   precision that is more than 2730 channels at M <= 2 (the same with fp64_scan = 1),
 *   334 at M = 16, 168 at M = 32, 63 at M = 64.
 *   The first call on each device looks up the array's address (one-time set-up);
 *   make that first call before any stream capture.  All calls share the array:
 *   calls whose work overlaps on the GPU (other streams or threads) race and must be
 *   serialised by the caller.  Nothing needs clearing between calls.
 */
dfilt_status dfilt_forward_noalloc(const float *x, const float *b, const float *a,
                                   const float *zi, float *y, int64_t B, int64_t T, int N, int M,
                                   const dfilt_opts *opts, void *stream);

/*
 * Forward mode (Jacobian-vector product) of a fixed-shape batch: the directional
 * derivative dy of the forward's output along tangents of its inputs.  The paper
 * derives the reverse mode (Sec. 3.1) and notes that forward mode follows the same
 * way (Sec. 5); differentiating A(z) y = B(z) x (+ zi injected) gives
 *     v[n] = sum_{k=0..N} (b_k dx[n-k] + db_k x[n-k]) - sum_{k=1..M} da_k y[n-k]
 *     dy   = the all-pole filter 1/A(z) applied to v, TDF-II initial state dzi
 * (x, dx, y zero at negative times).
 *   x   [B,T]      the forward's input (may be NULL when db is NULL)
 *   y   [B,T]      the forward's output (may be NULL when da is NULL)
 *   b   [B,N+1]    numerator (may be NULL when dx is NULL)
 *   a   [B,M]      denominator a_1..a_M (required)
 *   dx [B,T], db [B,N+1], da [B,M], dzi [B,M]   tangents; NULL = zero
 *   dy  [B,T]      output (must not alias any input)
 *   ws, ws_bytes   workspace of at least dfilt_jvp_workspace_size bytes, 16-byte
 *                  aligned (it holds v, so it grows with B*T)
 * opts selects the algorithm of the recursion as for dfilt_forward; the optional
 * finite-output check applies to dy.  Asynchronous on `stream` like every entry point.
 */
dfilt_status dfilt_jvp_workspace_size(int64_t B, int64_t T, int N, int M,
                                      const dfilt_opts *opts, size_t *ws_bytes);
dfilt_status dfilt_jvp(const float *x, const float *y, const float *b, const float *a,
                       const float *dx, const float *db, const float *da, const float *dzi,
                       float *dy, void *ws, size_t ws_bytes, int64_t B, int64_t T, int N, int M,
                       const dfilt_opts *opts, void *stream);

/*
 * The general linear recurrence of App. B (the operator the paper benchmarks at
 * M = 2), batched over B independent channels, each with its own dense A:
 *     v(n+1) = A v(n) + z(n),   n = 0..T-1,   v(0) = v0
 * and its backward (App. A, Eqs. dLdz and dLdvBA): dL/dz is the same recurrence run
 * with A^T on the time-reversed dL/dv from a zero state; dL/dv0 = A^T dL/dz(0);
 * dL/dA = sum_n dL/dz(n) v(n)^T with v(n) the state before step n.
 *   A   [B,M,M]    row-major per channel (row i produces v_i)
 *   v0  [B,M]      initial state; NULL = zero
 *   z   [B,T,M]    inputs, step-major (the M entries of a step contiguous)
 *   v   [B,T,M]    outputs v(1..T)
 *   gv  [B,T,M]    upstream gradient dL/dv(1..T)
 *   gA [B,M,M], gv0 [B,M]   gradients, each may be NULL (not wanted); v may be NULL
 *                  when gA is NULL
 *   gz  [B,T,M]    gradient dL/dz (required: the other two are formed from it)
 *   ws, ws_bytes   workspace of at least fwd_ws / bwd_ws bytes, 16-byte aligned
 * Supported 1 <= M <= 4 (DFILT_ERR_UNSUPPORTED above).  FP32 arithmetic; the powers
 * of A the chunked scan uses are formed in FP64.  dL/dA sums in a fixed order.
 */
dfilt_status dfilt_ss_workspace_size(int64_t B, int64_t T, int M, size_t *fwd_ws,
                                     size_t *bwd_ws);
dfilt_status dfilt_ss_forward(const float *A, const float *v0, const float *z, float *v,
                              void *ws, size_t ws_bytes, int64_t B, int64_t T, int M,
                              void *stream);
dfilt_status dfilt_ss_backward(const float *A, const float *v0, const float *v, const float *gv,
                               float *gA, float *gv0, float *gz, void *ws, size_t ws_bytes,
                               int64_t B, int64_t T, int M, void *stream);

/*
 * Parameter-varying direct form (Sec. 5: the derivation extends to coefficients that
 * change over time).  Reading: each output sample n has its own coefficients, as the
 * difference equation of Eq. rtf written per sample,
 *     y[n] = sum_{k=0..N} b[n][k] x[n-k] - sum_{k=1..M} a[n][k-1] y[n-k],
 * with x[n < 0] = 0 and past outputs y[-1-j] = ypast[j].  The backward takes each
 * coefficient at the output it produced:
 *     u[n] = gy[n] - sum_{k=1..M} a[n+k][k-1] u[n+k],   u[n >= T] = 0
 *     grad_x[n] = sum_k b[n+k][k] u[n+k],   grad_b[n][k] = u[n] x[n-k],
 *     grad_a[n][k-1] = -u[n] y[n-k] (ypast before n = 0),
 *     grad_ypast[j] = -sum_{k=j+1..M} a[k-1-j][k-1] u[k-1-j].
 *   x, y, gy, gx   [B,T]
 *   b, gb          [B,T,N+1]   per-sample numerators (row n: b[n][0..N])
 *   a, ga          [B,T,M]     per-sample denominators a_1..a_M (a_0 = 1)
 *   ypast, gypast  [B,M]       y[-1], ..., y[-M]; ypast NULL = zero
 *   gx, gb, ga, gypast may each be NULL (not wanted)
 *   ws, ws_bytes   workspace of at least dfilt_tv_workspace_size bytes, 16-byte aligned
 * 1 <= M <= 4 (DFILT_ERR_UNSUPPORTED above), 0 <= N <= M.  FP32 arithmetic: a chunked
 * scan over the per-step companion matrices, the runs of steps combined by the paper's
 * associative operator (Sec. 3.2) with a different A per step.
 */
dfilt_status dfilt_tv_workspace_size(int64_t B, int64_t T, int N, int M, size_t *ws_bytes);
dfilt_status dfilt_tv_forward(const float *x, const float *b, const float *a, const float *ypast,
                              float *y, void *ws, size_t ws_bytes, int64_t B, int64_t T, int N,
                              int M, void *stream);
dfilt_status dfilt_tv_backward(const float *gy, const float *x, const float *y, const float *b,
                               const float *a, const float *ypast, float *gx, float *gb,
                               float *ga, float *gypast, void *ws, size_t ws_bytes, int64_t B,
                               int64_t T, int N, int M, void *stream);

/*
 * The same recurrence with A given by its eigendecomposition, A = V diag(lam) V^-1 (the
 * paper's Diag-EXT, Sec. 3.2 and Sec. 4; applicable when A is diagonalisable): the
 * state in the eigenbasis q = V^-1 v evolves element by element,
 *     q(n+1) = lam * q(n) + V^-1 z(n),  q(0) = V^-1 v0,  v(n) = Re(V q(n)),
 * and the backward is the same operator for A^T = V^-T diag(lam) V^T on the
 * time-reversed dL/dv from a zero state (App. A, Eq. dLdz), then
 * dL/dv0 = A^T dL/dz(0) and dL/dA = sum_n dL/dz(n) v(n)^T (Eq. dLdvBA), with v(n) the
 * state before step n: the gradients are those of the dense operator above, so dL/dA
 * needs no derivative of the eigendecomposition.
 *   lam   [B,M]     eigenvalues, complex as interleaved (re, im) floats (8-byte aligned)
 *   V     [B,M,M]   eigenvectors as columns, row-major, complex (8-byte aligned)
 *   Vinv  [B,M,M]   the inverse of V, row-major, complex (8-byte aligned)
 *   v0 [B,M], z [B,T,M], v [B,T,M], gv [B,T,M], gz [B,T,M], gA [B,M,M], gv0 [B,M]:
 *                   real, as for dfilt_ss_forward / dfilt_ss_backward (v0 NULL = zero;
 *                   gA, gv0 NULL = not wanted; v may be NULL when gA is NULL)
 *   ws, ws_bytes    workspace of at least fwd_ws / bwd_ws bytes, 16-byte aligned
 * A real A's complex eigenpairs must come in conjugate pairs (as numpy's or torch's
 * eig returns them) for V q to be real; its imaginary part is dropped.  Supported
 * 1 <= M <= 4 (DFILT_ERR_UNSUPPORTED above).  Complex FP32 arithmetic; the powers of
 * lam the chunked scan uses come from FP64 squaring; dL/dA sums in a fixed order.
 */
dfilt_status dfilt_diag_workspace_size(int64_t B, int64_t T, int M, size_t *fwd_ws,
                                       size_t *bwd_ws);
dfilt_status dfilt_diag_forward(const float *lam, const float *V, const float *Vinv,
                                const float *v0, const float *z, float *v, void *ws,
                                size_t ws_bytes, int64_t B, int64_t T, int M, void *stream);
dfilt_status dfilt_diag_backward(const float *lam, const float *V, const float *Vinv,
                                 const float *v0, const float *v, const float *gv, float *gA,
                                 float *gv0, float *gz, void *ws, size_t ws_bytes, int64_t B,
                                 int64_t T, int M, void *stream);

/*
 * Direct-form initial conditions: past inputs xpast[B,N] = (x[-1], ..., x[-N]) and past
 * outputs ypast[B,M] = (y[-1], ..., y[-M]) (the convention of SciPy's lfiltic and
 * MATLAB's filtic) mapped to the TDF-II state zi[B,M] that dfilt_forward takes (Sec. 2
 * pairs the direct form with its transposed form):
 *     zi[m] = sum_{k=m+1..N} b_k x[m-k] - sum_{k=m+1..M} a_k y[m-k]
 * xpast or ypast may be NULL (zero).  dfilt_ic_df1_backward is the adjoint of that map:
 * from gzi = dL/dzi (dfilt_backward's grad_zi) it writes
 *     gxpast[j-1] = sum_m gzi[m] b_{m+j},   gypast[j-1] = -sum_m gzi[m] a_{m+j}
 * and ADDS the past values' terms to the filter's coefficient gradients:
 *     gb[k] += sum_{m<k} gzi[m] x[m-k],   ga[k-1] -= sum_{m<k} gzi[m] y[m-k]
 * so that gb, ga from dfilt_backward become the gradients of the filter with past
 * values.  Each output may be NULL (not wanted).  Device pointers; asynchronous.
 */
dfilt_status dfilt_ic_df1(const float *b, const float *a, const float *xpast,
                          const float *ypast, float *zi, int64_t B, int N, int M,
                          void *stream);
dfilt_status dfilt_ic_df1_backward(const float *b, const float *a, const float *xpast,
                                   const float *ypast, const float *gzi, float *gxpast,
                                   float *gypast, float *gb, float *ga, int64_t B, int N, int M,
                                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DFILT_H */
