/*
 * gtt.h -- C ABI of the GB300 Generalized Tensor Transform library (libgtt.so).
 *
 * The transform (Def. 2.3 of arXiv 2507.02420, "Generalized tensor
 * transforms and their applications in classical and quantum computing"):
 *
 *     y = G_N x,   G_N = W (x) W (x) ... (x) W  (n factors),   N = b^n,
 *
 * for a b x b base matrix W.  Element form (Sec. 2.6):
 *
 *     y[p] = sum_q prod_{j=0}^{n-1} W[p_j][q_j] x[q],
 *
 * where p = sum_j p_j b^j and q = sum_j q_j b^j are base-b digit expansions
 * (digit 0 least significant) and W[i][j] is row i, column j, 0-based
 * (Sec. 2.1).  This is the "natural ordering" of the paper: no digit
 * reversal and no sequency reordering.  The fast algorithm of Sec. 3
 * (Algorithm 1) applies W to one digit at a time; its cost is O(N b log_b N).
 *
 * Conventions shared by every call below
 * --------------------------------------
 * - Vectors are contiguous and batch-major: `batch` vectors of N elements,
 *   vector v occupying elements [v*N, (v+1)*N).
 * - Element types (gtt_dtype_t): F64 = double, F32 = float, C64 = interleaved
 *   (float re, float im), C128 = interleaved (double re, double im),
 *   I32 = int32 whose arithmetic wraps modulo 2^32 (computed in uint32).
 * - Device pointers (x, y, dx, dy) must be 16-byte aligned device memory of
 *   the plan's device; a misaligned or NULL pointer returns
 *   GTT_ERR_INVALID_ARG.  The caller owns them.  In-place use (y == x) is
 *   allowed; partially overlapping buffers are not.
 * - Every device call is asynchronous on `stream` (a cudaStream_t passed as
 *   void*; NULL is the legacy default stream).  Errors are returned as status
 *   codes and never abort the process; gtt_last_error() gives a message for
 *   the calling thread.  CUDA errors map to GTT_ERR_CUDA.
 * - A plan may be used from one host thread at a time.
 */
#ifndef GTT_H_
#define GTT_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gtt_plan_s *gtt_plan_t;
typedef struct gtt_group_s *gtt_group_t;
typedef void *gtt_stream_t; /* cudaStream_t */

typedef enum {
    GTT_F64 = 0,
    GTT_F32 = 1,
    GTT_C64 = 2,
    GTT_C128 = 3,
    GTT_I32 = 4
} gtt_dtype_t;

typedef enum {
    GTT_OK = 0,
    GTT_ERR_INVALID_ARG = 1, /* bad size, pointer, alignment or enum value      */
    GTT_ERR_UNSUPPORTED = 2, /* valid request this build does not implement      */
    GTT_ERR_ALLOC = 3,       /* device or host allocation failed                 */
    GTT_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed      */
    GTT_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired               */
    GTT_ERR_INTERNAL = 6
} gtt_status_t;

/* Arithmetic of the mode contractions (gtt_plan_set_precision). */
typedef enum {
    GTT_PREC_AUTO = 0,   /* library choice, the default: BF16X3 for b = 16 FP32 with
                            n >= 3 (faster, and at least as accurate), else FP32      */
    GTT_PREC_FP32 = 1,   /* FP32 FMA on CUDA cores                                  */
    GTT_PREC_BF16X3 = 2, /* tcgen05 BF16 products of 3-piece splits, FP32 accumulate */
    GTT_PREC_BF16X2 = 4, /* b = 16 FP32, opt-in: tcgen05 BF16 products of 2-piece
                            splits (x0 W0 + x0 W1 + x1 W0), about 2^-16 relative
                            per mode; the cheaper reading of split BF16, kept to
                            compare with BF16X3                                     */
    GTT_PREC_TF32X3 = 3  /* opt-in, tcgen05 TF32 products of 2-piece splits (three
                            products; x rounded to nearest TF32, A operand in tensor
                            memory), FP32 accumulate.  b = 16 FP32: each mode on the
                            tensor cores, about 2^-21 relative per mode.  complex64,
                            b = 4: pairs of digits as one base-16 digit with W (x) W,
                            the digits left over in each pass on CUDA cores in FP32,
                            two HBM round trips for n = 13 (slower than FP32 on
                            GB300)                                                   */
} gtt_precision_t;

/*
 * gtt_plan_create -- validate a transform and prepare it on the current CUDA
 * device.  Definition: Def. 2.3 (G_N = W^{(x)n}).
 *   out    receives the plan (owned by the caller; free with gtt_plan_destroy).
 *   b      base, 2 <= b <= 16.
 *   n      number of digits, n >= 1; N = b^n.
 *   W      HOST pointer to b*b elements of `dtype`'s element type, row-major
 *          (W[i*b + j] is row i, column j).  Copied; the caller keeps ownership.
 *          For GTT_I32 the entries are int32.
 *   dtype  element type of W, x and y.
 *   batch  number of vectors per call, >= 1.
 * The plan owns device copies of W, of W^H (W^T for real types) and of any
 * workspace, and a fusion schedule (mode groups and tile shapes) chosen from
 * the autotune cache when one is loaded, else by a fixed rule.
 * Errors: GTT_ERR_INVALID_ARG (b, n, batch or dtype out of range, NULL out/W,
 * batch*N above 2^40 elements), GTT_ERR_ALLOC, GTT_ERR_CUDA.
 */
gtt_status_t gtt_plan_create(gtt_plan_t *out, int b, int n, const void *W, gtt_dtype_t dtype,
                             long long batch);

/*
 * gtt_plan_create_mixed -- the heterogeneous transform of the remark after
 * Def. 2.3: G_N = W_0 (x) W_1 (x) ... (x) W_{n-1} (Kronecker product in this
 * order) with W_k of size b_k x b_k, 2 <= b_k <= 16, N = prod b_k.  W_0 acts
 * on the most significant index and W_{n-1} on the fastest-varying one:
 * y[p] = sum_q prod_k W_k[p_k][q_k] with p = (...((p_0 b_1 + p_1) b_2 + p_2)...).
 *   radices  HOST array of n ints b_0 .. b_{n-1}.
 *   W        HOST pointer: W_0, W_1, ..., W_{n-1} back to back, each row-major
 *            b_k x b_k of `dtype`'s element type.
 * The plan runs CUDA-core passes over the digits, fastest first: adjacent
 * factors whose sizes multiply to at most 16 form one digit, transformed by
 * their Kronecker product (formed in double precision, or modulo 2^32 for
 * I32, and rounded once); consecutive digits then share a pass, one stage
 * per digit, as long as a tile of at most 48 KiB holds them, so most such
 * transforms take one to three HBM round trips (gtt_forward, gtt_inverse
 * with the adjoints, the host-buffer calls, gtt_filter, gtt_compress and
 * gtt_decompress).  gtt_plan_set_w takes the same concatenated layout.  The
 * backward, explicit schedules and the autotuner return GTT_ERR_UNSUPPORTED
 * for such a plan.  Errors: GTT_ERR_INVALID_ARG (NULL pointers, n < 1, a b_k
 * outside [2, 16], sizes), GTT_ERR_ALLOC, GTT_ERR_CUDA.
 */
gtt_status_t gtt_plan_create_mixed(gtt_plan_t *out, int n, const int *radices, const void *W, gtt_dtype_t dtype,
                                   long long batch);

/* Replace the plan's base matrix (HOST pointer, same layout and type as in
 * gtt_plan_create) without rebuilding its schedule; used when W is trained.
 * Calls already queued on a stream keep the W they were launched with. */
gtt_status_t gtt_plan_set_w(gtt_plan_t plan, const void *W);

/* Select the arithmetic of the mode contractions (gtt_precision_t).
 * GTT_PREC_BF16X3 and GTT_PREC_BF16X2 require b = 16, dtype F32 and n >= 3; GTT_PREC_TF32X3
 * requires the same, or b = 4, dtype C64 and n = 7 + 6k (k >= 0): a 7-digit pass and k
 * 6-digit passes, each one HBM round trip (thread-block clusters of four CTAs
 * exchange one digit through distributed shared memory); otherwise
 * GTT_ERR_UNSUPPORTED.  A tensor-core path has one fixed schedule:
 * gtt_plan_set_schedule and gtt_plan_set_passes install a CUDA-core schedule
 * and so switch the plan to FP32; gtt_plan_set_pipeline only affects later
 * CUDA-core schedules and the backward; gtt_plan_autotune leaves a
 * tensor-core plan unchanged. */
gtt_status_t gtt_plan_set_precision(gtt_plan_t plan, int precision);

/*
 * gtt_plan_set_schedule -- replace the plan's fusion schedule by the fixed
 * rule with the given limits: passes whose tiles hold at most max_tile_bytes
 * (one shared-memory tile per CTA, <= 220 KiB) and, for passes above the
 * lowest digits, contiguous runs of at least min_run_bytes where the lower
 * digits allow it.  Used by the autotuner and by tests that sweep schedules.
 * Errors: GTT_ERR_INVALID_ARG (limits out of range), GTT_ERR_CUDA.
 */
gtt_status_t gtt_plan_set_schedule(gtt_plan_t plan, long long max_tile_bytes,
                                   long long min_run_bytes);

/*
 * gtt_plan_set_passes -- set the fusion schedule explicitly.  Pass k applies
 * digits[k] consecutive modes (the first pass starts at digit 0, each next
 * pass where the previous one ended; the digits must sum to n) to tiles of
 * b^digits[k] rows of runs[k] contiguous elements.  For k > 0, runs[k] must
 * divide b^(digits before pass k).  The first pass has no lower digits:
 * runs[0] = k means tiles of k consecutive blocks of b^digits[0] contiguous
 * elements (k must divide batch * b^(n - digits[0])).  A tile (rows x run)
 * must fit 220 KiB.  Errors: GTT_ERR_INVALID_ARG (bad counts, sums, runs or
 * sizes), GTT_ERR_UNSUPPORTED, GTT_ERR_CUDA.
 */
gtt_status_t gtt_plan_set_passes(gtt_plan_t plan, int count, const int *digits, const long long *runs);

/*
 * gtt_plan_autotune -- enumerate the candidate schedules (mode groups of at
 * most four passes, run lengths), rank them by a model of their HBM and FMA
 * time, and time the max_candidates (<= 0: 64) best-ranked ones in every
 * pipeline variant (no TMA, TMA with 1..3 buffers) on scratch buffers of the
 * plan's size; the six fastest are timed again over more runs.  The winner
 * goes into the plan and into the process-wide autotune cache, keyed by GPU name, b, n,
 * dtype and batch.  Allocates and frees two data-sized device buffers;
 * synchronizes the device.  gtt_plan_create applies a cached schedule when
 * one exists; the environment variable GTT_AUTOTUNE_CACHE names a cache file
 * loaded at the first plan creation, and GTT_AUTOTUNE=on tunes uncached
 * shapes at creation.
 * gtt_autotune_cache_load / _save -- merge a cache file into the process
 * cache / write the process cache (one JSON object per line).
 */
gtt_status_t gtt_plan_autotune(gtt_plan_t plan, int max_candidates);
gtt_status_t gtt_autotune_cache_load(const char *path);
gtt_status_t gtt_autotune_cache_save(const char *path);

/*
 * gtt_plan_set_pipeline -- choose how the forward/inverse passes stage their
 * tiles: use_tma != 0 streams tiles through `nbuf` (1..4) shared-memory
 * buffers with tensor-memory-accelerator copies where the tile geometry allows
 * (b a power of two, 128-byte rows); use_tma == 0 uses plain loads and stores.
 * Rebuilds the schedule with the current limits.  Default: use_tma = 1,
 * nbuf = 2.  Errors: GTT_ERR_INVALID_ARG (nbuf out of range), GTT_ERR_CUDA.
 */
gtt_status_t gtt_plan_set_pipeline(gtt_plan_t plan, int use_tma, int nbuf);

/*
 * gtt_plan_set_chunking -- L2-resident execution of the leading passes.  The
 * leading passes of the schedule that only touch digits below some digit s
 * (blocks of b^s consecutive elements, batch items included) run on chunks of
 * at most `elems` elements (whole blocks) one chunk after the other, so each
 * such pass after the first reads the previous pass's output from L2 instead
 * of HBM; the remaining passes then run over all the data.  0 = off (the
 * default); -1 = automatic (48 MiB chunks when the data exceed 96 MiB).  It
 * takes effect only when at least two passes share a chunk.  Results are
 * bitwise identical; only the launch order changes.  elems < -1 returns
 * GTT_ERR_INVALID_ARG.
 */
gtt_status_t gtt_plan_set_chunking(gtt_plan_t plan, long long elems);

/*
 * gtt_plan_check -- wait for the device and report whether any kernel of this
 * plan gave up a bounded wait (GTT_ERR_TIMEOUT; the flag is then cleared).
 * Kernels never spin without limit: an expired wait records the error, drains
 * the kernel's own copies and returns.
 */
gtt_status_t gtt_plan_check(gtt_plan_t plan);

/*
 * gtt_forward -- y = G_N x for each of the plan's `batch` vectors, natural
 * ordering (Sec. 2.6 element form; Sec. 3 fast algorithm).
 *   x  device, batch*N elements (read).   y  device, batch*N elements (written).
 */
gtt_status_t gtt_forward(gtt_plan_t plan, const void *x, void *y, gtt_stream_t stream);

/*
 * gtt_inverse -- x = (W^H)^{(x)n} y = G_N^dagger y (Sec. 4: the inverse GTT used
 * for reconstruction).  This is the adjoint transform; it equals G_N^{-1}
 * only when W is unitary.  For the +-1 integer Hadamard W it returns 2^n x.
 */
gtt_status_t gtt_inverse(gtt_plan_t plan, const void *y, void *x, gtt_stream_t stream);

/*
 * gtt_backward -- reverse-mode derivative of y = G_N x for a real loss L
 * (not in the paper; PyTorch's conjugate convention for complex types):
 *     dx = (W^H)^{(x)n} dy,
 *     dW = sum_k sum_{mode-k fibres} g_{k+1} a_k^H,
 * with a_0 = x, a_{k+1} the result of applying W to digit k of a_k, and
 * g_{k+1} = dL/da_{k+1}.
 *   x_saved  device, batch*N elements: the forward input.
 *   dy       device, batch*N elements: dL/dy.
 *   dx       device, batch*N elements or NULL (not computed).
 *   dW       device, b*b elements of the element type, row-major, or NULL;
 *            overwritten with the sum over the whole batch.  The sum is taken
 *            in a fixed order, so repeated calls give identical bits.
 * dx may alias dy but not x_saved (GTT_ERR_INVALID_ARG: a checkpoint may be
 * written to dx before x_saved is read for the last time).  Floating-point
 * dtypes only (GTT_ERR_UNSUPPORTED for I32).
 */
gtt_status_t gtt_backward(gtt_plan_t plan, const void *x_saved, const void *dy, void *dx, void *dW,
                          gtt_stream_t stream);

/*
 * gtt_forward_saving -- gtt_forward that also keeps, in ckpt, the activation
 * entering the second pass of the plan's backward schedule (digits below the
 * backward's split applied), which gtt_backward would otherwise recompute
 * with an extra forward pass (not in the paper).  The forward runs its own
 * schedule; the pass ending at the split writes ckpt, the next pass reads it.
 *   x     device, batch*N elements (read).   y  device, batch*N (written).
 *   ckpt  device, batch*N elements (written); must not alias x or y.
 * Available when the backward schedule has two passes and the forward
 * schedule has a pass boundary at its split digit (e.g. FP32 b = 8, n = 5..7,
 * with the default schedule); otherwise GTT_ERR_UNSUPPORTED and nothing is
 * launched.
 */
gtt_status_t gtt_forward_saving(gtt_plan_t plan, const void *x, void *y, void *ckpt, gtt_stream_t stream);

/*
 * gtt_backward_saved -- gtt_backward with the checkpoint that
 * gtt_forward_saving wrote for the same x (and the same W): the backward
 * passes only, no recompute pass.  Arguments as gtt_backward, plus ckpt
 * (device, batch*N elements, read; distinct from x_saved and dy; dx may alias
 * it).  GTT_ERR_UNSUPPORTED where gtt_forward_saving is.
 */
gtt_status_t gtt_backward_saved(gtt_plan_t plan, const void *x_saved, const void *ckpt, const void *dy, void *dx,
                                void *dW, gtt_stream_t stream);

/*
 * gtt_backward_noalloc -- the same results as gtt_backward, computed without
 * allocating any device memory (the paper has no counterpart to this call).
 * For callers that must not allocate on the device from inside the library:
 * code running under a framework's caching allocator that has already
 * reserved the device's memory (where a stray cudaMalloc can fail or fragment
 * the pool), or latency-critical loops where cudaMalloc/cudaFree would
 * synchronize the device.
 *   x, dy, dW as in gtt_backward.  dx is required (non-NULL) and must alias
 *   neither dy nor x: it also holds the checkpoint between the two backward
 *   passes.  The kernels and their order are those of gtt_backward with the
 *   same dx, so dx and dW are bitwise equal to gtt_backward's.
 * Scratch: the dW partials live in a fixed 1 MiB array in the library's
 * device globals (held by every GPU that loads the library until exit).
 * Every call looks up that array's device address with the plan's device
 * current; the first call also builds the plan's backward schedule on the
 * host, so make that first call before any stream capture.  All calls share
 * the array and each overwrites what it reads; calls whose kernels overlap on
 * the GPU (other streams, other plans) race on it and must be serialised.
 * Errors: GTT_ERR_INVALID_ARG when dx is NULL or aliases dy or x, when the
 * transform needs more than two backward passes (a data-sized checkpoint),
 * or when its dW partials exceed the 1 MiB array; otherwise as gtt_backward.
 */
gtt_status_t gtt_backward_noalloc(gtt_plan_t plan, const void *x_saved, const void *dy, void *dx,
                                  void *dW, gtt_stream_t stream);

/*
 * gtt_filter -- natural-order spectral filtering (Sec. 4.3.2, the classical
 * reading of Algorithm 3): y = G_N^dagger (mask * G_N x) for every vector of
 * the batch, where the mask keeps the coefficients of index p < cut
 * (keep_low != 0, low-pass) or p >= cut (keep_low == 0, high-pass) and zeroes
 * the others; the index is the natural ordering of the spectrum.  x and y are
 * device buffers of batch*N elements with the plan's conventions (y == x is
 * allowed).  y holds the spectrum between the two transforms; the masked
 * range is zeroed by a write-only kernel.  Errors: GTT_ERR_INVALID_ARG (NULL or
 * misaligned pointers, cut outside [0, N]), GTT_ERR_CUDA.
 */
gtt_status_t gtt_filter(gtt_plan_t plan, const void *x, void *y, long long cut, int keep_low,
                        gtt_stream_t stream);

/*
 * gtt_compress -- the classical steps of the compression protocol of
 * Sec. 4.1.5: spectrum = G_N x (device, batch*N elements, may equal x), then
 * for every vector the k coefficients of largest magnitude: indices[v*k + j]
 * (device int64) and values[v*k + j] (device, the plan's element type), j
 * ordered by |c| descending and, between equal magnitudes, by the larger
 * index first.  |c|^2 is computed in the plan's real precision with
 * round-to-nearest products and sum (no fused multiply-add).  1 <= k <=
 * min(N, 4096).  The first call allocates a plan-owned selection workspace.
 * Errors: GTT_ERR_INVALID_ARG (NULL or misaligned pointers, k out of range),
 * GTT_ERR_UNSUPPORTED (I32), GTT_ERR_ALLOC, GTT_ERR_CUDA.
 *
 * gtt_decompress -- the reconstruction: y = G_N^dagger s for every vector,
 * where s holds values[v*k + j] at index indices[v*k + j] and zero elsewhere
 * (indices outside [0, N) are skipped; of repeated indices one value is
 * kept; the result is not re-normalised).  y: device, batch*N elements.
 * Where the plan's first pass runs on contiguous tiles of the CUDA-core or
 * TMA pass kernels, that pass runs only on the tiles holding kept indices
 * (the same values); it uses the plan's selection workspace, so compress
 * and decompress calls of one plan on different streams must not overlap.  Same
 * errors.
 */
gtt_status_t gtt_compress(gtt_plan_t plan, const void *x, void *spectrum, long long k, long long *indices,
                          void *values, gtt_stream_t stream);
gtt_status_t gtt_decompress(gtt_plan_t plan, const long long *indices, const void *values, long long k, void *y,
                            gtt_stream_t stream);

/*
 * gtt_forward_host / gtt_inverse_host -- the same transforms on HOST buffers:
 * copy x (batch*N elements) to plan-owned device memory, transform, copy the
 * result back into y, and wait for `stream`.  Host buffers may be pageable;
 * page-locked buffers copy faster.  The device staging buffer is allocated on
 * the first call and kept by the plan.
 */
gtt_status_t gtt_forward_host(gtt_plan_t plan, const void *x_host, void *y_host,
                              gtt_stream_t stream);
gtt_status_t gtt_inverse_host(gtt_plan_t plan, const void *y_host, void *x_host,
                              gtt_stream_t stream);

/*
 * gtt_selftest_bounded_wait -- check, on the current device and without any
 * fault, that the bounded waits of the library's pipelined kernels give up:
 * one warp waits on an mbarrier that nothing arrives on, using the kernels'
 * try-wait primitive, for at most `polls` polls (1 .. 2^20), and reports the
 * expiry through a device flag, as the pass kernels do before
 * gtt_plan_check returns GTT_ERR_TIMEOUT.  *expired = 1 when the wait expired
 * (the expected outcome).  Synchronizes `stream`.  No counterpart in the paper.
 * Errors: GTT_ERR_INVALID_ARG (polls out of range, NULL expired),
 * GTT_ERR_ALLOC, GTT_ERR_CUDA.
 */
gtt_status_t gtt_selftest_bounded_wait(int polls, int *expired, gtt_stream_t stream);

/*
 * gtt_plan_describe -- write a one-line JSON description of the plan's
 * schedule (passes, digits per pass, run length, tile bytes, kernels
 * launched per transform) into buf (NUL-terminated, truncated to len).
 */
gtt_status_t gtt_plan_describe(gtt_plan_t plan, char *buf, size_t len);

/*
 * gtt_plan_set_timing -- when enable != 0, every kernel the plan launches is
 * bracketed by two CUDA events recorded on the launch stream.
 * gtt_plan_timing -- wait for the recorded events and write, as one line of
 * JSON, per kernel: its name, number of launches and summed device time (ms)
 * since the previous gtt_plan_timing call; then forget the records.
 */
gtt_status_t gtt_plan_set_timing(gtt_plan_t plan, int enable);
gtt_status_t gtt_plan_timing(gtt_plan_t plan, char *buf, size_t len);

/* ----------------------------------------------------------------------
 * Grouped transforms: many independent transforms of uneven b, n and dtype
 * (each y = W^{(x)n} x of Def. 2.3 with its own W) executed by ONE
 * persistent kernel launch, captured once in a CUDA graph.
 * -------------------------------------------------------------------- */
typedef struct {
    int b;              /* 2..8 or 16                                         */
    int n;              /* >= 1                                               */
    gtt_dtype_t dtype;  /* GTT_F32 or GTT_C64                                 */
    const void *W;      /* HOST, b*b elements row-major (copied at creation)  */
    const void *x;      /* device, N = b^n elements, 16-byte aligned          */
    void *y;            /* device, N elements, 16-byte aligned (may equal x)  */
    int inverse;        /* 0: y = G_N x;  1: y = G_N^dagger x (W^H)           */
} gtt_request_t;

/*
 * gtt_group_create -- plan `count` requests for one graph launch.  Each
 * distinct (b, n, dtype) gets its mode-group schedule from the autotune cache
 * (gtt_plan_autotune / GTT_AUTOTUNE_CACHE) or the fixed rule.  Work items are
 * (request, pass, tile); a pass of a request starts after the request's
 * previous pass (a bounded device-side wait; expiry raises GTT_ERR_TIMEOUT in
 * gtt_group_check).  Requests of 2 MiB or more run instead as a chain of
 * their shape's pass kernels (with their own W) on four side streams of the
 * same graph, beside the persistent kernel.  The pointers in the requests are fixed for the group's
 * lifetime.  Errors: GTT_ERR_INVALID_ARG, GTT_ERR_UNSUPPORTED (b or dtype
 * outside the supported set), GTT_ERR_ALLOC, GTT_ERR_CUDA.
 */
gtt_status_t gtt_group_create(gtt_group_t *out, int count, const gtt_request_t *reqs);
/* Run every request of the group: one graph launch (a counter reset, the
 * persistent kernel and the large requests' pass chains) on `stream`; the
 * graph is captured on the first call. */
gtt_status_t gtt_group_execute(gtt_group_t group, gtt_stream_t stream);
/* Wait for the device; GTT_ERR_TIMEOUT if a bounded wait expired (then cleared). */
gtt_status_t gtt_group_check(gtt_group_t group);
/* One-line JSON: requests, elements, work items, segments, grid, shared
 * memory, and the large requests run as pass chains (count, launches, streams). */
gtt_status_t gtt_group_describe(gtt_group_t group, char *buf, size_t len);
gtt_status_t gtt_group_destroy(gtt_group_t group);

/* Release the plan and everything it owns.  NULL is accepted. */
gtt_status_t gtt_plan_destroy(gtt_plan_t plan);

/* Message describing the last error raised on the calling thread ("" if none). */
const char *gtt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GTT_H_ */
