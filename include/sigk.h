/*
 * sigk.h -- C-ABI of the GB300 signature-kernel library (libsigk.so).
 *
 * What is computed.  For piecewise-linear paths x, y (sequences of points in
 * R^d, linearly interpolated), the signature kernel k(x,y) = K(1,1), where K
 * solves the Goursat problem  d^2K/(ds dt) = <x'(s), y'(t)> K  with K = 1 on
 * both axes (Sec. 2.1, Definition "Signature Kernel").  K is evaluated tile by
 * tile with the tile-centred local power series of Sec. 2.3 (Proposition
 * "tile-centred expansion", proof in App. A.6), swept over the tile grid in
 * anti-diagonal (wavefront) order (algorithm of App. C.1), with the boundary
 * data of each tile passed on as truncated polynomial coefficients.  Tile
 * (i,j) couples x-segment i with y-segment j; its coefficient is
 * c_ij = <x_{i+1} - x_i, y_{j+1} - y_j> (unit local tiles).
 *
 * Memory and ownership.  Every array argument is caller-owned DEVICE memory
 * (the library never allocates or frees device memory), except where a
 * parameter says "host".  Scratch comes from the caller through a workspace
 * (ws, ws_bytes) whose size sigk_workspace_size() returns; ws must be 256-byte
 * aligned and must not be used by another call that runs at the same time.
 *
 * Path batches.  A batch of n paths is one packed row-major FP32 array of
 * shape (sum_p len[p]) x d plus a DEVICE int64 vector len[n]: path p occupies
 * rows [off_p, off_p + len[p]) with off the exclusive prefix sum of len.  By
 * default a row is a POINT and len[p] counts points (>= 1; a path of one point
 * has no segment and k = 1 with every other path).  With
 * SIGK_FLAG_INCREMENTS a row is a segment increment and len[p] counts
 * segments (>= 0).  d is shared by all paths of a call, 1 <= d <= 8192
 * (d <= 16 keeps the increments in registers; larger d computes each strip's
 * coefficients first, see the kernel notes; sigk_backward: d <= 1024).
 *
 * Precision.  Inputs are FP32.  The series arithmetic is FP32 with a
 * float-float corner value and a per-edge power-of-two exponent; results are
 * FP64.  Accuracy is set by the truncation parameters in sigk_opts, which
 * sigk_plan() chooses from a target relative tolerance.
 *
 * Calls are asynchronous on `stream`.  The returned status covers argument
 * validation and launch; errors found on the device (a bounded wait that ran
 * out, non-finite data) are recorded in the workspace and returned by
 * sigk_sync_status() after the stream has drained.  No call throws.
 */
#ifndef SIGK_H
#define SIGK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIGK_OK = 0,
    SIGK_ERR_ARG = -1,        /* null pointer, bad size, d out of range, bad opts */
    SIGK_ERR_LENGTH = -2,     /* a length below its minimum or above 2^31-1 */
    SIGK_ERR_NONFINITE = -3,  /* NaN or Inf met on the device */
    SIGK_ERR_WORKSPACE = -4,  /* ws too small or misaligned */
    SIGK_ERR_CUDA = -5,       /* a CUDA runtime call failed (see sigk_last_error) */
    SIGK_ERR_TIMEOUT = -6,    /* a bounded inter-warp wait ran out on the device */
    SIGK_ERR_ACCURACY = -7,   /* sigk_plan: no order up to 16 meets the tolerance, even
                                 at the finest refinement tried (*opts_out still holds
                                 that finest plan) */
    SIGK_ERR_UNSUPPORTED = -8, /* a combination this library does not provide */
    SIGK_ERR_BOUNDS = -9      /* a device-side bounds check failed (only in a library
                                 built with SIGK_DEBUG, which checks every work item's
                                 buffer regions before touching them) */
} sigk_status;

/* Operation codes for sigk_workspace_size / sigk_plan. */
enum { SIGK_OP_PAIRS = 0, SIGK_OP_GRAM = 1, SIGK_OP_MMD = 2 };

/* opts flags */
enum {
    SIGK_FLAG_INCREMENTS = 1,  /* rows are increments, len counts segments */
    SIGK_FLAG_GRAM_FULL = 2,   /* Gram of X with itself: compute both triangles
                                  independently instead of mirroring */
    SIGK_FLAG_MMD_BIASED = 4,  /* MMD^2 V-statistic instead of the U-statistic */
    SIGK_FLAG_FP64 = 8,        /* solve every tile in FP64: point differences,
                                  the increment Gram, refinement scaling and the
                                  tile map (forward ops only; sigk_backward
                                  rejects it).  For ill-conditioned pairs --
                                  strong coupling over long paths, oscillating
                                  kernels -- whose FP32 result carries a
                                  rounding error above the tolerance.  FP64
                                  runs at 1/64 of the FP32 rate on this GPU. */
    SIGK_FLAG_PAIR_MAJOR = 16, /* schedule each pair's strips as consecutive
                                  work items (smaller seam ring) instead of the
                                  default strip-major order, where strip l of
                                  every pair is scheduled before strip l+1 of
                                  any, longest pairs first, whenever the ring
                                  for whole strips fits in 8 GiB.  Results are
                                  identical; only the schedule differs. */
    SIGK_FLAG_REPLAY = 32,     /* sigk_backward: never store the tile records;
                                  the adjoint replays every strip from its
                                  stored seam instead (smaller workspace, more
                                  arithmetic).  Results are identical. */
    SIGK_FLAG_NO_TENSOR = 128, /* d > 16: form the increment Gram with FP32 FMA
                                  (a register-blocked micro-GEMM, FP32 accuracy)
                                  instead of the tensor cores (exact 8-bit digit
                                  products accumulated on tcgen05, float-float
                                  accuracy; used for 16 < d <= 1024).  For
                                  comparisons. */
    SIGK_FLAG_TEST_WITHHOLD_SEAM = 64  /* fault-injection hook for tests of the
                                  bounded waits: in the inference forward of
                                  sigk_pairs / sigk_gram / sigk_mmd (d <= 16),
                                  the first work item of the schedule never
                                  publishes its outgoing seam, so the strip that
                                  consumes it waits until wait_ms runs out and
                                  the call reports SIGK_ERR_TIMEOUT through
                                  sigk_sync_status; its outputs are then
                                  undefined.  No other effect. */
};

/* Truncation and scheduling parameters.  NULL = defaults (order 8, rings 4,
 * max_len 8193, wait_ms 4000).
 *   order: degree P of the edge polynomials (the truncation order N of the
 *          coefficient matrices, App. A.7); supported 4..16, rounded up to an
 *          even value.
 *   rings: number n of Neumann iterations per tile (powers of c_ij kept,
 *          Sec. 2.3 / App. B: the local Neumann iteration), 1 <= n <= min(order, 8);
 *          compiled into the kernels: the FP32 solvers take 2..8, the FP64
 *          solver an even count (1 rounds up to 2, and odd counts round up
 *          under SIGK_FLAG_FP64).
 *   The FP32 solvers keep the entry c^m w B of the tile matrix (ring m,
 *   edge coefficient of degree k) when m <= n, m + k <= P and
 *   2m + k <= 2n + 1: a power of c counts twice against the degree of the
 *   edge data, as c (a product of two increments) is of the order of the
 *   square of a coupling or smaller.  No kept entry reaches a degree above
 *   2n, so these solvers run with P clamped to 2n (same results).  The FP64
 *   solver (SIGK_FLAG_FP64) keeps every entry with m <= n and p, q <= P.
 *   flags: SIGK_FLAG_*.
 *   grid_ctas: persistent grid size (0 = occupancy-derived, one wave).
 *   max_len: upper bound on the segments of the path that a pair sweeps
 *            (the longer path of a pair may be split over warps instead),
 *            counted after refinement; sizes the seam ring.  A pair that needs
 *            more fails with SIGK_ERR_LENGTH (reported by sigk_sync_status).
 *            0 = 8193.
 *   refine_c: 0 = off.  Otherwise every path p is refined: each of its
 *            segments is split into s_p equal collinear pieces, s_p = the
 *            power of two >= max_i |dz_i| / sqrt(refine_c) (at most 64), so that every
 *            tile satisfies |c| <= refine_c by Cauchy-Schwarz.  Exact (the
 *            kernel is invariant under collinear insertion); it trades more
 *            tiles for tiles the series resolves in FP32 (large |c| needs
 *            orders and rings beyond 16 and 8, and negative c cancels).
 *   wait_ms: budget of every bounded inter-warp wait on the device, in
 *            milliseconds (0 = 4000; at most 600000).  A wait that runs out
 *            records SIGK_ERR_TIMEOUT, with the waited address, target and last
 *            value seen in the workspace header, and makes every warp of the
 *            launch return.
 *   ring_tol: 0 = every tile keeps `rings` Neumann iterations.  Otherwise the
 *            tensor-core forward (16 < d <= 1024, FP32) chooses the count per
 *            tile, as the local Neumann iteration of App. B stops when the
 *            next term is negligible: a tile with coefficient c needs the
 *            smallest of 2, 4, 6, 8 (capped at rings) with
 *            |c|^(n+1) / ((n+1)!)^2 <= ring_tol
 *            (the first dropped ring, relative to the edge data), and the
 *            tiles a warp solves in one step use the largest count among them.
 *            sigk_plan sets it to tol / (100 L1 L2) of the largest pair, a
 *            tenth of an equal share of its ring-sum rule.
 *            sigk_ring_histogram reports the counts used.  (The d <= 16
 *            kernel keeps the fixed count: on its workloads every tile needs
 *            the planned count, and the per-step choice cost 10 %.) */
typedef struct {
    int order;
    int rings;
    int flags;
    int grid_ctas;
    int64_t max_len;
    float refine_c;
    int wait_ms;
    float ring_tol;
} sigk_opts;

/* [The one-strip memory of the wavefront sweep, App. C.1 and the O(l P)
 * memory statement of the complexity discussion, Sec. 3.]
 * Device workspace bytes needed by sigk_pairs/sigk_gram/sigk_mmd for the
 * given batch sizes (n_x, n_y = number of paths; for SIGK_OP_PAIRS n_x = n_y =
 * number of pairs; for SIGK_OP_GRAM pass n_y = 0 for a Gram of X with itself).
 * Depends on the lengths only through opts->max_len.  Returns 0 on bad
 * arguments. */
size_t sigk_workspace_size(int op, int64_t n_x, int64_t n_y, int d, const sigk_opts* opts);

/* [k(x,y) = K(1,1): Sec. 2.1, Definition "Signature Kernel"; solved tile by
 * tile with the tile-centred expansion, Sec. 2.3 / App. A.6; swept in
 * anti-diagonal order, App. C.1.]
 * k_out[p] = k(x_p, y_p) for n_pairs independent pairs (ragged lengths).
 * X, len_x describe the x_p, Y, len_y the y_p (each a batch of n_pairs
 * paths).  k_out: device FP64[n_pairs]. */
sigk_status sigk_pairs(const float* X, const int64_t* len_x, const float* Y,
                       const int64_t* len_y, int64_t n_pairs, int d, double* k_out,
                       void* ws, size_t ws_bytes, void* stream, const sigk_opts* opts);

/* [The Gram matrix of App. A.7 (Proposition on the truncated Gram matrix)
 * and of the kernel experiments of Sec. 3.]
 * Gram matrix G[a*n_y + b] = k(x_a, y_b), row-major device FP64[n_x*n_y].
 * Y == NULL (and n_y ignored) means Y = X: G is n_x x n_x; unless
 * SIGK_FLAG_GRAM_FULL, only a <= b is computed and mirrored. */
sigk_status sigk_gram(const float* X, const int64_t* len_x, int64_t n_x, const float* Y,
                      const int64_t* len_y, int64_t n_y, int d, double* G, void* ws,
                      size_t ws_bytes, void* stream, const sigk_opts* opts);

/* [The paper has no MMD: a reduction of the Gram blocks of Sec. 2.1's
 * kernel, computed in FP64.]
 * Signature-kernel MMD^2 between samples X (m paths) and Y (n paths):
 * mean_{a!=b} k(x_a,x_b) + mean_{a!=b} k(y_a,y_b) - 2 mean k(x_a,y_b)
 * (U-statistic; SIGK_FLAG_MMD_BIASED: V-statistic with all terms), reduced in
 * FP64 on the device.  mmd2_out: device FP64[1]; gram_out (optional, device
 * FP64[(m+n)^2]) receives the Gram of the concatenated sample [X; Y]. */
sigk_status sigk_mmd(const float* X, const int64_t* len_x, int64_t m, const float* Y,
                     const int64_t* len_y, int64_t n, int d, double* mmd2_out,
                     double* gram_out, void* ws, size_t ws_bytes, void* stream,
                     const sigk_opts* opts);

/* [The checkpointed wavefront boundaries of the adjoint; no counterpart in
 * the paper.]
 * Workspace bytes for sigk_backward (same arguments as sigk_workspace_size).
 * Includes the forward seam store, which needs up to
 * n_pairs * (ceil(max_len/32) - 1) * max_len * (order + 4) floats, and,
 * unless SIGK_FLAG_REPLAY is set, the store of tile records when it takes at
 * most 128 GiB: n_pairs * ceil(max_len/32) * (max_len + 32) * 32 * R floats,
 * R = 4 * floor((order + 6) / 4) (one record per tile: the tile's incoming
 * left edge and its exponent decisions, written by the forward and read back
 * by the adjoint). */
size_t sigk_backward_workspace_size(int op, int64_t n_x, int64_t n_y, int d, const sigk_opts* opts);

/* Gradients by the adjoint of the solver (reverse-mode differentiation of the
 * truncated FP32 scheme; the paper has no gradient -- this is the adjoint of
 * the tile map of Sec. 2.3 swept in reverse wavefront order).
 * The call runs a training forward that stores the right-edge seam of every
 * 32-row strip (checkpointed wavefront boundaries) and, for d <= 16 when they
 * fit the budget above, every tile's record; then the adjoint kernel, which
 * per strip forms the strip's coefficients, replays the strip from its stored
 * seam (only when the records were not stored), sweeps it in reverse --
 * rebuilding every tile's inputs by inverting the tile's bottom-to-top update
 * -- and chains dk/dc_ij to the increments with two contractions over the
 * strip.  d <= 1024 (FP32 coefficients).
 *   op, X, len_x, n_x, Y, len_y, n_y, d: as in sigk_pairs / sigk_gram /
 *     sigk_mmd (SIGK_OP_GRAM with Y == NULL: Gram of X with itself).
 *   grad_out (device FP64): upstream gradient of the op's output --
 *     [n_pairs] (PAIRS), [n_x * n_y] row-major (GRAM; n_x * n_x when
 *     Y == NULL), [1] (MMD).
 *   grad_X, grad_Y (device FP32, same layout as X and Y, or NULL to skip):
 *     OVERWRITTEN with dL/dX, dL/dY (L = <grad_out, output>); gradients are
 *     with respect to the points, or to the increments with
 *     SIGK_FLAG_INCREMENTS.  For a Gram of X with itself only grad_X is used.
 *   value_out (device FP64): receives the forward output (k values, Gram,
 *     or MMD^2); required for PAIRS and GRAM, optional for MMD.
 * Errors on the device are reported by sigk_sync_status. */
sigk_status sigk_backward(int op, const float* X, const int64_t* len_x, int64_t n_x,
                          const float* Y, const int64_t* len_y, int64_t n_y, int d,
                          const double* grad_out, float* grad_X, float* grad_Y,
                          double* value_out, void* ws, size_t ws_bytes, void* stream,
                          const sigk_opts* opts);

/* [Adjoint of the tile map of Sec. 2.3, as sigk_backward.]
 * The two halves of sigk_backward, for callers that keep the forward's state
 * until the upstream gradient is known (an autograd forward, then its
 * backward).  sigk_forward_train is the training forward of sigk_backward: it
 * writes the op's output to value_out (as sigk_backward does) and leaves the
 * stored seams and tile records in ws.  sigk_adjoint then runs the adjoint
 * from that state: same op, n_x, n_y (0 for a Gram of X with itself), d and
 * opts; ws, ws_bytes (sigk_backward_workspace_size), X, Y and their lengths
 * unchanged since the forward.  grad_out, grad_X, grad_Y as in sigk_backward
 * (gradients are overwritten).  sigk_adjoint reads what the forward wrote
 * on the device: give it the same stream, or one ordered after the forward.
 * It may run again on the same state with another grad_out.  The workspace
 * carries a signature of the training forward (op, sizes, options, layout);
 * if it does not hold a successful training forward of this call's
 * arguments, sigk_adjoint touches nothing and sigk_sync_status reports
 * SIGK_ERR_ARG.  Errors on the device are reported by sigk_sync_status. */
sigk_status sigk_forward_train(int op, const float* X, const int64_t* len_x, int64_t n_x,
                               const float* Y, const int64_t* len_y, int64_t n_y, int d,
                               double* value_out, void* ws, size_t ws_bytes, void* stream,
                               const sigk_opts* opts);
sigk_status sigk_adjoint(int op, int64_t n_x, int64_t n_y, int d, const double* grad_out,
                         float* grad_X, float* grad_Y, void* ws, size_t ws_bytes, void* stream,
                         const sigk_opts* opts);

/* Same result as sigk_pairs, for callers that cannot allocate device memory
 * (code that runs where cudaMalloc is not allowed or not wanted: inside a
 * region governed by someone else's memory pool or allocator, or a runtime
 * that forbids side allocations).  The paper has no counterpart: this is an
 * interface convenience.  It takes no workspace: its scratch is a fixed
 * 32 MiB device array inside libsigk.so, which every GPU that loads the
 * library holds until the process exits.  It calls no cudaMalloc, cudaFree
 * or other allocating routine.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture on the device.
 *   - Problems whose scratch does not fit in 32 MiB (many pairs, long swept
 *     paths, high order) are rejected with SIGK_ERR_WORKSPACE before any
 *     launch; use sigk_pairs with a caller workspace for those.
 *   - All calls share the one array, and each call resets the parts that must
 *     start at zero; calls that overlap on the GPU (different streams, or
 *     different host threads) race on it and must be serialised by the caller.
 * Device-side errors are read back with sigk_static_sync_status. */
sigk_status sigk_pairs_static(const float* X, const int64_t* len_x, const float* Y,
                              const int64_t* len_y, int64_t n_pairs, int d, double* k_out,
                              void* stream, const sigk_opts* opts);

/* [No counterpart in the paper.]  sigk_sync_status for the static scratch of
 * sigk_pairs_static. */
sigk_status sigk_static_sync_status(void* stream);

/* A-priori truncation choice (App. C.3: order search from the largest
 * coupling in the grid).  Runs the planner and a statistics kernel on the
 * device that forms every tile coefficient of the pair table (a strip
 * micro-GEMM, nothing stored) and reduces them per pair to the largest |c|,
 * the ring sums sum |c|^m (m = 2..9) and the couplings C = max over rows and
 * columns of |<dx_i, y_J - y_0>| and |<x_I - x_0, dy_j>| (the size of the
 * edge coefficients, a_p ~ C^p/(p!)^2); then picks the smallest order P and
 * rings n >= 2 with max(L1,L2) C^(P+1)/((P+1)!)^2 <= tol/10 and
 * sum|c|^(n+1)/((n+1)!)^2 <= tol/4 (the ring sum adds the dropped terms of
 * all tiles as if coherent, which overstates the measured truncation error
 * 3-4 times on Brownian Grams), and raises n until 2n >= P - 4, so
 * that the FP32 truncation (see order above) reaches degree P - 4 or more.
 * If a tile has |c| > 1 or no order up
 * to 16 fits, it sets refine_c = 1, 1/4, ... and plans the refined problem.
 * Synchronises `stream`.  Writes into *opts_out (other fields copied from
 * opts_in when given; max_len raised to the longest swept path, refined).
 * Returns SIGK_ERR_ACCURACY, with *opts_out written, when the rule is not met
 * even at the finest refinement tried (or at the caller's refine_c).
 * When the tuning cache (sigk_autotune) holds the planned call's shape class,
 * its layout (grid_ctas, schedule and Gram-path flags) is merged into
 * *opts_out. */
sigk_status sigk_plan(int op, const float* X, const int64_t* len_x, int64_t n_x,
                      const float* Y, const int64_t* len_y, int64_t n_y, int d, double tol,
                      void* ws, size_t ws_bytes, void* stream, const sigk_opts* opts_in,
                      sigk_opts* opts_out);

/* Autotuner of the launch layout (the paper has no counterpart: its JAX
 * implementation has one fixed layout).  With the truncation fixed by
 * opts_in (order, rings, refinement, ring tolerance), it times the op
 * (SIGK_OP_PAIRS / GRAM / MMD, arguments as in sigk_pairs / sigk_gram /
 * sigk_mmd) under each candidate layout on the caller's inputs -- persistent
 * grid of the full occupancy, 3 or 2 CTAs per SM (the wavefront's width);
 * strip-major or pair-major schedule; and, when allow_fma_gram is non-zero
 * and 16 < d <= 1024, the FP32 FMA increment Gram instead of the tensor-core
 * one (FP32 instead of float-float coefficients) -- with CUDA events on
 * `stream` (one warm-up and two timed calls each; synchronises it).  The
 * fastest goes to *opts_out (grid_ctas and the flags SIGK_FLAG_PAIR_MAJOR,
 * SIGK_FLAG_NO_TENSOR; every other field as opts_in), its time per call to
 * *ms_out, and into the library's in-process cache under the call's shape
 * class (sigk_tune_key), which sigk_plan consults.  out_scratch: device FP64
 * output of the op's size (k values, Gram or MMD^2).  Candidates whose
 * workspace exceeds ws_bytes are skipped; SIGK_ERR_WORKSPACE if none fits. */
sigk_status sigk_autotune(int op, const float* X, const int64_t* len_x, int64_t n_x,
                          const float* Y, const int64_t* len_y, int64_t n_y, int d,
                          double* out_scratch, void* ws, size_t ws_bytes, void* stream,
                          const sigk_opts* opts_in, int allow_fma_gram, sigk_opts* opts_out,
                          double* ms_out);

/* [No counterpart in the paper.]
 * Shape class of a call (host only): op, batch sizes, d, the swept-length
 * bound rounded up to a power of two, order, rings and the problem flags, as
 * a string into buf (>= 96 bytes). */
sigk_status sigk_tune_key(int op, int64_t n_x, int64_t n_y, int d, const sigk_opts* opts,
                          char* buf, size_t buf_len);

/* [No counterpart in the paper.]
 * The tuning cache (host only, shared by the process's threads):
 * put stores a class's layout (grid_ctas, the flags SIGK_FLAG_PAIR_MAJOR and
 * SIGK_FLAG_NO_TENSOR of `flags`, time); get merges a stored layout into
 * *opts (SIGK_ERR_ARG when the class is absent); save writes the cache as
 * text, one class per line; load adds a saved file's classes. */
sigk_status sigk_tune_cache_put(const char* key, int grid_ctas, int flags, double ms);
sigk_status sigk_tune_cache_get(const char* key, sigk_opts* opts, double* ms);
sigk_status sigk_tune_cache_save(const char* path);
sigk_status sigk_tune_cache_load(const char* path);
int64_t sigk_tune_cache_size(void);
void sigk_tune_cache_clear(void);

/* [No counterpart in the paper: the bounded waits of the persistent
 * wavefront.]
 * Waits for `stream`, then returns and clears the device status recorded in
 * ws by earlier calls: SIGK_OK; SIGK_ERR_TIMEOUT, SIGK_ERR_LENGTH or
 * SIGK_ERR_BOUNDS, after which the call's outputs are undefined (the launch
 * stopped); or SIGK_ERR_NONFINITE, when some output is NaN or infinite (from
 * non-finite input data, or beyond the exponent range), in which case every
 * other output is valid. */
sigk_status sigk_sync_status(void* ws, size_t ws_bytes, void* stream);

/* [Tiles of the App. C.1 sweep, for the work accounting.]
 * Counters of the last call on this workspace (synchronises `stream`):
 * out[0] = tiles solved by the forward, out[1] = lane-tiles including strip
 * padding, out[2] = tiles solved by the adjoint kernel, out[3] = tiles the
 * adjoint kernel replayed (0 when the forward stored the tile records). */
sigk_status sigk_counters(void* ws, size_t ws_bytes, void* stream, double* out4);

/* [The per-tile Neumann iteration counts of App. B.]
 * Tiles solved by the last forward on this workspace with at most 2, 3-4,
 * 5-6 and 7-8 Neumann rings (out4[0..3]; synchronises `stream`); all zero
 * unless opts->ring_tol was set. */
sigk_status sigk_ring_histogram(void* ws, size_t ws_bytes, void* stream, double* out4);

/* [No counterpart in the paper.]
 * Launch configuration the library would use for these arguments (host
 * query, no launch): out6 = {persistent grid (CTAs), CTAs per SM from the
 * occupancy query, threads per CTA, dynamic shared memory bytes per CTA, rows
 * per lane, kernel family (0: d <= 16 register kernel, 1: FMA two-phase,
 * 2: tensor-core)}; with train != 0, the adjoint kernel's. */
sigk_status sigk_launch_info(int op, int64_t n_x, int64_t n_y, int d, const sigk_opts* opts,
                             int train, int* out6);

/* [No counterpart in the paper.]
 * Profiling hook: when both are non-NULL, later calls on this host thread
 * record the two CUDA events (cudaEvent_t) on the call's stream immediately
 * before and after the solver kernel launch, so that a caller can time the
 * solver alone.  Pass NULL, NULL to stop. */
void sigk_profile_events(void* ev_start, void* ev_stop);

/* [No counterpart in the paper.]  Thread-local message for the last error
 * returned on this host thread. */
const char* sigk_last_error(void);

/* [No counterpart in the paper.]  Library version string. */
const char* sigk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SIGK_H */
