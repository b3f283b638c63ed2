/*
 * iccg.h -- C ABI of the GB300 block-multicolor ICCG library (libiccg.so).
 *
 * The library solves A x = b for a sparse SPD matrix A with the conjugate
 * gradient method preconditioned by IC(0), whose forward and backward
 * substitutions run in block-multicolor order: colors one after another,
 * the blocks of one color in parallel, the rows of a block in order
 * (Suzuki, "Comparison of Algebraic Block Multi-Coloring and Leiden Methods
 * for Parallel Preconditioning in the ICCG Method", Sec. 3 and Alg. 1).
 *
 * General conventions
 *   - Every function returns an iccg_status and never aborts or traps.
 *   - Sparse matrices are CSR: rowptr int64[n+1], colind int32[nnz] (0-based),
 *     val double[nnz]; both triangles stored, a diagonal entry in every row,
 *     symmetric pattern.  nnz must be below 2^31.
 *   - Vectors are in the caller's (original) row numbering; the library
 *     applies the block-multicolor permutation internally.
 *   - Array arguments of iccg_setup / iccg_solve / iccg_precond / iccg_spmv
 *     may be host or device pointers (the library asks the CUDA runtime which
 *     one it got).  The caller owns them; the library copies what it keeps.
 *   - All device work of a context runs on the stream given to iccg_setup.
 *     Calls on one context must not overlap; separate contexts are
 *     independent.
 *   - Host helpers (iccg_block_*, iccg_color_order) take host pointers only.
 */
#ifndef ICCG_H_
#define ICCG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iccg_ctx iccg_ctx;   /* opaque; owned by the library */
typedef void *iccg_stream_t;        /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  ICCG_OK = 0,
  ICCG_ERR_ARG = 1,           /* invalid argument (sizes, CSR, permutation, pointers) */
  ICCG_ERR_COLORING = 2,      /* two blocks of one color share an edge */
  ICCG_ERR_BREAKDOWN = 3,     /* IC(0) pivot not positive; see iccg_last_error */
  ICCG_NOT_CONVERGED = 4,     /* maxit reached; x and the history are valid */
  ICCG_ERR_CUDA = 5,          /* a CUDA runtime call failed; see iccg_last_error */
  ICCG_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  ICCG_ERR_NONFINITE = 7,     /* NaN/Inf met in the iteration */
  ICCG_ERR_UNIMPLEMENTED = 8,
  ICCG_ERR_STATE = 9          /* call order violated (e.g. solve before factor) */
} iccg_status;

typedef struct {
  int32_t precond_fp32;       /* 1: IC factors and substitutions stored and run in FP32
                                 with FP32 accumulation; IC(0) itself, the CG dots,
                                 alpha/beta and the x/r updates stay FP64 */
  int32_t warps_per_cta;      /* warps per CTA of the substitution kernels (a lane-tile
                                 CTA uses at most one warp per step); 1..16; 0 = 8,
                                 and 4 for the pair kernels (colors of two-row blocks) */
  int32_t rows_per_thread;    /* a group (the work of one CTA) holds up to
                                 32 * warps_per_cta * rows_per_thread rows of whole
                                 blocks; 1, 2, 4, 8, 16 or 32; 0 = 1 */
  int32_t no_graph;           /* 1: drive the PCG loop from the host instead of a
                                 CUDA graph with a device-side WHILE condition */
  int32_t no_pdl;             /* 1: launch kernels without programmatic dependent
                                 launch (no overlap of a kernel's prologue with the
                                 tail of the previous one) */
  int32_t solver;             /* ICCG_SOLVER_PHASED: one launch per phase (p update,
                                 SpMV, each color), the PCG loop a CUDA graph;
                                 ICCG_SOLVER_PERSISTENT: the whole solve in one
                                 cooperative launch whose phases are separated by
                                 grid barriers (groups only, no lane tiles);
                                 ICCG_SOLVER_AUTO (0) = phased */
  int32_t lane_block_max;     /* a color whose blocks all have at most this many rows
                                 runs one block per lane of a warp (32 blocks per
                                 warp, the block's rows in order); other colors run
                                 one CTA per group of blocks, level by level; 1..32,
                                 0 = 32, -1 = never (the persistent solver never
                                 uses lanes) */
  int32_t tile_mapping;       /* colors whose blocks have at most lane_block_max rows:
                                 ICCG_TILES_UNITS runs every such color as warp units
                                 (one warp per block, a lane per row, the in-block
                                 recurrence as a shuffle-broadcast column sweep;
                                 blocks of up to 1, 2, 4, 8 or 16 rows share a warp);
                                 lane tiles (32 blocks, one per
                                 lane): ICCG_TILES_CTA runs one CTA per tile (the
                                 tile's steps shared out over its warps, the in-block
                                 recurrence on one warp); ICCG_TILES_WARP one warp
                                 per tile (all steps in order, many tiles per CTA);
                                 ICCG_TILES_PAIR: colors of blocks of one or two rows
                                 one warp per tile with the block's rows in registers
                                 (pair kernels), other colors one CTA per tile;
                                 ICCG_TILES_AUTO (0): warp units for colors whose
                                 largest block has 5..32 rows, pair kernels for the
                                 colors whose blocks all have two rows, one CTA per
                                 tile otherwise */
  int32_t fuse_sweep;         /* layouts whose colors are all lane tiles of blocks of
                                 one or two rows: 1 runs each preconditioner sweep
                                 (every color forward and backward) as one
                                 cooperative launch with bounded grid barriers
                                 between colors (a wait longer than the limit of
                                 iccg_set_wait_limit ends the solve with
                                 ICCG_ERR_TIMEOUT); 2 runs only the tail of each
                                 sweep that way (the last colors, together at most
                                 n/32 rows, when they are such lane tiles: forward,
                                 fused and backward in one launch of one CTA per SM);
                                 0 (default) or -1 one launch per color; other
                                 layouts ignore it */
} iccg_opts;

enum { ICCG_SOLVER_AUTO = 0, ICCG_SOLVER_PERSISTENT = 1, ICCG_SOLVER_PHASED = 2 };
enum { ICCG_TILES_AUTO = 0, ICCG_TILES_CTA = 1, ICCG_TILES_WARP = 2, ICCG_TILES_PAIR = 3, ICCG_TILES_UNITS = 4 };

/* ------------------------------------------------------------------------
 * iccg_setup -- Sec. 3: the block-multicolor ordering renumbers rows color
 * by color, block by block; Alg. 1 then processes colors in sequence and the
 * blocks of a color in parallel.
 *
 *   ctx        out: new context (NULL on error)
 *   n, nnz     matrix order and stored entries (0 <= n, 0 <= nnz < 2^31)
 *   rowptr, colind, val   CSR of A in the original numbering
 *   perm       int32[n], perm[new] = old; a bijection on [0, n)
 *   block_ptr  int32[n_b+1], rows of block j are new rows
 *              [block_ptr[j], block_ptr[j+1]); strictly increasing, 0 .. n
 *   color_ptr  int32[n_c+1], blocks of color c are [color_ptr[c],
 *              color_ptr[c+1]); strictly increasing, 0 .. n_b
 *   opts       NULL = defaults
 *   stream     the CUDA stream all work of this context uses
 *
 * Checks the CSR (sorted or not, in range, diagonal present, symmetric
 * pattern), the permutation and pointer arrays, and the coloring invariant
 * that no stored entry joins two different blocks of one color
 * (ICCG_ERR_COLORING, offending block in iccg_last_error).  Copies the
 * permuted matrix and the per-color tile layout to the device.
 * ------------------------------------------------------------------------ */
iccg_status iccg_setup(iccg_ctx **ctx, int32_t n, int64_t nnz,
                       const int64_t *rowptr, const int32_t *colind, const double *val,
                       const int32_t *perm, const int32_t *block_ptr, const int32_t *color_ptr,
                       int32_t n_b, int32_t n_c, const iccg_opts *opts, iccg_stream_t stream);

/* ------------------------------------------------------------------------
 * iccg_factor -- Sec. 3: IC(0) with zero fill-in of the reordered matrix,
 * L L^T form (Alg. 1 divides by L_ii): L has the pattern of tril(A_hat) and
 * (L L^T)_ij = a_hat_ij on it.  Runs on the device in FP64, color by color
 * like Alg. 1.  A pivot that is not positive (or not finite) returns
 * ICCG_ERR_BREAKDOWN; iccg_last_error gives the first such row in the
 * original numbering.  May be called again (recomputes the same factor).
 * ------------------------------------------------------------------------ */
iccg_status iccg_factor(iccg_ctx *ctx);

/* ------------------------------------------------------------------------
 * iccg_solve -- preconditioned CG (Sec. 1) with the IC(0) preconditioner
 * applied by block-multicolor forward/backward substitution (Alg. 1 and the
 * reverse sweep described after it); stops when ||r||_2/||b||_2 <= tol
 * (Sec. 4 uses tol = 1e-8) with r the recursively updated residual.
 *
 *   b          double[n], right-hand side (host or device)
 *   x          double[n], in: x0, out: solution (host or device)
 *   tol, maxit stopping tolerance (>= 0) and iteration cap (>= 0)
 *   iters      host int32*, out: iterations done (may be NULL)
 *   res_hist   host double[maxit+1], out: ||r_k||/||b|| for k = 0..iters
 *              (may be NULL)
 *
 * b = 0 gives x = 0 and 0 iterations.  Returns ICCG_NOT_CONVERGED when maxit
 * is reached (x and history valid) and ICCG_ERR_NONFINITE on NaN/Inf.
 * Requires a successful iccg_factor.  The persistent solver (opts.solver =
 * ICCG_SOLVER_PERSISTENT; the default is the phased solver) returns
 * ICCG_ERR_TIMEOUT when a grid-barrier wait gave up (a phase longer than the
 * wait limit, 4 s unless iccg_set_wait_limit set another); the context stays
 * usable and the phased solver has no device-side waits.
 * ------------------------------------------------------------------------ */
iccg_status iccg_solve(iccg_ctx *ctx, const double *b, double *x, double tol, int32_t maxit,
                       int32_t *iters, double *res_hist);

/* z = (L L^T)^{-1} r with the block-multicolor substitutions (Alg. 1 and the
 * backward sweep); r, z double[n] in the original numbering. */
iccg_status iccg_precond(iccg_ctx *ctx, const double *r, double *z);

/* q = A p with the library's SpMV kernel (Table 8's SpMV phase); p, q
 * double[n] in the original numbering. */
iccg_status iccg_spmv(iccg_ctx *ctx, const double *p, double *q);

/* Copy the IC(0) factor of the permuted matrix to host arrays laid out as
 * the lower triangle of A_hat in CSR order (columns ascending, diagonal last
 * in each row): lval double[nnz_lower]; *nnz_lower receives the count (pass
 * lval = NULL to query it). */
iccg_status iccg_get_factor(iccg_ctx *ctx, double *lval, int64_t *nnz_lower);

/* Per-phase device time of one solve.  ms[6] receives the summed
 * milliseconds of: 0 init, 1 p update + SpMV, 2 forward colors, 3 fused last
 * color, 4 backward colors (with the closing reduction), 5 everything (CUDA
 * events around the solve); launches[6] the number of kernel launches (phased
 * solver: host-driven loop, one event pair around every kernel) or of grid
 * barriers (persistent solver: the time each barrier is left, recorded on the
 * device).  Same arguments and results as iccg_solve. */
iccg_status iccg_profile_solve(iccg_ctx *ctx, const double *b, double *x, double tol,
                               int32_t maxit, int32_t *iters, double *ms, int64_t *launches);

/* Device time of the SpMV phase as a PCG iteration of iccg_solve launches it
 * (p = z + beta p, then q = A p with <p,q>: Table 8's "SpMV" part of an
 * iteration), averaged over `reps` back-to-back launches on the context's
 * stream after one warm-up (CUDA events, same launch attributes as the
 * solve).  *ms receives milliseconds per phase.  Requires iccg_factor;
 * overwrites the context's solve vectors (the next iccg_solve starts from its
 * own inputs, so results are unaffected). */
iccg_status iccg_time_spmv_phase(iccg_ctx *ctx, int32_t reps, double *ms);

/* Layout facts of a context, out[18]: n, nnz, n_b, n_c, number of groups (a
 * group = consecutive whole blocks of one color, at most 32 * warps_per_cta *
 * rows_per_thread rows, or one larger block; one CTA each), number of groups
 * too large for the shared-memory plan, strictly-lower entries nL, deepest
 * in-group level count, largest group (rows), number of lane tiles (32
 * blocks, one per lane), number of colors run as lane tiles, number of
 * those run one warp per tile and as pair kernels (tile_mapping), number of
 * colors run as warp units, 1 when each sweep is one cooperative launch,
 * then the library's kernel launches: of one iccg_factor (one per in-block
 * level of the lane-tile and warp-unit colors, one per group color, and the
 * finishing pass), of one PCG iteration of iccg_solve (p update, SpMV and the
 * sweep's color launches), and of an iccg_solve's start and end (input
 * permutation, residual SpMV, the first sweep, output permutation). */
iccg_status iccg_info(const iccg_ctx *ctx, int64_t out[18]);

/* Wall-time limit (ns) of every device-side wait of this context: the grid
 * barriers of the persistent solver and of the cooperative sweep
 * (opts.fuse_sweep; Alg. 1's colors are separated by one barrier each
 * there).  A wait that runs past it makes the kernel stop at once and
 * iccg_solve return ICCG_ERR_TIMEOUT; the context stays usable.  0 restores
 * the default (4 s).  Per-color launches have no device-side waits. */
iccg_status iccg_set_wait_limit(iccg_ctx *ctx, uint64_t wait_ns);

iccg_status iccg_last_error(const iccg_ctx *ctx, int64_t *row_or_block, const char **msg);
void iccg_destroy(iccg_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batched solve (extension: many systems, several right-hand sides each, in
 * one launch).  Each system is the ICCG of iccg_solve (Alg. 1 substitutions
 * inside standard PCG) run for all its right-hand sides at once; the systems
 * are independent.  The whole solve is one cooperative kernel launch (the
 * PCG loop runs inside it) replayed as a CUDA graph.
 *
 *   iccg_batch_create  ctxs[nsys]: factored contexts on one device, all with
 *                      the same precond_fp32, set up with lane_block_max = -1
 *                      (CTA-group layout, blocks of at most 64 rows); the
 *                      batch borrows them (destroy the batch first) and runs
 *                      on ctxs[0]'s stream.  nrhs in 1..32.  opts may be NULL
 *                      (warps_per_cta 0 = 8, ctas_per_sm 0 = as many as fit,
 *                      autotune 1 = time every candidate shape on a short
 *                      solve and keep the fastest, reserved must be 0).
 *                      Errors: ICCG_ERR_ARG (arguments, layouts), ICCG_ERR_STATE
 *                      (a context not factored), ICCG_ERR_CUDA.
 *   iccg_batch_solve   B[s], X[s]: double[nrhs * n_s], right-hand side j of
 *                      system s at B[s][j * n_s ..] in the original numbering
 *                      (host or device); X[s] holds x0 on entry and x on
 *                      return.  Stops each right-hand side at ||r||/||b|| <=
 *                      tol or maxit iterations.  iters / status (may be NULL):
 *                      int32[nsys * nrhs]; res_hist (may be NULL, or entries
 *                      NULL): res_hist[s] = host double[(maxit + 1) * nrhs],
 *                      entry (k, j) = ||r_k||/||b|| of right-hand side j (0
 *                      past its last iteration).  Returns ICCG_OK when every
 *                      right-hand side converged, else the worst status.
 *   iccg_batch_tune    re-runs the shape search: every candidate (warps per
 *                      CTA x CTAs per SM x CTA-split exponent, then rows per
 *                      thread 1 / 2 / 4 at the best of those) solves B (as in
 *                      iccg_batch_solve, from x0 = 0, to tol / maxit; host or
 *                      device), or, with B = NULL, random right-hand sides for
 *                      20 iterations; the fastest is kept and *best_ms (may be
 *                      NULL) gets its time.
 *   iccg_batch_set_wait_limit  wall-time limit (ns) of the per-system barrier
 *                      waits inside the batched kernel (0: the default, 4 s);
 *                      a system whose wait runs out stops and its right-hand
 *                      sides report ICCG_ERR_TIMEOUT; the batch stays usable.
 *   iccg_batch_info    out[7]: warps per CTA, CTAs per SM, grid, padded nrhs,
 *                      largest block, 3 x the exponent e of the CTA split
 *                      (CTAs per system proportional to n^e; e = 1 or 4/3,
 *                      chosen by the tuner with the shape), rows per thread
 *                      (consecutive rows a chain of right-hand-side lanes takes
 *                      per pass of the SpMV and the p update).
 * The paper has no batched solver; this serves many independent systems
 * (e.g. the learned-blocking sweep) and multiple right-hand sides.
 * ------------------------------------------------------------------------ */
typedef struct iccg_batch iccg_batch;
typedef struct {
  int32_t warps_per_cta;
  int32_t ctas_per_sm;
  int32_t autotune;
  int32_t rows_per_thread;    /* 0 (1), 1, 2 or 4 */
  int32_t reserved[4];
} iccg_batch_opts;

iccg_status iccg_batch_create(iccg_batch **batch, iccg_ctx *const *ctxs, int32_t nsys, int32_t nrhs,
                              const iccg_batch_opts *opts);
iccg_status iccg_batch_solve(iccg_batch *batch, const double *const *B, double *const *X, double tol,
                             int32_t maxit, int32_t *iters, int32_t *status, double *const *res_hist);
iccg_status iccg_batch_tune(iccg_batch *batch, const double *const *B, double tol, int32_t maxit,
                            double *best_ms);
iccg_status iccg_batch_set_wait_limit(iccg_batch *batch, uint64_t wait_ns);
iccg_status iccg_batch_info(const iccg_batch *batch, int32_t out[7]);
iccg_status iccg_batch_last_error(const iccg_batch *batch, const char **msg);
void iccg_batch_destroy(iccg_batch *batch);

/* ------------------------------------------------------------------------
 * iccg_spmv_dot_noalloc -- q = A p and *pq = <p, q> with no device
 * allocation at all.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory where they need the
 * product (latency-critical loops that must not meet the allocator's
 * implicit device synchronisation, host frameworks that own all device
 * memory through their own pool and forbid allocations behind their back).
 *
 *   n                       rows, 0 <= n <= ICCG_NOALLOC_MAX_ROWS (else ICCG_ERR_ARG)
 *   rowptr, colind, val     CSR of A (int64 rowptr, int32 colind, FP64), DEVICE pointers
 *   p                       double[n] device input;  q  double[n] device output
 *   pq                      one double, device output
 *   stream                  the CUDA stream to run on; it must belong to the
 *                           current device (else ICCG_ERR_ARG, nothing launched)
 *
 * Scratch (one partial per CTA and the reduction's arrival counters, about
 * 137 KB) is a fixed array in the library's device image, held by every GPU
 * that loads the library until the process exits.  All calls share it: the
 * counters are cleared at the start of every call, and two calls whose work
 * overlaps on the GPU race and give wrong results.  The first call on each
 * device looks up the array's address (cudaGetSymbolAddress) and caches it.
 * The sum is deterministic (fixed order).
 * ICCG_ERR_CUDA when a CUDA call of this entry point failed (an error left
 * pending by earlier unrelated work is not consumed).
 * ------------------------------------------------------------------------ */
#define ICCG_NOALLOC_MAX_ROWS 4194304
iccg_status iccg_spmv_dot_noalloc(int32_t n, const int64_t *rowptr, const int32_t *colind,
                                  const double *val, const double *p, double *q, double *pq,
                                  iccg_stream_t stream);

/* ------------------------------------------------------------------------
 * Host-side blocking helpers (production implementations; host pointers).
 * ------------------------------------------------------------------------ */

/* Adjacency graph of A (Sec. 3): undirected, edge {i,j} iff i != j and a_ij
 * or a_ji is stored.  gptr int64[n+1]; gadj int32[*m] neighbours ascending.
 * Pass gadj = NULL to get *m (2 x edges) only. */
iccg_status iccg_graph(int32_t n, const int64_t *rowptr, const int32_t *colind,
                       int64_t *gptr, int32_t *gadj, int64_t *m);

/* ABMC blocking (Sec. 3; block size s = ceil(n/n_b), Sec. 5.1): a seed is
 * taken among the unassigned nodes and its neighbours are added from a FIFO
 * candidate set until the block has s nodes; an empty candidate set is
 * refilled with the smallest unassigned node.  block_of int32[n]. */
iccg_status iccg_block_abmc(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t s,
                            int32_t *block_of, int32_t *n_b);

/* Leiden blocking (Sec. 4, Sec. 6.1; Traag, Waltman & van Eck 2019).
 * quality 0 = modularity (Eq. 1, resolution gamma), 1 = CPM (Eq. 2,
 * threshold gamma); n_iter full Leiden iterations (paper: 2), randomness
 * beta (paper: 0.01), seed (paper: 42).  Communities are numbered by first
 * appearance.  block_of int32[n]. */
iccg_status iccg_block_leiden(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t quality,
                              double gamma, int32_t n_iter, double beta, uint64_t seed,
                              int32_t *block_of, int32_t *n_b);

/* Leiden block order (Sec. 6.1): relabel blocks by size, descending (ties:
 * smaller first row first). */
iccg_status iccg_sort_blocks_desc(int32_t n, int32_t n_b, int32_t *block_of);

/* Greedy block coloring (Sec. 3; Sec. 5.1) followed by the block-multicolor
 * ordering (colors ascending, blocks ascending, rows ascending).
 * color_of int32[n_b]; perm int32[n]; block_ptr int32[n_b+1];
 * color_ptr int32[n_b+1] (first n_c+1 entries used). */
iccg_status iccg_color_order(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t n_b,
                             const int32_t *block_of, int32_t *color_of, int32_t *n_c,
                             int32_t *perm, int32_t *block_ptr, int32_t *color_ptr);

/* ------------------------------------------------------------------------
 * Device-side blocking (the same results as the host helpers above, computed
 * on the GPU).  All array arguments are device pointers on `stream`; scalar
 * outputs (m, n_c) are host pointers, filled before return (each call
 * synchronizes `stream`).  Scratch is allocated stream-ordered and freed
 * before return.  ICCG_ERR_ARG on invalid input (checked on the device
 * before use), ICCG_ERR_CUDA on a CUDA error.
 *
 *   iccg_dev_graph        the graph of Sec. 3 (edge {i,j} iff a_ij or a_ji is
 *                         stored, i != j), rows sorted: gptr int64[n+1],
 *                         gadj int32 of capacity 2 nnz, *m = gptr[n]; equal
 *                         to iccg_graph's.
 *   iccg_dev_color_order  greedy block coloring (Sec. 3, Sec. 5.1: blocks
 *                         in index order, the smallest color no adjacent
 *                         block with a smaller index has) and the
 *                         block-multicolor ordering; outputs as for
 *                         iccg_color_order (color_of int32[n_b], perm
 *                         int32[n], block_ptr int32[n_b+1], color_ptr
 *                         int32[n_b+1], *n_c), equal to its results.  The
 *                         blocks are colored in waves: a block as soon as
 *                         all its smaller neighbours are.
 *   iccg_dev_sort_blocks_desc  Leiden block order (Sec. 6.1): blocks
 *                         relabelled by size descending, ties by smallest
 *                         row; equal to iccg_sort_blocks_desc.
 *   iccg_dev_block_leiden Leiden blocking (Sec. 4, Sec. 6.1) on the device:
 *                         quality 0 = modularity (Eq. 1), 1 = CPM (Eq. 2),
 *                         resolution gamma, n_iter passes.  The same quality
 *                         and gains as iccg_block_leiden, in a parallel form
 *                         that does not reproduce the host's partition:
 *                         local moving in synchronous sub-rounds (moves to
 *                         smaller labels, then to larger ones, no two nodes
 *                         swapping), refinement choosing the largest
 *                         non-negative gain (no randomness), aggregation as
 *                         on the host; every community is then split into
 *                         its connected components.  Deterministic.
 *                         block_of int32[n] (device, labels 0..n_b-1, not
 *                         size-sorted), *n_b (host).
 * ------------------------------------------------------------------------ */
iccg_status iccg_dev_graph(int32_t n, const int64_t *rowptr, const int32_t *colind, int64_t nnz, int64_t *gptr,
                           int32_t *gadj, int64_t *m, iccg_stream_t stream);
iccg_status iccg_dev_color_order(int32_t n, const int64_t *gptr, const int32_t *gadj, int64_t m, int32_t n_b,
                                 const int32_t *block_of, int32_t *color_of, int32_t *n_c, int32_t *perm,
                                 int32_t *block_ptr, int32_t *color_ptr, iccg_stream_t stream);
iccg_status iccg_dev_sort_blocks_desc(int32_t n, int32_t n_b, int32_t *block_of, iccg_stream_t stream);
iccg_status iccg_dev_block_leiden(int32_t n, const int64_t *gptr, const int32_t *gadj, int64_t m, int32_t quality,
                                  double gamma, int32_t n_iter, int32_t *block_of, int32_t *n_b,
                                  iccg_stream_t stream);

/* Level-set ordering, the level scheduling of the triangular solves (Sec. 2)
 * expressed as a block-multicolor ordering: level_of[i] = 0 when no
 * neighbour j < i exists, else 1 + max level_of[j] over the neighbours j < i;
 * rows of one level are never adjacent, so each level is a color of one-row
 * blocks.  perm int32[n] (levels ascending, rows ascending within a level),
 * block_ptr int32[n+1] (= 0..n), color_ptr int32[n+1] (first n_lev+1 used),
 * *n_lev the number of levels.  The IC(0) factor and the substitutions in
 * this order are those of the natural order (every adjacent pair keeps its
 * relative order), so iccg_setup with these arrays gives the GPU
 * level-scheduled ICCG of the natural ordering. */
iccg_status iccg_level_order(int32_t n, const int64_t *gptr, const int32_t *gadj, int32_t *level_of,
                             int32_t *n_lev, int32_t *perm, int32_t *block_ptr, int32_t *color_ptr);

/* Intra-block level sets for oversized blocks: a block-multicolor ordering
 * (perm, block_ptr, color_ptr, as for iccg_setup; CSR host arrays of A) is
 * refined by splitting every block of more than max_rows rows into its
 * in-block dependency levels (level 0: rows with no earlier row of their
 * block in the pattern; otherwise one more than the deepest such row), each
 * level of a color becoming a color of one-row blocks placed after the
 * color's small blocks.  Rows of one such level are never adjacent and every
 * adjacent pair keeps its relative order, so the IC(0) factor and the
 * substitutions of the refined ordering are those of the input ordering,
 * with all rows of a level of a color resolved in parallel.  Outputs:
 * perm_out int32[n], block_ptr_out int32[n+1], color_ptr_out int32[n+1]
 * (first *n_c_out + 1 used), *n_b_out, *n_c_out. */
iccg_status iccg_split_levels(int32_t n, const int64_t *rowptr, const int32_t *colind, const int32_t *perm,
                              const int32_t *block_ptr, const int32_t *color_ptr, int32_t n_b, int32_t n_c,
                              int32_t max_rows, int32_t *perm_out, int32_t *block_ptr_out,
                              int32_t *color_ptr_out, int32_t *n_b_out, int32_t *n_c_out);

/* Diagnostics (host only, no device): builds the layout iccg_setup would
 * build for these inputs (groups of at most group_rows rows, lane tiles for
 * colors of blocks of at most lane_max rows, 0 = none; with use_units, warp
 * units for every color of blocks of at most 32 rows) and checks the index ranges and
 * orderings the kernels rely on.  report[4]: lane tiles plus warp units,
 * groups, failed checks, the tile / unit / group / color of the first failure
 * (-1 none); *what (may be NULL) names the first failed check.  ICCG_OK,
 * ICCG_ERR_STATE when a check failed, or the validation error of iccg_setup. */
iccg_status iccg_check_layout(int32_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
                              const double *val, const int32_t *perm, const int32_t *block_ptr,
                              const int32_t *color_ptr, int32_t n_b, int32_t n_c, int32_t group_rows,
                              int32_t lane_max, int32_t use_units, int64_t report[4], const char **what);

/* ------------------------------------------------------------------------
 * Learned blocking (extension; the paper selects block sizes and
 * resolutions by sweeps, Table 2 and Sec. 6.1).
 *
 * iccg_features: ICCG_NFEATURES statistics of a CSR matrix (host pointers;
 * definitions in the source: log10 n, row-degree moments and maximum,
 * log10 nnz, diagonal-dominance statistics, bandwidth and mean entry
 * distance, an 8-bin histogram of off-diagonal counts, the off-diagonal
 * magnitude range).  ICCG_ERR_ARG on an invalid CSR.
 *
 * The MLP (two hidden ReLU layers of width h, FP32) maps standardised
 * features to ncls class logits (block size) and one regression output
 * (log resolution).  params: float[iccg_mlp_nparams(nf, h, ncls)] laid out
 * W1 [nf][h], b1 [h], W2 [h][h], b2 [h], W3 [h][ncls+1], b3 [ncls+1]
 * (device).  All arrays below are device pointers on `stream`.
 *   iccg_mlp_forward   X [batch][nf] -> out [batch][ncls+1]; act (may be
 *                      NULL, else float[2 * batch * h]) receives the two
 *                      hidden activations (layer 1, then layer 2).
 *   iccg_mlp_grad      loss = mean over the batch of the cross entropy of
 *                      softmax(out[:ncls]) against ycls (int32, 0..ncls-1)
 *                      plus wreg times the squared error of out[ncls]
 *                      against yreg; grad [nparams] and *loss (device float)
 *                      receive it.  work: float[batch * (4h + 2(ncls+1) + 1)].
 *   iccg_mlp_adam      one Adam step (bias-corrected, step >= 1) on params
 *                      with first / second moments m, v.
 * Every reduction runs in a fixed order: results are reproducible.
 * ------------------------------------------------------------------------ */
#define ICCG_NFEATURES 20
iccg_status iccg_features(int32_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                          double out[ICCG_NFEATURES]);
int64_t iccg_mlp_nparams(int32_t nf, int32_t hidden, int32_t ncls);
iccg_status iccg_mlp_forward(const float *params, int32_t nf, int32_t hidden, int32_t ncls, const float *X,
                             int32_t batch, float *out, float *act, iccg_stream_t stream);
iccg_status iccg_mlp_grad(const float *params, int32_t nf, int32_t hidden, int32_t ncls, const float *X,
                          const int32_t *ycls, const float *yreg, float wreg, int32_t batch, float *grad,
                          float *loss, float *work, iccg_stream_t stream);
iccg_status iccg_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t nparams, float lr,
                          float beta1, float beta2, float eps, int32_t step, iccg_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* ICCG_H_ */
