/*
 * idbf.h - C interface of the GB300 interpolative decomposition butterfly factorization.
 *
 * The library approximates a complementary low-rank N x N kernel matrix K(x_i, xi_j) by the
 * product of L + 1 block-sparse factors (Pang, Ho and Yang, "Interpolative Decomposition
 * Butterfly Factorization", Eq. 1):
 *
 *     K ~ U^L ... U^h S^h V^h ... V^L,   N = n0 2^L,
 *
 * built from (eps, k) interpolative decompositions of sampled blocks (Sec. 2.1) organised by
 * leaf-root complementary skeletonization and recursive matrix splitting (Secs. 2.2-2.4), and
 * applies it to blocks of vectors in O(N log N) (Sec. 1).
 *
 * Conventions shared by every call:
 *   - All functions return an idbf_status; nothing throws across this interface.
 *   - Vectors are caller-owned DEVICE memory on the plan's device: column-major blocks of
 *     N rows and nrhs columns with leading dimension ld >= N, interleaved complex
 *     (re, im). complex128 = two doubles, complex64 = two floats.
 *   - Calls that take a `stream` (a cudaStream_t passed as void*; NULL = legacy default
 *     stream) are stream-ordered and return before the GPU work ends, except where stated.
 *   - A plan is bound to the CUDA device that was current when it was created; calls on it
 *     must be made with that device current. A plan is not thread-safe: calls on the same
 *     plan from several host threads must be serialised by the caller.
 *
 * Factor layout (the "butterfly layout", shared by idbf_import_factors and idbf_save):
 *   Level l = 0..L in apply order. Level l has m = 2^L nodes; node j reads segments 2j and
 *   2j+1 of boundary l-1 (rows j*n0 .. j*n0+n0-1 of x when l = 0) and writes segments
 *   (j / H) 2H + j % H + c H, c = 0, 1, of boundary l with H = 2^(L-l) (rows of y when
 *   l = L). Boundary b = 0..L-1 holds 2m segments; seg_len[b][i] is the length of segment i.
 *   Each node has two blocks c = 0, 1 holding a dense complex matrix M_c (rows x cols) and
 *   index lists q_c, p_c. With u = concat(in_0, in_1) and t = concat(out_0, out_1):
 *     levels l <  h_V (column IDs, V):   out_c = u[q_c] + M_c u[p_c],   |q_c| = rows, |p_c| = cols
 *     level  l == h_V (middle factor S): out_c = M_c u
 *     levels l >  h_V (row IDs, U):      t[q_c] += in_c,  t[p_c] += M_c in_c,
 *                                        |q_c| = cols = |in_c|, |p_c| = rows
 *   h_V = floor(L/2). On the U side M_c is the transpose T^T of the row ID's interpolation
 *   block, so U = Lambda [I T]^T (Sec. 2.1, row ID); on the V side M_c = T of the column ID
 *   V = [I T] Lambda^* (Sec. 2.1, Lemma 2.1).
 */
#ifndef IDBF_H
#define IDBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct idbf_plan_s* idbf_plan;

typedef enum {
  IDBF_OK = 0,
  IDBF_EINVAL = 1,       /* an argument is invalid (null pointer, size, mode); nothing was done */
  IDBF_ENOMEM = 2,       /* device or host memory exhausted, or the planned bytes exceed free memory */
  IDBF_ECUDA = 3,        /* a CUDA runtime call failed; idbf_last_cuda_error() names it */
  IDBF_ERANKCAP = 4,     /* warning: some ID stopped at its maximum rank min(k, samples) with columns left (accuracy may exceed eps) */
  IDBF_ETIMEOUT = 5,     /* a bounded device-side wait gave up; the results of the call are invalid */
  IDBF_EFORMAT = 6,      /* factor arrays or a saved file are inconsistent */
  IDBF_EUNSUPPORTED = 7  /* valid request the library does not handle (e.g. storage absent for a mode) */
} idbf_status;

/* ---- kernels (the numerical examples of Sec. 3) ---------------------------------------- */
/* IDBF_KERNEL_FIO1D: K(x, xi) = exp(2 pi i (x xi + c(x) |xi|))   (Example 1, Eq. 1D-FIO)
 *   c_profile 0: c(x) = (2 + sin(2 pi x) sin(4 pi x)) / 3
 *   c_profile 1: c(x) = (2 + 0.2 sin(2 pi x)) / 16   (Example 1 as printed)
 *   c_profile 2: c(x) = 0
 * IDBF_KERNEL_DFT:   K(x, xi) = exp(sign 2 pi i x xi), sign = +1 or -1   (Example 3)
 * IDBF_KERNEL_J0:    K(x, xi) = J_0(x xi), the Schloemilch expansion of Example 2 (Eq. S) on
 *                    x_k = (k-1)/N, xi_n = n pi; a real kernel (zero imaginary parts); J_0 is
 *                    CUDA's j0; sign and c_profile are ignored */
#define IDBF_KERNEL_FIO1D 0
#define IDBF_KERNEL_DFT 1
#define IDBF_KERNEL_J0 2
typedef struct {
  int32_t kind;
  int32_t sign;
  int32_t c_profile;
  int32_t reserved;
} idbf_kernel;

/* ---- construction parameters (Sec. 2.1 and Sec. 3) ------------------------------------- */
#define IDBF_SAMPLE_MOCK_CHEBYSHEV 0 /* default; Sec. 2.1 */
#define IDBF_SAMPLE_RANDOM 1         /* uniform without replacement, SplitMix64 stream per ID */
#define IDBF_SAMPLE_ALL 2            /* no sampling (every candidate); exact-mode checks */

/* arithmetic of the IDs' column-pivoted Householder QR and back substitution (Sec. 2.1):
 * FP64 (default), or double-float (binary32 pairs, 48 significant bits) for the O(ns b k) updates
 * with the O(b)-per-step scalars in FP64, which runs on the FP32 pipes (the build is bound by
 * the FP64 pipe otherwise); both far more accurate than any tolerance eps >= 1e-12 needs */
#define IDBF_QR_FP64 0
#define IDBF_QR_DF64 1

/* storage formats of the factor entries on the device (bit i of a storage mask = format i) */
#define IDBF_STORE_C128 0 /* complex FP64, 16 B per entry */
#define IDBF_STORE_DF64 1 /* complex double-float: (re_hi, re_lo, im_hi, im_lo) floats, 16 B */
#define IDBF_STORE_C64 2  /* complex FP32, 8 B per entry */

typedef struct {
  double eps;             /* ID tolerance (Eq. acc); k_eps = #leading |R_jj| > eps |R_11| */
  double oversample;      /* t: t*k rows/columns sampled per ID (Eq. pivotedQR2); paper: 1 */
  double oversample_leaf; /* t at the leaf step (k = n0 there); <= 0 means "same as t" */
  int32_t leaf;           /* n0: points per leaf; N = n0 2^L with L >= 2 */
  int32_t rank_cap;       /* k; 0 = min(#rows, #columns) of each block ("k = min{m,n}") */
  int32_t sampling;       /* IDBF_SAMPLE_* */
  int32_t storage;        /* IDBF_STORE_* format the factors are kept in after the build */
  uint64_t seed;          /* random sampling stream seed */
  int32_t qr_arith;       /* IDBF_QR_* arithmetic of the pivoted QR of every ID */
  int32_t reserved;       /* 0 */
} idbf_params;

/* Fill p with the defaults: eps 1e-6, t 1, t_leaf = t, n0 64, k = min dims, Mock-Chebyshev,
 * C128 storage, seed 0, FP64 QR. */
void idbf_default_params(idbf_params* p);

/* idbf_build - construct the IDBF of K on the point sets X = {x_i} and Omega = {xi_j}
 * (Secs. 2.2-2.4) on the current device.
 *   x_host, xi_host: N host doubles each, both sorted ascending (the dyadic trees of Sec. 1
 *                    are taken over index ranges, leaf j = points j*n0 .. j*n0+n0-1).
 *   The kernel entries are sampled and the per-node IDs computed by batched device kernels
 *   (FP64 column-pivoted Householder QR, FP64 back-substitution). The call is synchronous on
 *   `stream` (it returns when the plan is complete) and allocates device memory owned by the
 *   returned plan. Returns IDBF_ERANKCAP (with a valid plan) when an ID hit rank_cap.
 *   Errors: EINVAL (N not n0 2^L, L < 2, unsorted points, bad kernel/params), ENOMEM, ECUDA. */
idbf_status idbf_build(const idbf_kernel* kernel, const double* x_host, const double* xi_host,
                       int64_t N, const idbf_params* params, void* stream, idbf_plan* out);

/* idbf_build_leaves - idbf_build on trees whose 2^L leaves are given by offsets: the dyadic
 * trees of Sec. 1 built by partitioning the domains of X and Omega (coordinate-based trees; see
 * idbf_dyadic_leaves), as Example 3 needs for randomly placed points. Row leaf j holds the points
 * x_host[row_leaf_off[j] .. row_leaf_off[j+1]) and column leaf j the points
 * xi_host[col_leaf_off[j] .. col_leaf_off[j+1]); offsets rise from 0 to N (2^L + 1 each, host
 * memory), leaves may be empty, N is any size >= 1, L >= 2, params->leaf is ignored. An ID of a
 * block with no rows or no sampled columns has rank 0 (no skeleton, every index redundant). The
 * plan runs the per-node level kernels only (see idbf_import_factors). Otherwise as idbf_build.
 * Errors: EINVAL (offsets, L, unsorted points, params), ENOMEM, ECUDA. */
idbf_status idbf_build_leaves(const idbf_kernel* kernel, const double* x_host, const double* xi_host,
                              int64_t N, int32_t L, const int64_t* row_leaf_off,
                              const int64_t* col_leaf_off, const idbf_params* params, void* stream,
                              idbf_plan* out);

/* idbf_dyadic_leaves - the leaves of the dyadic tree of depth L over the domain [lo, hi) (Sec. 1):
 * leaf j is [lo + (hi - lo) (j / 2^L), lo + (hi - lo) ((j + 1) / 2^L)), so that a point on an
 * interior edge belongs to the leaf on its right; off[j] (2^L + 1 entries, host memory) is the
 * number of points below the left edge of leaf j and off[2^L] = n. points: n ascending host
 * doubles inside [lo, hi). Host computation, no GPU work. Errors: EINVAL. */
idbf_status idbf_dyadic_leaves(const double* points, int64_t n, double lo, double hi, int32_t L,
                               int64_t* off);

/* idbf_kernel_matvec_rows - ground truth of Sec. 3 (the direct matvec u^d) on selected rows:
 *   y[r] = sum_{j < N} K(x[rows[r]], xi[j]) v[j],  r < nrows,
 * O(nrows N) FP64 work on the current device. x, xi: N doubles; rows: nrows int64 row indices
 * (< N, not checked on the device); v: N complex128; y: nrows complex128; all device pointers.
 * Stream-ordered. Errors: EINVAL, ECUDA. */
idbf_status idbf_kernel_matvec_rows(const idbf_kernel* kernel, const double* x, const double* xi,
                                    int64_t N, const int64_t* rows, int64_t nrows, const void* v,
                                    void* y, void* stream);

/* ---- import of host factors in the butterfly layout (used for oracle parity) ----------- */
typedef struct {
  int64_t N;
  int32_t n0;
  int32_t L;
  const int32_t* seg_len;  /* [L][2m] segment lengths at boundaries 0..L-1 */
  const int32_t* blk_rows; /* [L+1][m][2] rows of M_c */
  const int32_t* blk_cols; /* [L+1][m][2] columns of M_c */
  const int64_t* blk_moff; /* [L+1][m][2] offset of M_c in mat, in complex entries */
  const int64_t* blk_ioff; /* [L+1][m][2] offset of q_c (then p_c) in idx */
  const double* mat;       /* mat_len interleaved complex128 entries, each M_c row-major */
  int64_t mat_len;
  const int32_t* idx;      /* idx_len int32 indices */
  int64_t idx_len;
  /* Leaves of uneven size (coordinate-based dyadic trees of Sec. 1, Example 3): m + 1 offsets
   * each, rising from 0 to N; leaf j of x (columns, read by level 0) is x[col_leaf_off[j] ..
   * col_leaf_off[j+1]) and leaf j of y (rows, written by level L) is y[row_leaf_off[j] ..
   * row_leaf_off[j+1]). Leaves and segments may be empty. NULL (both) = leaves of n0 points. */
  const int64_t* row_leaf_off;
  const int64_t* col_leaf_off;
} idbf_host_factors;

/* idbf_import_factors - copy factors given in host memory into a new plan stored in format
 * `storage`. Every size and index is validated before any device work (EFORMAT on any
 * inconsistency). Without leaf offsets, leaves hold n0 >= 1 points each with N = n0 2^L and
 * every segment is non-empty. With leaf offsets (Example 3: random points, coordinate-based
 * trees), N is any size >= 1, n0 is ignored (0), leaves and segments may be empty, and blocks
 * with no columns contribute zeros. Plans with leaves of uneven size run the per-node level
 * kernels (FP64, double-float and FP32, any number of right-hand sides, forward and adjoint,
 * idbf_apply_noalloc) and, for one right-hand side, the streaming kernels and fused level
 * pairs; the warp-per-node, register-tiled and tensor-core kernels, batches and checkpoints
 * refuse them (EUNSUPPORTED; an apply then uses the per-node kernel). Offsets that are all equal
 * are the uniform case. Synchronous. */
idbf_status idbf_import_factors(const idbf_host_factors* f, int32_t storage, void* stream,
                                idbf_plan* out);

/* ---- apply (Eq. 1) ---------------------------------------------------------------------- */
#define IDBF_MODE_FP64 0   /* C128 storage, complex128 vectors, FP64 FMA */
#define IDBF_MODE_DF64 1   /* DF64 storage, complex128 vectors, double-float (FP32 pair) arithmetic */
#define IDBF_MODE_FP32 2   /* C64 storage, complex64 vectors, FP32 FMA */
#define IDBF_MODE_TF32X3 3 /* C64 storage, complex64 vectors, 3xTF32 tensor-core block products
                           * (tcgen05, FP32 accumulation; forward only; blocks of <= 256 rows) */
#define IDBF_MODE_TF32X3_S64 4 /* as IDBF_MODE_TF32X3 on every level but the middle factor S^h
                               * (Eq. finishIDBF), whose products and sums run on the CUDA cores
                               * in double-float (DF64 storage of that level, preferred) or FP64
                               * (C128 storage); complex64 vectors on both of its sides. Needs C64
                               * on the other levels (see idbf_set_level_storage); forward only */

/* idbf_apply - y = K x for an N x nrhs block: x -> V levels -> S -> U levels -> y.
 *   x, y: device pointers (may not alias), ld >= N, element type set by `mode` (above).
 *   Uses a workspace owned by the plan; a call with a larger nrhs than any before allocates
 *   it (cudaMalloc, synchronising), so reserve it with idbf_reserve before graph capture.
 *   Errors: EINVAL, EUNSUPPORTED (storage for `mode` absent), ENOMEM, ECUDA. */
idbf_status idbf_apply(idbf_plan plan, const void* x, void* y, int64_t nrhs, int64_t ld,
                       int32_t mode, void* stream);

/* idbf_apply_adjoint - y = K^* x: the factors in reverse order, each block conjugate-
 * transposed (U-leaf^* first, V-leaf^* last). Same arguments and errors as idbf_apply. */
idbf_status idbf_apply_adjoint(idbf_plan plan, const void* x, void* y, int64_t nrhs, int64_t ld,
                               int32_t mode, void* stream);

/* idbf_apply_noalloc - y = K x like idbf_apply, except that the library allocates no device
 * memory during the call. The paper has no counterpart of this call; it exists for callers that
 * must not allocate: a framework whose own caching allocator already holds nearly all device
 * memory (a cudaMalloc would fail or fragment it), a latency-critical serving loop that cannot
 * absorb the device-wide synchronisation that cudaMalloc and cudaFree imply, or a process that
 * has to know its full device footprint when the library loads.
 *   Scope: forward apply only, modes IDBF_MODE_FP64, IDBF_MODE_DF64 and IDBF_MODE_FP32 (same
 *   arguments as idbf_apply). Every level runs the per-node level kernel (variant 0 of
 *   idbf_autotune), not the autotuned streaming or register-tiled kernels, so a call is slower
 *   than idbf_apply and its double-float / FP32 results differ from idbf_apply's in the summation
 *   order only: they agree within that mode's rounding error (FP64: to ~1e-15 relative).
 *   Workspace: a fixed array of IDBF_NOALLOC_SCRATCH_BYTES compiled into the library. Every GPU
 *   that loads the library holds one such array until the process exits. A call needs
 *   32 * nrhs * segment_entries bytes (segment_entries as reported by idbf_stats); a larger
 *   request returns IDBF_EUNSUPPORTED before any GPU work (the FIO benchmark kernel fits for
 *   N up to 2^18 with one right-hand side), as does a level whose per-node kernel would need
 *   more than 200 KB of shared memory (all levels are checked before the first launch).
 *   The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 *   with that device current) and caches it for the life of the process's primary context on
 *   that device (after cudaDeviceReset no plan, and no cached address, remains valid): make that
 *   first call before any stream capture.
 *   All calls on a device share the one array, and it keeps whatever the previous call left in
 *   it; nothing in it has to start at zero, because every level overwrites each segment before
 *   the next level reads it. Calls whose GPU work overlaps (other streams, other plans, other
 *   host threads) race on the array and produce wrong results: serialise them.
 *   Errors: EINVAL (also for IDBF_MODE_TF32X3), EUNSUPPORTED (size above the limit, or storage
 *   for `mode` absent), ECUDA. */
#define IDBF_NOALLOC_SCRATCH_BYTES (64ull << 20)
idbf_status idbf_apply_noalloc(idbf_plan plan, const void* x, void* y, int64_t nrhs, int64_t ld,
                               int32_t mode, void* stream);

/* idbf_autotune - for the single-right-hand-side forward apply in `mode` (FP64, DF64 or FP32),
 * time every kernel variant of every level (0: the per-node kernel; 1-6: the streaming kernel
 * with three shared-memory ring layouts, node inputs copied by the producer warp or loaded by
 * the consumers; 7: one warp per node, for levels of short blocks; 8-13: 1-6 with the columns
 * of blocks of at most 96 rows split between up to four thread groups, whose partial sums are
 * added at the end; 14-15: a fourth ring layout with four CTAs per SM and small stages, for
 * levels of short blocks, with the split; 16-19: levels l and l + 1 fused in one launch of the
 * streaming kernel, ring layouts A-D: each CTA takes two nodes of level l and the two nodes of
 * level l + 1 that read their four output segments, which stay in shared memory, the radix-2
 * case of level fusion) `reps` times with CUDA events on `stream`, and keep the cheapest cover
 * of the levels by single levels and fused pairs in the plan (idbf_stats reports the variant of
 * every level; both levels of a fused pair report the pair's variant). Later idbf_apply calls
 * use the choices; results are identical up to the summation order of the double-float / FP32
 * partial sums. Synchronous; allocates two N-vector temporaries. *apply_ms (if not NULL)
 * receives the summed best times. FP64 runs variants 0 and 7 only.
 * Errors: EINVAL, EUNSUPPORTED (storage for `mode` absent), ENOMEM, ECUDA. */
idbf_status idbf_autotune(idbf_plan plan, int32_t mode, int32_t reps, void* stream, float* apply_ms);

/* idbf_set_level_variants - set the forward kernel variant of every level for `mode` directly
 * (n = L + 1 values in 0..IDBF_NUM_FWD_VARIANTS-1, -1 = default; n = 0 clears), e.g. to restore the
 * choices of an earlier idbf_autotune. Levels are read from 0 upwards: a pair variant (16-19) on
 * level l covers levels l and l + 1 (the entry of level l + 1 is then not read); on level L it
 * runs level L alone. A variant that does not fit a level falls back to the default, then to
 * variant 0. */
#define IDBF_NUM_FWD_VARIANTS 20
idbf_status idbf_set_level_variants(idbf_plan plan, int32_t mode, const int32_t* variants, int32_t n);

/* idbf_set_tc_split - operand splitting of the 3xTF32 tensor-core mode: 0 = x_hi + x_lo with
 * x_hi = tf32(x) and three products (default), 1 = x_lo also rounded to TF32, 2 = four products
 * (adds x_lo y_lo). */
idbf_status idbf_set_tc_split(idbf_plan plan, int32_t split_mode);

/* idbf_reserve - allocate the apply workspace for up to nrhs right-hand sides now. */
idbf_status idbf_reserve(idbf_plan plan, int64_t nrhs);

/* idbf_set_level_storage - as idbf_set_storage for level `level` (0..L, apply order) alone, e.g.
 * to keep the middle factor (level h_V = floor(L/2)) in C128 or DF64 for IDBF_MODE_TF32X3_S64
 * while every other level holds C64 only. Synchronous. Errors: EINVAL, EUNSUPPORTED (a wider
 * format asked of a level that holds only C64), ENOMEM, ECUDA. */
idbf_status idbf_set_level_storage(idbf_plan plan, int32_t level, uint32_t mask, void* stream);

/* idbf_set_storage - keep exactly the formats in `mask` (bit IDBF_STORE_*). Missing formats
 * are converted from a present one (C128 preferred as the source; C128 <-> DF64 in place when
 * only one of them is kept). Stream-ordered; ENOMEM leaves the plan unchanged. */
idbf_status idbf_set_storage(idbf_plan plan, uint32_t mask, void* stream);

/* idbf_sync_status - wait for `stream`, then report whether any bounded device-side wait of this
 * plan's kernels gave up since the last call (IDBF_ETIMEOUT; the outputs of those calls are
 * invalid) and clear the record. Every wait in the library's kernels ends after a time limit
 * instead of hanging; IDBF_OK otherwise. */
idbf_status idbf_sync_status(idbf_plan plan, void* stream);

/* idbf_debug_set_wait - fault injection for tests: set the time limit of the device-side waits
 * (default 2 s) and, with producer_enabled = 0, make the streaming kernels' producer issue no
 * copies so that every consumer wait runs out. Not for production use. */
idbf_status idbf_debug_set_wait(idbf_plan plan, uint64_t limit_ns, int32_t producer_enabled);

/* ---- uneven batches: many operators in one persistent launch ---------------------------- */
typedef struct idbf_batch_s* idbf_batch;

/* idbf_batch_create - prepare the forward apply of nops plans (any N each), plan o with nrhs[o]
 * right-hand sides, in `mode` (FP64, DF64 or FP32), as ONE persistent kernel launch captured in a
 * CUDA graph (plans with leaves of n0 points; uneven leaves: EUNSUPPORTED). Work items
 * (operator, level, run of nodes, block of right-hand sides) are queued in
 * level order and taken by persistent CTAs; an item waits (bounded) until the previous level of
 * its operator is complete. Operators from a size up can be left out of the launch and applied
 * on their own (idbf_batch_set_split, chosen by idbf_batch_autotune). Allocates each operator's
 * level workspace; the plans must outlive the batch and must not be changed (storage) while it
 * exists. Synchronous. */
idbf_status idbf_batch_create(const idbf_plan* plans, int32_t nops, const int64_t* nrhs, int32_t mode,
                              idbf_batch* out);

/* idbf_batch_apply - y[o] = K_o x[o] for every operator o (device pointers, column-major N_o x
 * nrhs[o] blocks with leading dimension ld[o] >= N_o, element type of `mode`): one graph launch
 * on `stream` after a small copy of the pointer table, then idbf_apply for each operator above
 * the split (idbf_batch_set_split). */
idbf_status idbf_batch_apply(idbf_batch b, const void* const* x, void* const* y, const int64_t* ld,
                             void* stream);

/* idbf_batch_autotune - time the batch for every tiling of idbf_batch_set_tiling below (for the
 * mixed tiling 7 also its row threshold in {32, 64, 96, 128, 192}) and nodes per item in
 * {1, 2, 4}, then, unless a split was set with idbf_batch_set_split, every split with the best
 * tiling (and the tilings again if the split changed); reps launches each, on the given buffers;
 * tilings whose shared memory exceeds 200 KB are skipped. Keeps the fastest; *best_ms receives
 * its time per idbf_batch_apply. Synchronous. */
idbf_status idbf_batch_autotune(idbf_batch b, const void* const* x, void* const* y, const int64_t* ld,
                                int32_t reps, void* stream, float* best_ms);

/* idbf_batch_set_tiling - choose the tiling by hand: `tile` indexes the autotuner's list above
 * (0: (1,1), 1: (4,2), 2: (8,2), 3: (8,4) per-thread right-hand sides; 4: 8 and 5: 16 right-hand
 * sides per item in 4 x 4 register tiles over streamed factor columns, 6: 32 in 4 x 8 tiles;
 * 7: mixed per level, 16 per item in register tiles where a level's blocks have more than a row
 * threshold (64 unless the autotuner chose another), else 8 per item, 4 per thread; 4-7 in FP32
 * and FP64 only, 6 in FP32 only), nodes_per_item in {1, 2, 4}. IDBF_EUNSUPPORTED if the
 * tile does not exist for the batch's precision or its shared memory exceeds 200 KB (the
 * previous tiling is then kept), IDBF_EINVAL for other values. Synchronous. */
idbf_status idbf_batch_set_tiling(idbf_batch b, int32_t tile, int32_t nodes_per_item);

/* idbf_batch_set_split - operators with N >= min_separate_n leave the persistent launch: each
 * runs through idbf_apply (its own per-level kernels, stream-ordered after the launch) within
 * idbf_batch_apply; INT64_MAX keeps every operator in the launch. Large operators fill the GPU
 * by themselves, and without them the launch needs less shared memory per CTA. A split set here
 * is kept by idbf_batch_autotune. min_separate_n = 0 (the state after idbf_batch_create) lets
 * idbf_batch_autotune choose it among INT64_MAX and the N of each operator; until then every
 * operator is in the launch. IDBF_EUNSUPPORTED if the remaining launch does not fit the current
 * tiling (the previous split is then kept), IDBF_EINVAL for a negative value. This goes beyond
 * the paper, which applies one operator at a time. Synchronous. */
idbf_status idbf_batch_set_split(idbf_batch b, int64_t min_separate_n);

/* idbf_batch_split - the current split and the number of operators applied through idbf_apply. */
idbf_status idbf_batch_split(idbf_batch b, int64_t* min_separate_n, int32_t* separate_ops);

/* idbf_batch_info - the current tiling: right-hand sides and nodes per work item, number of
 * items, persistent CTAs (0 and 0 when every operator runs through idbf_apply). */
idbf_status idbf_batch_info(idbf_batch b, int32_t* rhs_per_item, int32_t* nodes_per_item, int32_t* items,
                            int32_t* ctas);

/* idbf_batch_sync_status - wait for `stream`; IDBF_ETIMEOUT if a bounded wait of the batch kernel
 * (or of an operator applied through idbf_apply) gave up since the last call (its results are
 * invalid), IDBF_OK otherwise. */
idbf_status idbf_batch_sync_status(idbf_batch b, void* stream);

/* idbf_batch_debug_set_wait - fault injection for tests: set the time limit of the batch
 * kernel's dependency waits (default 2 s) and, with extra_target > 0, raise the completion count
 * that the first operator's level-1 items wait for above the number of level-0 items, so that
 * those waits run out (a failure made on the host: no device fault). Each such item is then
 * skipped and counted as done, and idbf_batch_sync_status reports IDBF_ETIMEOUT. (limit, 0)
 * restores normal operation. Re-captures the graph. Not for production use. */
idbf_status idbf_batch_debug_set_wait(idbf_batch b, uint64_t limit_ns, int32_t extra_target);

/* idbf_batch_destroy - release the batch (synchronises the device first; NULL is a no-op). */
void idbf_batch_destroy(idbf_batch b);

/* ---- statistics ------------------------------------------------------------------------- */
#define IDBF_MAX_LEVELS 48
typedef struct {
  int64_t N;
  int32_t n0, L, h_v, h_u;
  uint32_t storage_mask;
  int32_t rank_saturated;                  /* IDs that stopped at their maximum rank, not by eps */
  int64_t entries;                         /* stored factor entries (T and S blocks) */
  int64_t index_entries;                   /* stored int32 skeleton/redundant indices */
  int64_t level_entries[IDBF_MAX_LEVELS];  /* per level l = 0..L in apply order */
  int32_t level_kmin[IDBF_MAX_LEVELS];     /* min / max output segment length of level l */
  int32_t level_kmax[IDBF_MAX_LEVELS];
  int64_t segment_entries;                 /* max over boundaries of the summed segment lengths */
  double build_seconds;                    /* wall time of idbf_build (0 for imported plans) */
  int64_t device_bytes;                    /* device memory held by the plan */
  int32_t level_variant[3][IDBF_MAX_LEVELS]; /* forward kernel per storage format and level (-1: default) */
  uint32_t level_storage[IDBF_MAX_LEVELS];   /* storage formats held by level l (bit IDBF_STORE_*) */
  int64_t boundary_entries[IDBF_MAX_LEVELS]; /* summed segment lengths of boundary b = 0..L-1 (the
                                                vector entries level b writes and level b+1 reads) */
} idbf_stats_t;

/* idbf_stats - fill *s (host memory). Synchronous, no GPU work. */
idbf_status idbf_stats(idbf_plan plan, idbf_stats_t* s);

/* ---- checkpoint ------------------------------------------------------------------------- */
/* idbf_save - write the factors (butterfly layout, complex128 entries) to a flat binary file
 * with a versioned header. Requires C128 or DF64 storage. Synchronous.
 * idbf_load - read such a file into a new plan stored as `storage`. EFORMAT on a bad file. */
idbf_status idbf_save(idbf_plan plan, const char* path);
idbf_status idbf_load(const char* path, int32_t storage, void* stream, idbf_plan* out);

/* idbf_clone - a new plan on the same device holding a device-to-device copy of every factor,
 * index list and storage format of `plan` (and its autotuned level variants), e.g. to give
 * identical operators of a batch factor memory of their own without building them again.
 * Synchronous on `stream`. Errors: EINVAL (NULL, other device current), ENOMEM, ECUDA. */
idbf_status idbf_clone(idbf_plan plan, void* stream, idbf_plan* out);

/* idbf_destroy - free the plan and all device memory it owns (NULL is a no-op). Synchronises
 * the device first so that no queued work still reads the factors. */
void idbf_destroy(idbf_plan plan);

const char* idbf_strerror(idbf_status s);
/* Name of the last CUDA error seen by this library on the calling thread ("" if none). */
const char* idbf_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IDBF_H */
