/*
 * tsqr.h -- C ABI of the GB300 TSQR / CAQR library (libtsqr_gb300.so).
 *
 * The library factors a tall-skinny m x n matrix A (m >= n) stored in a 1-D
 * block-row layout (Section 2, the problem statement of TSQR) into
 *     A = Q R,   R upper triangular with diag(R) >= 0,
 * where Q is kept implicitly as a product of block-diagonal orthogonal
 * factors, one per tree level, as in Eq. TSQR_binarytree_4 (Section 2.1):
 * one Householder QR per leaf (row block), then structured QRs of stacked R
 * triangles up a reduction tree.  CAQR
 * (Section 3) factors a general m x n matrix panel by panel with TSQR and
 * applies each panel's Q^T to the trailing matrix.
 *
 * Conventions shared by every entry point:
 *   - All matrix pointers are DEVICE pointers; matrices are column-major,
 *     element (i, j) at p[i + j * ld], with ld >= number of rows.
 *   - Element type: the FP64 entry points take double; the _f32 entry points
 *     take float storage and keep column norms, Householder vectors and tau
 *     generation in FP64 (the mixed-precision form).  Entry points that take
 *     a handle and a void* operate in the handle's element type.
 *   - Every call is asynchronous on `stream` (NULL = the legacy default
 *     stream) and returns after enqueuing its kernels.  The return value
 *     reports argument, launch and allocation errors only.  Device-side
 *     conditions (non-finite input, a bounded wait that gave up) are latched
 *     in the handle's status word and returned by tsqr_sync_status().
 *   - Return codes: 0 on success; -i if argument i (1-based) is invalid, in
 *     the style of LAPACK's info; a positive TSQR_ERR_* code otherwise.
 *   - Quick returns: m = 0 or n = 0 succeed and enqueue nothing.  m < n is
 *     an argument error (the paper assumes m >= n, Section 2).
 *   - Handles are opaque and library-owned; free them with tsqr_q_destroy
 *     (or caqr_q_destroy).  A handle BORROWS the matrix A it factored: the
 *     leaf Householder vectors live in A's storage, so the caller keeps A
 *     alive and unmodified until the handle is destroyed.  A handle is used
 *     by one stream at a time.
 */
#ifndef TSQR_GB300_H
#define TSQR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tsqr_stream_t; /* same type as cudaStream_t */
typedef struct tsqr_q_s* tsqr_q_t;         /* TSQR Q-tree handle */
typedef struct caqr_q_s* caqr_q_t;         /* CAQR handle: one Q-tree per panel */

enum tsqr_status_code {
  TSQR_OK = 0,
  TSQR_ERR_CUDA = 1,        /* a CUDA runtime call failed */
  TSQR_ERR_NOMEM = 2,       /* device workspace allocation failed */
  TSQR_ERR_TIMEOUT = 3,     /* a device-side bounded wait gave up */
  TSQR_ERR_NONFINITE = 4,   /* NaN or Inf met in a column norm or pivot */
  TSQR_ERR_UNSUPPORTED = 5, /* shape / precision combination not supported */
  TSQR_ERR_HANDLE = 6,      /* NULL, destroyed or mismatched handle */
  TSQR_ERR_TOO_LARGE = 7    /* problem exceeds tsqr_factor_r_noalloc's static scratch */
};

enum tsqr_precision {
  TSQR_PREC_FP64 = 0,     /* FP64 storage and arithmetic */
  TSQR_PREC_FP32 = 1,     /* FP32 storage and products; FP64 norms, vectors, tau */
  TSQR_UPDATE_BF16X3 = 2, /* CAQR only: FP32 storage; leaf-block trailing updates on the
                             tensor cores as three BF16 products (hi*hi + hi*lo + lo*hi)
                             accumulated in FP32; FP64 norms, vectors, tau */
  TSQR_UPDATE_TF32X3 = 3  /* CAQR only: the same with three TF32 products (kind::tf32);
                             the split keeps about 21 bits, the tensor cores' FP32
                             accumulation then limits the result (about 2^-19 of the
                             sum of |products| measured, against 2^-16 for BF16) */
};

/* Bits of tsqr_opts_t.flags (TSQR handles only; CAQR takes update_precision instead). */
enum tsqr_flags {
  /* FP32 handles with n <= 64: the leaf stage of tsqr_apply_qt (Q^T C, the
     trailing-update product of Section 3.1) runs on the tensor cores as three
     BF16 products per FP32 product, accumulated in FP32, like CAQR's
     TSQR_UPDATE_BF16X3.  Other handles: TSQR_ERR_UNSUPPORTED. */
  TSQR_FLAG_APPLY_BF16X3 = 1,
  /* Hybrid reduction tree (Section 2.1: the flat tree inside a processor,
     a q-ary tree across processors): the leaves are cut into chains of
     consecutive leaves, one chain per resident CTA; each chain is a flat
     tree -- its first leaf an ordinary leaf QR, every later leaf i the QR of
     [R; A_i] with the chain's running R -- and the q-ary tree (arity from
     opts) runs over the chains' R factors.  Leaves are n rows shorter than
     the default so that the stacked tile fits; every leaf keeps its
     Householder vectors in A (dense for the stacked steps) and its T.
     Not with TSQR_FLAG_APPLY_BF16X3 or tsqr_factor_form_host. */
  TSQR_FLAG_HYBRID_TREE = 2,
  /* Flat tree (Section 2.1's sequential TSQR, Eq. TSQR_seq_runtime): one
     chain over all leaves, one CTA streams the whole matrix. */
  TSQR_FLAG_FLAT_TREE = 4,
  /* Recursive leaf QR (Elmroth and Gustavson's RGEQR3, named in Sections
     2.1 and 3.3 for the local QR): each leaf factors its left half of
     columns recursively, updates the right half with the left half's
     I - Y T Y^T, factors the right half, and merges the two T factors; one
     column is the base case.  Same outputs as the default leaf.  n <= 64;
     not with the hybrid or flat tree. */
  TSQR_FLAG_RECURSIVE_LEAF = 8,
  /* As TSQR_FLAG_APPLY_BF16X3 with three TF32 products (TSQR_UPDATE_TF32X3). */
  TSQR_FLAG_APPLY_TF32X3 = 16
};

/* Tuning knobs; a zero field means "choose automatically". */
typedef struct tsqr_opts_s {
  int64_t leaf_rows; /* nominal leaf height h (>= n); rows per leaf block (Section 2.1) */
  int32_t arity;     /* reduction-tree arity q >= 2 (Section 2.1: any tree is valid) */
  int32_t flags;     /* 0 or TSQR_FLAG_* bits; unknown bits are an argument error */
} tsqr_opts_t;

/* ---------------------------------------------------------------- TSQR -- */

/*
 * tsqr_factor: R and the Q-tree of A (Section 2.1, Eqs. TSQR_binarytree_1..4).
 *   m, n   : rows and columns, m >= n >= 0.
 *   A      : device, m x n, lda >= max(1, m).  Overwritten: each leaf's rows
 *            hold its Householder vectors below the diagonal (unit diagonal
 *            implicit) and the leaf R factor on and above it.
 *   R      : device, n x n, ldr >= max(1, n).  Receives R with diag(R) >= 0;
 *            entries below the diagonal are set to 0.
 *   opts   : NULL or tuning knobs (leaf height, tree arity).
 *   q      : receives a new handle; NULL to discard Q (R only).
 * Leaves are consecutive row blocks of height h; the last leaf takes the
 * remainder, merged into the previous leaf when it would have fewer than n
 * rows.  Tree nodes factor q stacked upper triangles without touching their
 * zeros (Section 2.1, structured local QR; Section 2.2, 2n^3/3 flops per
 * binary node).  The signs d = sign(diag R_root) (sign(0) = +1) are applied
 * to R and recorded in the handle, so apply/form calls use Q D.
 */
int tsqr_factor(int64_t m, int64_t n, double* A, int64_t lda, double* R, int64_t ldr,
                const tsqr_opts_t* opts, tsqr_q_t* q, tsqr_stream_t stream);
int tsqr_factor_f32(int64_t m, int64_t n, float* A, int64_t lda, float* R, int64_t ldr,
                    const tsqr_opts_t* opts, tsqr_q_t* q, tsqr_stream_t stream);

/*
 * Plan-once form: tsqr_q_create allocates a handle and all of its device
 * workspace for an m x n problem (precision TSQR_PREC_*); tsqr_refactor then
 * factors a new matrix of that shape with no allocation, which makes the
 * call safe inside CUDA stream capture.  tsqr_factor = create + refactor.
 */
int tsqr_q_create(int64_t m, int64_t n, int32_t precision, const tsqr_opts_t* opts, tsqr_q_t* q,
                  tsqr_stream_t stream);
int tsqr_refactor(tsqr_q_t q, void* A, int64_t lda, void* R, int64_t ldr, tsqr_stream_t stream);

/*
 * tsqr_apply_qt: C <- Q^T C for the square m x m Q of the handle, C m x k
 * (device, ldc >= m).  Applied as the transpose of Eq. TSQR_binarytree_4:
 * leaf factors first, then tree levels bottom-up, then D on rows 0..n-1.
 * The top n rows of the result are the unique product with the thin Q; the
 * remaining rows depend on the tree.  k = 0 is a quick return.
 */
int tsqr_apply_qt(tsqr_q_t q, int64_t k, void* C, int64_t ldc, tsqr_stream_t stream);

/* tsqr_apply_q: C <- Q C (reverse order: D, tree top-down, leaves). */
int tsqr_apply_q(tsqr_q_t q, int64_t k, void* C, int64_t ldc, tsqr_stream_t stream);

/*
 * tsqr_form_q: the thin Q (m x n, device, ldq >= m) = Q_tree [I_n; 0] D
 * (Section 2.1: Q factors with n columns).  Q must not alias A.
 */
int tsqr_form_q(tsqr_q_t q, void* Q, int64_t ldq, tsqr_stream_t stream);

/*
 * tsqr_form_q_mul: Q_thin X (m x k, device, ldq >= m) for X (n x k, device,
 * ldx >= n), formed like tsqr_form_q from [X; 0] instead of [I_n; 0]: the
 * rank-local block of the thin Q in parallel TSQR (Section 2.1), where X is
 * that rank's n-row block of the Q of the stacked R factors.  The signs D are
 * included (Q_thin X = Q_tree [D X; 0]).  Q must not alias A or X.
 */
int tsqr_form_q_mul(tsqr_q_t q, int64_t k, const void* X, int64_t ldx, void* Q, int64_t ldq, tsqr_stream_t stream);

/*
 * tsqr_factor_form_host: A = QR of a HOST matrix, with thin Q and R written
 * back to HOST memory (Section 2.1: factor, then the Q factor with n
 * columns), for data that lives on the host.  One call = tsqr_refactor +
 * tsqr_form_q + the host transfers:
 *   - a page-locked A_host (cudaHostAlloc or cudaHostRegister) is read by
 *     the leaf kernel itself over the host link, leaf by leaf; a pageable
 *     one goes to the device in chunks of leaves on a copy stream owned by
 *     the handle while the leaves already there are factored on `stream`;
 *   - after the tree and the tree part of Q: with a device Q, Q comes back
 *     chunk by chunk (copy stream) as its leaves are formed; with Q = NULL
 *     the form kernels store Q straight into Q_host, which must then be
 *     page-locked;
 *   - R goes to R_host after the tree (by a kernel when R_host is
 *     page-locked, else by a copy).
 *   A_host (m x n, column-major, lda_host >= m), read only; Q_host (m x n,
 *   ldq_host >= m) and R_host (n x n upper triangular, diag >= 0,
 *   ldr_host >= n), written.
 *   A, R: device buffers of the same shapes (lda >= m, ldr >= n),
 *   caller-owned; A ends holding the Householder vectors (the handle
 *   borrows it, as after tsqr_refactor), R the R factor.  Q: a device
 *   buffer (ldq >= m) that ends holding the thin Q, or NULL; not A.
 * Asynchronous on `stream`: when `stream` reaches the end of the call, all
 * host outputs are written; until then A_host must not change (the kernels
 * or copies may still be reading it).  Returns TSQR_OK, TSQR_ERR_HANDLE,
 * TSQR_ERR_UNSUPPORTED (hybrid or flat trees), -i for argument i (2..13)
 * invalid (-10 also for Q = NULL with a pageable Q_host), or a CUDA error
 * code.
 */
int tsqr_factor_form_host(tsqr_q_t q, const void* A_host, int64_t lda_host, void* Q_host, int64_t ldq_host,
                          void* R_host, int64_t ldr_host, void* A, int64_t lda, void* Q, int64_t ldq, void* R,
                          int64_t ldr, tsqr_stream_t stream);

/*
 * tsqr_sync_status: waits for the handle's work on `stream`, returns and
 * clears the latched device status (TSQR_OK, TSQR_ERR_NONFINITE, ...).
 */
int tsqr_sync_status(tsqr_q_t q, tsqr_stream_t stream);

/*
 * tsqr_q_info: shape and plan of a handle.  Any output pointer may be NULL.
 * levels counts tree levels above the leaves.
 */
int tsqr_q_info(tsqr_q_t q, int64_t* m, int64_t* n, int32_t* precision, int64_t* leaves,
                int64_t* leaf_rows, int32_t* arity, int32_t* levels);

/* ------------------------------------------------------ least squares -- */

/*
 * tsqr_lstsq: least-squares solutions X = argmin ||A X - B||_F of the
 * factored A (m x n, full column rank) for k right-hand sides, the use of
 * TSQR that Section 1 starts from, with the square Q applied as its tree:
 *     Q^T B = [C; D],   X = R^{-1} C,   ||A x_j - b_j||_2 = ||D(:, j)||_2.
 *   q     : handle of A from tsqr_factor / tsqr_refactor (not destroyed).
 *   R     : device, the n x n R of that factorisation (ldr >= n).
 *   B     : device, m x k (ldb >= m), overwritten by Q^T B.
 *   X     : device, n x k (ldx >= n), receives the solutions; may not alias B.
 *   rnorm : device array of k entries receiving the residual norms, or NULL.
 * Element type: the handle's.  A zero or non-finite diagonal entry of R
 * (rank-deficient A) latches TSQR_ERR_NONFINITE in the handle's status.
 * rnorm needs k <= 65535 and k doubles of stream-ordered temporary memory
 * (cudaMallocAsync); FP64 sums of squares (entries beyond about 1e150 in
 * magnitude overflow).  Asynchronous on `stream`.
 */
int tsqr_lstsq(tsqr_q_t q, const void* R, int64_t ldr, int64_t k, void* B, int64_t ldb, void* X, int64_t ldx,
               void* rnorm, tsqr_stream_t stream);

/*
 * tsqr_solve_r: X <- R^{-1} X for upper-triangular R (n x n, n <= 128,
 * ldr >= n) and X (n x k, ldx >= n), device arrays of `precision`
 * (TSQR_PREC_FP64 or TSQR_PREC_FP32), by back substitution on the device.
 * With the R-only variant of least squares that Section 1 mentions -- factor
 * [A, B] and keep only R = [R11, R12; 0, R22] -- the solution is
 * tsqr_solve_r on R11 and a copy of R12.  status: NULL, or a device int
 * that receives TSQR_ERR_NONFINITE's bit (value 1) when R has a zero or
 * non-finite diagonal entry.  Asynchronous on `stream`.
 */
int tsqr_solve_r(int64_t n, int64_t k, int32_t precision, const void* R, int64_t ldr, void* X, int64_t ldx,
                 int* status, tsqr_stream_t stream);

/*
 * tsqr_column_norms: norms[j] = ||B(:, j)||_2 for the m x k device matrix B
 * (ldb >= m, k <= 65535), FP64 sums of squares, written in `precision`
 * (the residual norms of the R-only variant are the column norms of R22).
 * Uses k doubles of stream-ordered temporary memory.
 */
int tsqr_column_norms(int64_t m, int64_t k, int32_t precision, const void* B, int64_t ldb, void* norms,
                      tsqr_stream_t stream);

/*
 * tsqr_q_part: copies one stored factor of a leaf or tree node of a factored
 * handle into `out` (device, caller-owned), asynchronously on `stream`:
 *   what = TSQR_PART_R   : the node's R before sign normalisation (n x n, ld n,
 *                          upper triangle; for leaves the leaf R_i of
 *                          Eq. TSQR_binarytree_1, for level l >= 1 the R of
 *                          Eqs. TSQR_binarytree_2/3);
 *          TSQR_PART_T   : its compact-WY T (n x n, ld n, upper triangular):
 *                          the product of its reflectors is I - Y T Y^T
 *                          (Schreiber and Van Loan, cited in Section 2.1);
 *          TSQR_PART_TAU : its n reflector coefficients tau;
 *          TSQR_PART_Y   : level >= 1 only: the q-1 upper-triangular blocks of
 *                          its Householder vectors below the unit top block
 *                          ((q-1) x n x n, each ld n; a leaf's Y is in A).
 *   level: 0 for leaves, 1..levels for tree levels; index < items on that
 *   level (with a hybrid tree, level-0 R is per chain, T and tau per leaf).
 * Elements are in the handle's storage type.  Returns TSQR_ERR_HANDLE for an
 * unfactored handle, -i for argument i out of range.
 */
enum tsqr_part { TSQR_PART_R = 0, TSQR_PART_T = 1, TSQR_PART_TAU = 2, TSQR_PART_Y = 3 };
int tsqr_q_part(tsqr_q_t q, int32_t what, int32_t level, int64_t index, void* out, tsqr_stream_t stream);

/* tsqr_q_chains: leaves per chain and number of chains (1 and the leaf
 * count unless the handle was planned with a hybrid or flat tree).  Either
 * pointer may be NULL. */
int tsqr_q_chains(tsqr_q_t q, int64_t* leaves_per_chain, int64_t* chains);

/* tsqr_q_destroy: frees the handle and its workspace (after its queued work). */
int tsqr_q_destroy(tsqr_q_t q);

/*
 * tsqr_factor_r_noalloc: R (n x n, diag(R) >= 0, zeros below the diagonal)
 * of the FP64 m x n matrix A, allocating no device memory.  The paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc -- code
 * running inside another allocator's callback, plugins of frameworks that
 * own all device memory, processes whose memory budget is fixed up front.
 *   Arguments as for tsqr_factor (A is overwritten by the leaf reflectors),
 *   without options or a Q handle: leaves of a power-of-two height (128
 *   rows at n = 64), binary tree, R-only kernels (no compact-WY T).
 *   n > 64 returns TSQR_ERR_UNSUPPORTED.
 *   Workspace comes from one static 64 MiB device array inside the library,
 *   held by every GPU that loads the library until the process exits.
 *   Problems whose tree workspace does not fit (about 3 * n*n*8 bytes per
 *   leaf; at n = 64, m up to roughly 87,000 rows) return TSQR_ERR_TOO_LARGE
 *   without touching the GPU.
 *   The first call on a device, and the first after that device's context
 *   was re-created (cudaDeviceReset), looks up the array's address: make it
 *   before any stream capture.  Calls share the array: calls whose GPU work
 *   overlaps (other streams, other host threads) race and must be
 *   serialised by the caller.  Device-side conditions are not reported.
 */
int tsqr_factor_r_noalloc(int64_t m, int64_t n, double* A, int64_t lda, double* R, int64_t ldr,
                          tsqr_stream_t stream);

/* ---------------------------------------------------------------- CAQR -- */

/*
 * caqr_factor: right-looking Householder QR whose panel factorisation is
 * TSQR (Section 3).
 *   A (device, m x n, lda >= m, m >= n) is overwritten by R in its upper
 *   triangle (diag(R) >= 0) and the panels' leaf Householder vectors below.
 *   b is the panel width (1 <= b; the last panel may be narrower).
 *   update_precision: TSQR_PREC_FP64 (caqr_factor, double storage), or
 *   TSQR_PREC_FP32 / TSQR_UPDATE_BF16X3 / TSQR_UPDATE_TF32X3 (caqr_factor_f32,
 *   float storage).
 * For panel j the trailing columns receive (Q_j D_j)^T: first the leaf
 * blocks, then the tree nodes on stacked b-row slices (Section 3.1), then
 * the panel's signs, so rows of R stay consistent without a later fix.
 * The next panel is factored on a handle-owned stream of the highest
 * priority while the rest of the trailing matrix is updated, and in FP64
 * half of each wide trailing update runs on a second handle-owned stream;
 * both join the caller's stream, so the call is complete when the work it
 * queued there is.  Calls with the same handle must not overlap.
 */
int caqr_factor(int64_t m, int64_t n, double* A, int64_t lda, int64_t b, int32_t update_precision,
                const tsqr_opts_t* opts, caqr_q_t* q, tsqr_stream_t stream);
int caqr_factor_f32(int64_t m, int64_t n, float* A, int64_t lda, int64_t b, int32_t update_precision,
                    const tsqr_opts_t* opts, caqr_q_t* q, tsqr_stream_t stream);

/*
 * Plan-once form of CAQR: caqr_q_create plans every panel of an m x n
 * problem with panel width b and allocates all panel workspaces at once;
 * caqr_refactor then factors a matrix of that shape (device, lda >= m; double
 * for TSQR_PREC_FP64, float otherwise) in place with no allocation of
 * device workspace.  caqr_factor = create + one factorisation.
 * Unless stage timing is on (caqr_q_set_timing), caqr_refactor captures its
 * panel loop into a CUDA graph on the first call for a given (A, lda) and
 * replays that graph on the caller's stream in later calls with the same
 * pair (a new pair is captured anew); the contents of A may change freely
 * between calls.  Errors of the capture are returned like launch errors.
 */
int caqr_q_create(int64_t m, int64_t n, int64_t b, int32_t update_precision, const tsqr_opts_t* opts,
                  caqr_q_t* q, tsqr_stream_t stream);
int caqr_refactor(caqr_q_t q, void* A, int64_t lda, tsqr_stream_t stream);

/* caqr_apply_qt: C (m x k, ldc >= m) <- Q^T C, panels in factorisation order. */
int caqr_apply_qt(caqr_q_t q, int64_t k, void* C, int64_t ldc, tsqr_stream_t stream);

/* caqr_apply_q: C <- Q C, panels in reverse order. */
int caqr_apply_q(caqr_q_t q, int64_t k, void* C, int64_t ldc, tsqr_stream_t stream);

/* caqr_form_q: thin Q (m x n, ldq >= m), Q must not alias A. */
int caqr_form_q(caqr_q_t q, void* Q, int64_t ldq, tsqr_stream_t stream);

int caqr_sync_status(caqr_q_t q, tsqr_stream_t stream);

/* Stage timing summed over every panel of a CAQR handle; the leaf-apply
 * stage is the trailing-matrix update (same semantics as the tsqr_ forms). */
int caqr_q_set_timing(caqr_q_t q, int32_t enable);
int caqr_q_stage_times(caqr_q_t q, double* ms, int64_t* launches, int32_t count);
int caqr_q_destroy(caqr_q_t q);

/* ------------------------------------------------------------ gradient -- */

/*
 * tsqr_qr_backward: the adjoint of the thin QR A = Q R (diag(R) > 0, full
 * column rank) for a loss with gradients dQ (m x n) and dR (n x n, only its
 * upper triangle is read).  The paper has no gradient; this is the standard
 * adjoint
 *     M = R dR^T - dQ^T Q,   dA = (dQ + Q copyltu(M)) R^{-T},
 * copyltu(M) = tril(M) + tril(M, -1)^T, computed on the device as a
 * tall-skinny reduction (dQ^T Q), an n x n step (M, R^{-1} by back
 * substitution, copyltu(M) R^{-T}) and a row-parallel product
 * dA = [dQ, Q] [R^{-T}; copyltu(M) R^{-T}].
 *   precision: TSQR_PREC_FP64 (double) or TSQR_PREC_FP32 (float) for every
 *   array; all arrays device, column-major; dA must not alias the inputs.
 *   status: NULL, or a device int that receives TSQR_ERR_NONFINITE's bit
 *   (value 1) when R has a zero or non-finite diagonal entry.
 * Temporary device memory comes from cudaMallocAsync on `stream`.
 */
int tsqr_qr_backward(int64_t m, int64_t n, int32_t precision, const void* Q, int64_t ldq, const void* R, int64_t ldr,
                     const void* dQ, int64_t lddq, const void* dR, int64_t lddr, void* dA, int64_t ldda, int* status,
                     tsqr_stream_t stream);

/* ------------------------------------------------------------- batched -- */

/*
 * Batched uneven TSQR: `count` independent problems A_i (m_i x n_i, m_i >=
 * n_i, 1 <= n_i <= 64) factored by ONE persistent kernel launch.  Each
 * problem gets its own leaves and tree (Section 2.1: every tree gives the same
 * R); the launch walks a device work list of all leaves, then all tree levels,
 * and a node starts when a device counter shows its children are done (a
 * bounded wait; a wait that gives up latches TSQR_ERR_TIMEOUT).
 */
typedef struct tsqr_batch_s* tsqr_batch_t;

typedef struct tsqr_batch_opts_s {
  int32_t tile_kb;  /* leaf tile budget in KB: h = largest power of two with n*h*elem <= tile_kb KB (0 = auto) */
  int32_t arity;    /* tree arity, 2..16 (0 = 2) */
  int32_t autotune; /* nonzero: time (tile_kb, arity) candidates on scratch matrices of these shapes, keep the fastest */
  int32_t reserved; /* must be 0 */
} tsqr_batch_opts_t;

/*
 * tsqr_batch_create: plans the batch and binds it to the matrices.
 *   m, n, lda, ldr : HOST arrays of count entries.
 *   A, R           : HOST arrays of count DEVICE pointers (column-major A_i,
 *                    overwritten like tsqr_factor's A; R_i receives n_i x n_i
 *                    R with diag >= 0, zeros below).
 *   precision      : TSQR_PREC_FP32 (FP32 storage, FP64 norms / tau) or FP64.
 * Allocates all workspace and the device work list; the matrices must stay
 * allocated while the handle lives.
 */
int tsqr_batch_create(int32_t count, const int64_t* m, const int64_t* n, void* const* A, const int64_t* lda,
                      void* const* R, const int64_t* ldr, int32_t precision, const tsqr_batch_opts_t* opts,
                      tsqr_batch_t* b, tsqr_stream_t stream);

/* tsqr_batch_factor: factors every bound matrix (counter reset + one persistent kernel launch). */
int tsqr_batch_factor(tsqr_batch_t b, tsqr_stream_t stream);

/* tsqr_batch_factor_graph: the same launch sequence, captured once into a CUDA graph and replayed. */
int tsqr_batch_factor_graph(tsqr_batch_t b, tsqr_stream_t stream);

/* tsqr_batch_info: chosen tile budget and arity, number of work items, device bytes held. */
int tsqr_batch_info(tsqr_batch_t b, int32_t* tile_kb, int32_t* arity, int64_t* items, int64_t* workspace_bytes);

int tsqr_batch_sync_status(tsqr_batch_t b, tsqr_stream_t stream);
int tsqr_batch_destroy(tsqr_batch_t b);

/* ----------------------------------------------------------- tracing -- */

/*
 * Per-stage device time of a handle's calls, measured with CUDA events that
 * the library records on each call's stream around its kernel launches.
 * Stages follow the cost terms of Section 2.2: the leaf QRs, the tree levels
 * (including the sign fix), the leaf block-reflector applications (apply,
 * form Q), and the tree-level applications.
 */
enum tsqr_stage {
  TSQR_STAGE_LEAF_FACTOR = 0,
  TSQR_STAGE_TREE_FACTOR = 1,
  TSQR_STAGE_LEAF_APPLY = 2,
  TSQR_STAGE_TREE_APPLY = 3,
  TSQR_NUM_STAGES = 4
};

/* tsqr_q_set_timing: enable != 0 clears the totals and starts recording,
 * enable == 0 stops recording (totals are kept). */
int tsqr_q_set_timing(tsqr_q_t q, int32_t enable);

/* tsqr_q_stage_times: waits for the recorded events and writes, for stages
 * 0..count-1, the summed milliseconds (ms[i]) and the number of kernel
 * launches (launches[i]) since timing was enabled.  Either array may be NULL. */
int tsqr_q_stage_times(tsqr_q_t q, double* ms, int64_t* launches, int32_t count);

/* -------------------------------------------------------------- misc -- */

/* Static string for a return code. */
const char* tsqr_status_string(int code);

/* Library version as major * 10000 + minor * 100 + patch. */
int tsqr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TSQR_GB300_H */
