/*
 * mbpcg.h -- C ABI of the GB300 (sm_103a) Multi-Basis Parallel Conjugate Gradient library.
 *
 * The method (Algorithm 1, Section 2 of the paper): solve one SPD system A x = b by running block
 * CG (Dubrulle-R form, Cholesky QR of Section 3) over s copies of the system that start from
 * s random initial guesses, and return the least-squares combination of the s iterates.
 * The paper's baseline, Chronopoulos-Gear CG (Section 1, Section 4), runs through the same API.
 *
 * Everything after create runs on the GPU: set-up, every iteration, the exit step and the
 * true-residual check. The library never falls back to a CPU path; without a usable CUDA
 * device every call returns MBPCG_ERR_CUDA.
 *
 * Memory and ownership
 *   - Functions without the _dev suffix take HOST pointers; they copy in and out on the handle's
 *     stream and return after the result is on the host.
 *   - Functions with the _dev suffix take DEVICE pointers (any allocation visible to the device,
 *     e.g. a torch tensor's data_ptr) and return after the result is written (the call ends with
 *     a synchronisation of the handle's stream).
 *   - The handle owns every internal buffer. They are sized at create for (n, nnz, s) and either
 *     allocated by the library (workspace == NULL) or carved out of a caller-provided device
 *     workspace of at least mbpcg_workspace_size_*() bytes (the caller keeps ownership and must
 *     keep it alive until mbpcg_destroy).
 *   - Blocks of s vectors crossing the ABI (U) are column-major n x s, as the paper stores dense
 *     matrices (Section 3). Inside, blocks are row-major with s padded to a power of two.
 *
 * Errors: every int-returning function returns an mbpcg_status. Nothing aborts or throws across
 * the ABI. mbpcg_last_error() gives a thread-local message for the last failure.
 * Threading: a handle is not thread-safe; distinct handles may be used concurrently.
 */
#ifndef MBPCG_H
#define MBPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbpcg_ctx* mbpcg_handle;

typedef enum {
  MBPCG_OK = 0,
  MBPCG_ERR_INVALID = 1,   /* bad argument, malformed CSR or non-finite A (checked at create) */
  MBPCG_ERR_OOM = 2,       /* device allocation failed or workspace too small */
  MBPCG_ERR_CUDA = 3,      /* CUDA runtime error (see mbpcg_last_error) */
  MBPCG_ERR_NOT_SPD = 4,   /* a diagonal entry is missing, not positive or not finite */
  MBPCG_NOT_CONVERGED = 5, /* maxit reached; x_out holds the best iterate */
  MBPCG_BREAKDOWN = 6,     /* a k x k Cholesky pivot was not positive; x_out holds the best iterate */
  MBPCG_ERR_TIMEOUT = 7    /* a bounded device-side wait (TMA/mbarrier) ran out of time */
} mbpcg_status;

/* Symmetric diagonal scaling of Section 1: D = diag(sqrt(A_jj)), the solver runs on
 * D^{-1} A D^{-1}; residual norms and the tolerance refer to the original system. */
typedef enum { MBPCG_PRECOND_NONE = 0, MBPCG_PRECOND_JACOBI = 1 } mbpcg_precond;

/* MBPCG = Algorithm 1 with s copies; CG = Chronopoulos-Gear CG with zero initial guess (the
 * paper's baseline, Section 4), s ignored. */
typedef enum { MBPCG_ALGO_MBPCG = 0, MBPCG_ALGO_CG = 1 } mbpcg_algo;

/* Arithmetic of the n-proportional work. FP64: everything in double precision on the FP64 pipe.
 * MIXED_FP32 (MBPCG only; CSR or dense A): the inner solves keep the n x s blocks and the (scaled)
 * matrix in FP32 (a dense A adds an FP32 copy, n x round_up(n, 32) floats, to the workspace) and do
 * the products and block updates in FP32 with FP32 accumulation; the s x s
 * Grams and norms are accumulated with FP64-class accuracy (compensated FP32 dot products, Ogita,
 * Rump & Oishi 2005), the s x s Cholesky steps run in FP64, and the true residual b - A x and x
 * itself are FP64: the true-residual restarts are an FP64 iterative refinement loop (at most 12
 * correction solves, each asked for at most 1e-5 relative reduction). Results therefore differ from
 * the FP64 path; the requested tol is still checked on the FP64 true residual.
 * MIXED_BF16 (2): reserved for a BF16 tensor-core inner solve of dense A; not built -- every
 * create call with it returns MBPCG_ERR_INVALID. A BF16 copy of A loses SPD-ness wherever
 * kappa(A) * 2^-8 is not small (kappa = 1e6 here), and at the condition numbers this library is
 * measured on the FP64 tensor-core product below is the faster dense solve.
 * FP64_TC (3; dense A, MBPCG only): the same FP64 solve, but the product A P runs on the tensor
 * cores by exact splitting of A and P into 8 signed base-128 digits (Ozaki scheme), FP16 operands
 * and FP32 accumulation in windows whose sums stay exact; every digit-pair level that can reach
 * 2^-60 of a row scale of A times a column scale of P is kept, so the result is at least as
 * accurate as an FP64 product (bound 1e-14 |A||P| entry by entry, tested). The digits of A take 8
 * bytes per entry of workspace. At s > 8 the k x k-row products of the block update and of the W/P
 * update (P T, (AP) T, (AP) Xi, V zeta^-1, P zeta^T) run on the tensor cores the same way (3 more
 * n x KP blocks of workspace); the Grams, the norms and the k x k steps stay FP64. */
typedef enum { MBPCG_FP64 = 0, MBPCG_MIXED_FP32 = 1, MBPCG_MIXED_BF16 = 2, MBPCG_FP64_TC = 3 } mbpcg_precision;

typedef struct {
  int32_t iterations;        /* inner iterations summed over restarts */
  int32_t restarts;          /* true-residual restarts taken (at most 3) */
  int32_t status;            /* mbpcg_status of the solve */
  int32_t best_col;          /* h = argmin_j ||R_j|| at the last exit test */
  int32_t ls_fallback;       /* 1 if the last exit used column h instead of the LS combination */
  int32_t reserved;
  double relres_recurrence;  /* ||R_h|| / ||b|| at the last exit test (original metric) */
  double relres_ls;          /* ||b - Bhat c|| / ||b|| of the last exit combination */
  double relres_true;        /* ||b - A x|| / ||b|| recomputed on the device from A */
  double seconds;            /* device time of the solve call (CUDA events) */
} mbpcg_info;

/* Workspace bytes a handle needs (device memory), for callers that allocate it themselves. */
size_t mbpcg_workspace_size_csr(int32_t n, int64_t nnz, int32_t s, int32_t algo, int32_t precision);
size_t mbpcg_workspace_size_dense(int32_t n, int32_t s, int32_t algo, int32_t precision);

/*
 * Create a solver for sparse A in CSR form (int32 row_ptr[n+1], int32 col_idx[nnz], double
 * vals[nnz], full symmetric storage, any column order within a row).
 *   mem       0: the three arrays are host pointers; 1: device pointers.
 *   s         number of copies, 1 <= s <= 32 (ignored for MBPCG_ALGO_CG).
 *   seed      seed of the counter-based generator used when mbpcg_solve gets U == NULL.
 *   workspace device buffer of mbpcg_workspace_size_csr() bytes, or NULL to let the library
 *             allocate; stream: a cudaStream_t, or NULL for a stream owned by the handle.
 * Validation: 1 <= n, 0 <= nnz < 2^31, row_ptr[0] = 0, row_ptr monotone, row_ptr[n] = nnz,
 * 0 <= col_idx < n, every value finite (MBPCG_ERR_INVALID); every row has a positive finite
 * diagonal (MBPCG_ERR_NOT_SPD). Symmetry is a precondition and is not checked.
 */
int mbpcg_create_csr(mbpcg_handle* out, int32_t n, int64_t nnz, const int32_t* row_ptr,
                     const int32_t* col_idx, const double* vals, int32_t s, int32_t precond,
                     int32_t algo, int32_t precision, uint64_t seed, int32_t mem, void* workspace,
                     size_t workspace_bytes, void* stream);

/* Create a solver for dense SPD A (column-major n x n doubles; A symmetric, so either triangle
 * may be read). Same conventions as mbpcg_create_csr; every entry must be finite
 * (MBPCG_ERR_INVALID). */
int mbpcg_create_dense(mbpcg_handle* out, int32_t n, const double* A_colmajor, int32_t s,
                       int32_t precond, int32_t algo, int32_t precision, uint64_t seed,
                       int32_t mem, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Solve A x = b to ||b - A x|| / ||b|| <= tol (Algorithm 1 with initial tolerance = convergence
 * tolerance = tol, as the paper's implementation sets them, Section 2).
 *   b     n doubles (host).     U: n x s column-major initial block (host) or NULL to draw it
 *         from Uniform(-1,1) with the handle's seed (SplitMix64, counter-based).
 *   maxit cap on inner iterations over all restarts (>= 1).
 *   x_out n doubles (host), caller-allocated. Filled on MBPCG_OK, MBPCG_NOT_CONVERGED and
 *         MBPCG_BREAKDOWN (best iterate). info may be NULL.
 * After the recurrence test passes, the residual b - A x is recomputed from A; while it exceeds
 * tol the solver restarts on the correction system (at most 3 times).
 */
int mbpcg_solve(mbpcg_handle h, const double* b, const double* U, double tol, int32_t maxit,
                double* x_out, mbpcg_info* info);

/* As mbpcg_solve with b, U (or NULL) and x_out in device memory. */
int mbpcg_solve_dev(mbpcg_handle h, const double* b, const double* U, double tol, int32_t maxit,
                    double* x_out, mbpcg_info* info);

/*
 * Diagnostic: run exactly `iters` iterations of Algorithm 1 (no exit test, no restart) from
 * the set-up with b and U (device pointers) and copy the state of the scaled system out to
 * device buffers, column-major n x s (X0, Xt, R, W, P) and s x s (Sigma). Any output pointer may
 * be NULL. MBPCG_ALGO_MBPCG handles only.
 */
int mbpcg_run_iterations_dev(mbpcg_handle h, const double* b, const double* U, int32_t iters,
                             double* X0, double* Xt, double* R, double* W, double* P,
                             double* Sigma);

/* How a solve drives its iteration loop. GRAPH (default): one CUDA graph launch per inner solve,
 * the loop being a device-side WHILE node. EAGER: the same kernels launched one by one from the
 * host, which checks the solve state every 16 iterations; meant for profilers (they do not see
 * kernel nodes of graphs with conditional nodes) and per-kernel timing. Results are identical. */
typedef enum { MBPCG_LAUNCH_GRAPH = 0, MBPCG_LAUNCH_EAGER = 1 } mbpcg_launch_mode;
int mbpcg_set_launch_mode(mbpcg_handle h, int32_t mode);

/* How the loop carries the residual block. EXPLICIT (default): R is updated every iteration as in
 * Algorithm 1 (R -= (A P) T). IMPLICIT: the Dubrulle-R identity R = W Sigma is used instead -- the
 * new residual block of an iteration is V Sigma, so its column norms (the best-basis test) are
 * sigma_j^T (V^T D^2 V) sigma_j from a Gram the iteration forms anyway (plus V^T D^2 V with
 * scaling), R is neither read nor written in the loop (16 n s bytes and n s^2 FMAs less per
 * iteration), and R is formed once before the exit. Not in the paper, which updates R explicitly;
 * results agree up to rounding. MBPCG handles with FP64 or FP64_TC precision only
 * (MBPCG_ERR_INVALID otherwise). Takes effect at the next solve. */
typedef enum { MBPCG_RESIDUAL_EXPLICIT = 0, MBPCG_RESIDUAL_IMPLICIT = 1 } mbpcg_residual_mode;
int mbpcg_set_residual_mode(mbpcg_handle h, int32_t mode);

/* Autotuner of the mixed-precision inner solve (MBPCG_MIXED_FP32 CSR handles; MBPCG_ERR_INVALID
 * otherwise: the dense FP32 product has one launch shape). At create the FP32 product A P -- the
 * dominant kernel of that solve -- is timed on the handle's own matrix in eleven shapes, given as
 * (variant, ctas_per_sm): the gather kernel (CTAs of 256 threads) with 4 or 8 nonzeros of a row in
 * flight per thread and 4, 8 or 16 CTAs per SM, (4,4) (4,8) (4,16) (8,4) (8,8) (8,16); the tiled
 * kernel, (0,2), when the matrix has a tiling plan; the wide-CTA kernel with 1024 threads, (1,1)
 * (1,2), and with 512 threads, (2,2) (2,4) (see mbpcg_get_product_kernel). CUDA events, three
 * launches each; the fastest is kept. Every shape sums each row the same way, so the shape changes
 * the time, never the result.
 *   mbpcg_get_spmm_tuning: the kept shape and the eleven measured times (microseconds per launch,
 *     in the order above; 0 for a shape not timed; times_us may be NULL).
 *   mbpcg_set_spmm_shape: impose one of the eleven shapes. */
int mbpcg_get_spmm_tuning(mbpcg_handle h, int32_t* unroll, int32_t* ctas_per_sm, float* times_us);
int mbpcg_set_spmm_shape(mbpcg_handle h, int32_t unroll, int32_t ctas_per_sm);

/* The product Y = A X of the handle's matrix, as the loop applies it (Algorithm 1: the A P of each
 * iteration). A is the stored operator: the matrix given at create, or D^-1/2 A D^-1/2 under
 * MBPCG_PRECOND_JACOBI. X and Y are device blocks of n rows x w columns, row-major, w the padded
 * block width (mbpcg_k_padded_width(s); 1 for MBPCG_ALGO_CG handles); FP64, or FP32 when fp32 != 0
 * (MBPCG_MIXED_FP32 handles only: the product of the inner solve). The caller owns both; X and Y
 * must not overlap. Enqueued on the handle's stream; returns without waiting. Uses the handle's
 * scratch (not to be called while a solve of the same handle runs on another thread). */
int mbpcg_apply_dev(mbpcg_handle h, int32_t fp32, const void* X, void* Y);

/* Which kernel forms the product (fp32 = 0: the FP64 product; 1: the FP32 product of a mixed
 * handle). CSR kernels: CSR_GATHER, each thread walks its row's nonzeros and gathers rows of P
 * through the caches (the FP64 product of the loop); CSR_WIDE (FP32 only), the same with CTAs of
 * 512 or 1024 threads, so that the rows an SM has in flight are few contiguous ranges whose rows of
 * P stay in L1; CSR_TILED, for CSR matrices of at least 65,536 rows whose tiles' columns fit a
 * shared-memory window (a plan built at create), the rows of P a tile reads are staged in shared
 * memory once and the nonzeros address them by 16-bit local indices. All sum each row in the order
 * of its nonzeros: A P is the same bits whichever runs; TILED groups the loop's Gram partials by
 * tile (other rounding). For FP64, GATHER is the loop's product, so a solve's result never
 * depends on a timing; it is timed at create on the handle's own matrix, with the loop's Gram, and
 * TILED when imposed -- times_us (may be NULL) receives the two measured microseconds per launch,
 * 0 when not timed. The plan of an FP64 handle is built on the host when CSR_TILED is first
 * imposed (a sort of every tile's columns: it is not paid at create); mixed handles build it at
 * create for the autotuner of mbpcg_get_spmm_tuning, which picks among all FP32 kernels.
 * mbpcg_set_product_kernel imposes the FP64 kernel of a CSR handle (CSR_TILED needs a plan;
 * MBPCG_ERR_INVALID when the matrix has none, or for a mixed handle). */
typedef enum {
  MBPCG_PRODUCT_CSR_GATHER = 0,
  MBPCG_PRODUCT_CSR_TILED = 1,
  MBPCG_PRODUCT_CSR_WIDE = 2,
  MBPCG_PRODUCT_DENSE = 3,
  MBPCG_PRODUCT_DENSE_TC = 4,
  MBPCG_PRODUCT_DENSE_FP32 = 5
} mbpcg_product_kernel;
int mbpcg_get_product_kernel(mbpcg_handle h, int32_t fp32, int32_t* kernel, float* times_us);
int mbpcg_set_product_kernel(mbpcg_handle h, int32_t kernel);

/* Rounding of the tensor-core product (MBPCG_FP64_TC handles; MBPCG_ERR_INVALID otherwise). The
 * product's digit-pair levels 0..4 are always summed exactly (int64); levels 5..8 (below 2^-49 of
 * the row and column scales) are, by default, carried in FP32 per window of 128 values of the
 * reduction index (MBPCG_ROUND_FP32_TAIL: error about 6e-16 ||A P|| on the benchmark system, and
 * iteration counts inside the band of the FP64 oracle). MBPCG_ROUND_ONCE keeps them as exact
 * integers too, so the product is rounded once, at the end (16 instead of 12 bytes of scratch per
 * partial, no FP32 rounding). Not in the paper: on a dense SPD system of n = 4096, kappa = 1e6,
 * s = 32, the solve then took 2144 iterations against 2354 with the default and 2388-2406 for the
 * FP64 method the paper describes -- its own product rounding slows that method there. Takes
 * effect at the next solve. */
typedef enum { MBPCG_ROUND_FP32_TAIL = 0, MBPCG_ROUND_ONCE = 1 } mbpcg_product_rounding;
int mbpcg_set_product_rounding(mbpcg_handle h, int32_t mode);

/* Batches of uneven systems/* Batches of uneven systems (NEXT row "batching"; not in the paper). A batch binds count existing
 * handles -- any mix of CSR and dense matrices, sizes, block widths, algorithms and precisions,
 * each created with MBPCG_LAUNCH_GRAPH -- and captures one inner solve of each (set-up, the
 * device-side WHILE loop, the exit) as an independent chain of ONE CUDA graph, built once at
 * mbpcg_batch_create. mbpcg_batch_solve_dev copies each member's b (and U) in on the member's
 * stream, launches the batch graph once on the batch's stream (the stream given at create, or one
 * of its own), so that the members' kernels run concurrently on the device, then runs each
 * member's true-residual restarts (or refinement steps) on the member's own graph and stream.
 * Every member runs the same kernels in the same order as a solo mbpcg_solve_dev, so its x and info
 * are bit-identical to a solo solve. b, U and x_out: arrays of count device pointers laid out as
 * for mbpcg_solve_dev (U may be NULL, or hold NULL entries: drawn from the handle's seed). info:
 * NULL or count entries. Returns MBPCG_OK when every member met tol, else the status of the first
 * member that did not (each member's own status is in info[i].status); errors as mbpcg_solve_dev.
 * A handle may belong to several batches, but two solves of one handle must not run at the same
 * time. mbpcg_batch_destroy releases the graph, not the handles. */
typedef struct mbpcg_batch_ctx* mbpcg_batch;
int mbpcg_batch_create(mbpcg_batch* out, const mbpcg_handle* handles, int32_t count, void* stream);
int mbpcg_batch_solve_dev(mbpcg_batch batch, const double* const* b, const double* const* U, double tol,
                          int32_t maxit, double* const* x_out, mbpcg_info* info);
void mbpcg_batch_destroy(mbpcg_batch batch);

/* Release a handle (NULL is ignored). */
void mbpcg_destroy(mbpcg_handle h);

const char* mbpcg_status_string(int status);
const char* mbpcg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
