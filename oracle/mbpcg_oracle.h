/*
 * MBPCG oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of the Multi-Basis Parallel Conjugate
 * Gradient method (Algorithm 1 of the paper, Section 2) and of the Chronopoulos-Gear CG it is
 * compared against (Section 1 and Section 4). Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it. It shares no code, header or constant with the CUDA
 * library and the CUDA library never calls it.
 *
 * Conventions
 *   - A is either CSR (row_ptr[n+1], col_idx[nnz], val[nnz], int32 indices) or dense column-major
 *     n*n (pass dense != NULL and the CSR pointers as NULL). A must be symmetric positive definite.
 *   - n*k blocks (U, X, R, W, P) are column-major, leading dimension n, as the paper stores dense
 *     matrices (Section 3).
 *   - k*k matrices are column-major, leading dimension k.
 *   - precond: 0 = none, 1 = symmetric diagonal (Jacobi) scaling of Section 1.
 *   - All tolerances are relative residual tolerances on the ORIGINAL system: ||b - A x|| / ||b||.
 *
 * Status codes (same numbering as the library's public header, written out independently):
 *   0 ok, 1 invalid argument, 4 non-positive diagonal with scaling, 5 not converged,
 *   6 breakdown (Cholesky pivot of a k*k Gram matrix not positive).
 *
 * Parity notes: every function below is pinned by tests that do not use the oracle itself
 * (closed forms, LAPACK/scipy solves, invariants of the method, brute force on tiny inputs).
 */
#ifndef MBPCG_ORACLE_H
#define MBPCG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t iterations;        /* inner iterations over all restarts */
  int32_t restarts;          /* number of true-residual restarts taken */
  int32_t status;
  int32_t best_col;          /* h of the final inner solve */
  int32_t ls_fallback;       /* 1 if the least-squares combination fell back to column h */
  int32_t pad;
  double relres_recurrence;  /* ||D R_h|| / ||b|| at the last exit test */
  double relres_ls;          /* ||b - Bhat c|| / ||b|| of the last exit (original metric) */
  double relres_true;        /* ||b - A x|| / ||b|| recomputed from A at the end */
} orc_info;

/* Called at the end of every full iteration (after the Sigma update) with the consistent state
 * X~^i, R^i, W^i, P^i, Sigma^i of the scaled system, and once with iter == 0 after set-up.
 * At the exit iteration it is called with exiting == 1 and X~, R updated (W, P, Sigma of the
 * previous iteration). X0 is the scaled initial guess. Pointers are valid during the call only. */
typedef void (*orc_iter_cb)(void* user, int32_t iter, int32_t exiting, int32_t restart,
                            const double* X0, const double* Xt, const double* R, const double* W,
                            const double* P, const double* Sigma);

/* Y = A X for an n*k column-major block X. */
int orc_matmat(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
               const double* dense, int32_t k, const double* X, double* Y);

/* Algorithm 1 with the readings listed in the design notes. U is n*k (column-major), used for
 * the first solve and for each true-residual restart. x_out (n) receives the solution in the
 * original variables; c_out (k, may be NULL) the least-squares coefficients of the last exit. */
int orc_mbpcg(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
              const double* dense, const double* b, const double* U, int32_t k, int32_t precond,
              double tol, int32_t maxit, int32_t max_restarts, double* x_out, double* c_out,
              orc_info* info, orc_iter_cb cb, void* user);

/* Chronopoulos-Gear CG (the paper's baseline "CG", Section 4), zero initial guess, on the
 * (optionally diagonally scaled) system, with the same true-residual restart rule as orc_mbpcg. */
int orc_cg_cgear(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                 const double* dense, const double* b, int32_t precond, double tol, int32_t maxit,
                 int32_t max_restarts, double* x_out, orc_info* info);

/* Runs exactly `iters` iterations of Algorithm 1 (no exit test, no restart) and returns the
 * raw state of the scaled system: Xt, R, W, P (n*k each), Sigma (k*k), X0 (n*k). Used by the
 * kernel-level parity tests. Returns 0 or 6 (breakdown). */
int orc_mbpcg_state(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                    const double* dense, const double* b, const double* U, int32_t k,
                    int32_t precond, int32_t iters, double* X0, double* Xt, double* R, double* W,
                    double* P, double* Sigma);

#ifdef __cplusplus
}
#endif
#endif
