/*
 * MBPCG oracle -- TEST INFRASTRUCTURE ONLY (see mbpcg_oracle.h).
 *
 * Plain FP64 C, single thread, no BLAS, no blocking, no fusion: each function writes out the
 * definition or the algorithm step it cites so that it can be checked against the paper by eye.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may use this file.
 */
#include "mbpcg_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_INVALID = 1, ORC_NOT_SPD = 4, ORC_NOT_CONVERGED = 5, ORC_BREAKDOWN = 6 };

/* Loops whose iterations are independent (one column, row or entry each, every sum inside one
 * iteration in its sequential order) are marked ORC_PAR. The parity build compiles without OpenMP
 * and ignores the mark; the timed CPU-baseline build (-fopenmp) shares those iterations among the
 * host cores, which changes no sum's order and so gives the same bits. */
#ifdef _OPENMP
#define ORC_PAR _Pragma("omp parallel for schedule(static)")
#define ORC_PAR2 _Pragma("omp parallel for collapse(2) schedule(static)")
#else
#define ORC_PAR
#define ORC_PAR2
#endif

typedef struct {
  int32_t n;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
  const double* dense; /* column-major n*n, or NULL */
} orc_mat;

/* ---------------------------------------------------------------- basic dense/sparse algebra */

/* Y = A X, X and Y column-major n*k. Dense A is walked column by column (axpy form). */
static void mat_block(const orc_mat* A, int32_t k, const double* X, double* Y) {
  const int32_t n = A->n;
  ORC_PAR
  for (int32_t j = 0; j < k; ++j) {
    const double* x = X + (size_t)j * n;
    double* y = Y + (size_t)j * n;
    if (A->dense) {
      for (int32_t i = 0; i < n; ++i) y[i] = 0.0;
      for (int32_t l = 0; l < n; ++l) {
        const double* a = A->dense + (size_t)l * n;
        const double xl = x[l];
        for (int32_t i = 0; i < n; ++i) y[i] += a[i] * xl;
      }
    } else {
      for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t p = A->row_ptr[i]; p < A->row_ptr[i + 1]; ++p) s += A->val[p] * x[A->col_idx[p]];
        y[i] = s;
      }
    }
  }
}

static double dot(int32_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* C (m*k) = A^T B for column-major A (n*m), B (n*k). */
static void gram(int32_t n, int32_t m, int32_t k, const double* A, const double* B, double* C) {
  ORC_PAR2
  for (int32_t a = 0; a < m; ++a)
    for (int32_t c = 0; c < k; ++c) C[a + (size_t)c * m] = dot(n, A + (size_t)a * n, B + (size_t)c * n);
}

/* C (n*k) = A (n*k) S (k*k); C must not alias A. */
static void block_times_small(int32_t n, int32_t k, const double* A, const double* S, double* C) {
  ORC_PAR
  for (int32_t j = 0; j < k; ++j)
    for (int32_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int32_t l = 0; l < k; ++l) s += A[i + (size_t)l * n] * S[l + (size_t)j * k];
      C[i + (size_t)j * n] = s;
    }
}

/* C (k*k) = S1 S2. */
static void small_times_small(int32_t k, const double* S1, const double* S2, double* C) {
  for (int32_t j = 0; j < k; ++j)
    for (int32_t i = 0; i < k; ++i) {
      double s = 0.0;
      for (int32_t l = 0; l < k; ++l) s += S1[i + l * k] * S2[l + j * k];
      C[i + j * k] = s;
    }
}

/* Upper Cholesky factor Z of an SPD k*k matrix G = Z^T Z (Z with positive diagonal).
 * Breakdown when a pivot is not finite or not above 64*eps*max_j G_jj. */
static int chol_upper(int32_t k, const double* G, double* Z) {
  double maxd = 0.0;
  for (int32_t j = 0; j < k; ++j) maxd = fmax(maxd, fabs(G[j + j * k]));
  memset(Z, 0, sizeof(double) * (size_t)k * k);
  for (int32_t j = 0; j < k; ++j) {
    double s = G[j + j * k];
    for (int32_t l = 0; l < j; ++l) s -= Z[l + j * k] * Z[l + j * k];
    if (!isfinite(s) || !(s > 64.0 * DBL_EPSILON * maxd)) return ORC_BREAKDOWN;
    const double zjj = sqrt(s);
    Z[j + j * k] = zjj;
    for (int32_t m = j + 1; m < k; ++m) {
      double t = G[j + m * k];
      for (int32_t l = 0; l < j; ++l) t -= Z[l + j * k] * Z[l + m * k];
      Z[j + m * k] = t / zjj;
    }
  }
  return ORC_OK;
}

/* Inverse of an SPD matrix from its upper Cholesky factor: G^{-1} = Z^{-1} Z^{-T}, column by
 * column through two triangular solves on the identity (Section 3: Xi applied through the
 * Cholesky factor, no explicit inversion of P^T A P). */
static void spd_inverse_from_chol(int32_t k, const double* Z, double* Ginv) {
  double* y = (double*)malloc(sizeof(double) * (size_t)k);
  for (int32_t j = 0; j < k; ++j) {
    /* Z^T y = e_j (forward substitution; Z^T is lower triangular) */
    for (int32_t i = 0; i < k; ++i) {
      double s = (i == j) ? 1.0 : 0.0;
      for (int32_t l = 0; l < i; ++l) s -= Z[l + i * k] * y[l];
      y[i] = s / Z[i + i * k];
    }
    /* Z x = y (back substitution) */
    for (int32_t i = k - 1; i >= 0; --i) {
      double s = y[i];
      for (int32_t l = i + 1; l < k; ++l) s -= Z[i + l * k] * Ginv[l + j * k];
      Ginv[i + j * k] = s / Z[i + i * k];
    }
  }
  free(y);
}

/* W = V Z^{-1} for an upper triangular Z: each row w solves w Z = v. */
static void right_solve_upper(int32_t n, int32_t k, const double* V, const double* Z, double* W) {
  ORC_PAR
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < k; ++j) {
      double s = V[i + (size_t)j * n];
      for (int32_t l = 0; l < j; ++l) s -= W[i + (size_t)l * n] * Z[l + j * k];
      W[i + (size_t)j * n] = s / Z[j + j * k];
    }
}

/* Cholesky QR of an n*k block (Section 3, after Fukaya et al. 2014): G = V^T V, Z = chol(G)
 * upper, Q = V Z^{-1}. Returns the status of the Cholesky step. */
static int cholesky_qr(int32_t n, int32_t k, const double* V, double* Q, double* Z) {
  double* G = (double*)malloc(sizeof(double) * (size_t)k * k);
  gram(n, k, k, V, V, G);
  int st = chol_upper(k, G, Z);
  if (st == ORC_OK) right_solve_upper(n, k, V, Z, Q);
  free(G);
  return st;
}

/* Least squares min_c ||y - M c|| by Householder QR of the n*k matrix M (destroyed).
 * Returns 0 on success, 1 when a Householder column is exactly zero. */
static int householder_lstsq(int32_t n, int32_t k, double* M, const double* y_in, double* c) {
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* rdiag = (double*)malloc(sizeof(double) * (size_t)k);
  memcpy(y, y_in, sizeof(double) * (size_t)n);
  int fail = 0;
  for (int32_t j = 0; j < k && !fail; ++j) {
    double* v = M + (size_t)j * n; /* column j, rows j..n-1 hold the reflector */
    double nx = 0.0;
    for (int32_t i = j; i < n; ++i) nx += v[i] * v[i];
    nx = sqrt(nx);
    if (nx == 0.0) { fail = 1; break; }
    const double alpha = (v[j] > 0.0) ? -nx : nx; /* H x = alpha e_1 */
    v[j] -= alpha;
    double vv = 0.0;
    for (int32_t i = j; i < n; ++i) vv += v[i] * v[i];
    rdiag[j] = alpha;
    if (vv == 0.0) continue;
    for (int32_t m = j + 1; m < k; ++m) { /* apply H = I - 2 v v^T / (v^T v) */
      double* col = M + (size_t)m * n;
      double s = 0.0;
      for (int32_t i = j; i < n; ++i) s += v[i] * col[i];
      s = 2.0 * s / vv;
      for (int32_t i = j; i < n; ++i) col[i] -= s * v[i];
    }
    double s = 0.0;
    for (int32_t i = j; i < n; ++i) s += v[i] * y[i];
    s = 2.0 * s / vv;
    for (int32_t i = j; i < n; ++i) y[i] -= s * v[i];
  }
  if (!fail) { /* R c = (Q^T y)[0:k]; R_jm (m > j) sits in M after the reflections */
    for (int32_t j = k - 1; j >= 0; --j) {
      double s = y[j];
      for (int32_t m = j + 1; m < k; ++m) s -= M[j + (size_t)m * n] * c[m];
      c[j] = s / rdiag[j];
    }
  }
  free(y);
  free(rdiag);
  return fail;
}

/* ------------------------------------------------------------------ diagonal scaling (Sec. 1) */

/* D_jj = sqrt(A_jj); the scaled matrix is D^{-1} A D^{-1} and d_j = 1/D_jj. With precond == 0,
 * d = 1 and the scaled matrix is A itself (the arrays are copied in both cases). */
static int scale_system(const orc_mat* A, int32_t precond, double* d, double** val_s, double** dense_s) {
  const int32_t n = A->n;
  for (int32_t i = 0; i < n; ++i) d[i] = 1.0;
  if (precond) {
    for (int32_t i = 0; i < n; ++i) {
      double aii = 0.0;
      if (A->dense) aii = A->dense[i + (size_t)i * n];
      else
        for (int32_t p = A->row_ptr[i]; p < A->row_ptr[i + 1]; ++p)
          if (A->col_idx[p] == i) aii += A->val[p];
      if (!(aii > 0.0) || !isfinite(aii)) return ORC_NOT_SPD;
      d[i] = 1.0 / sqrt(aii);
    }
  }
  if (A->dense) {
    *dense_s = (double*)malloc(sizeof(double) * (size_t)n * n);
    for (int32_t l = 0; l < n; ++l)
      for (int32_t i = 0; i < n; ++i) (*dense_s)[i + (size_t)l * n] = d[i] * A->dense[i + (size_t)l * n] * d[l];
  } else {
    const int32_t nnz = A->row_ptr[n];
    *val_s = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    for (int32_t i = 0; i < n; ++i)
      for (int32_t p = A->row_ptr[i]; p < A->row_ptr[i + 1]; ++p) (*val_s)[p] = d[i] * A->val[p] * d[A->col_idx[p]];
  }
  return ORC_OK;
}

static int validate(const orc_mat* A, int32_t k) {
  if (A->n < 1 || k < 1) return ORC_INVALID;
  if (A->dense) return ORC_OK;
  if (!A->row_ptr || A->row_ptr[0] != 0) return ORC_INVALID;
  for (int32_t i = 0; i < A->n; ++i) {
    if (A->row_ptr[i + 1] < A->row_ptr[i]) return ORC_INVALID;
    for (int32_t p = A->row_ptr[i]; p < A->row_ptr[i + 1]; ++p)
      if (A->col_idx[p] < 0 || A->col_idx[p] >= A->n) return ORC_INVALID;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ Algorithm 1 (one solve) */

typedef struct {
  int32_t iterations, status, best_col, ls_fallback;
  double relres_recurrence, relres_ls;
} core_result;

/*
 * One MBPCG solve of A x = rhs (Algorithm 1, Section 2) on the scaled matrix As (= D^{-1}AD^{-1}),
 * with d = diag(D^{-1}). Writes delta = the solution in ORIGINAL variables.
 *   force_iters >= 0: run exactly that many iterations, no exit test, and return the raw state;
 *   force_iters < 0: a normal solve.
 */
static void mbpcg_core(const orc_mat* As, const double* d, const double* rhs, const double* U, int32_t k,
                       double tol, int32_t maxit, int32_t restart, double* delta, double* c_out,
                       core_result* res, orc_iter_cb cb, void* user, int32_t force_iters, double* st_X0,
                       double* st_Xt, double* st_R, double* st_W, double* st_P, double* st_Sigma) {
  const int32_t n = As->n;
  const size_t nk = (size_t)n * k, kk = (size_t)k * k;
  double* X0 = (double*)calloc(nk, sizeof(double));
  double* Xt = (double*)calloc(nk, sizeof(double));
  double* R = (double*)calloc(nk, sizeof(double));
  double* W = (double*)calloc(nk, sizeof(double));
  double* P = (double*)calloc(nk, sizeof(double));
  double* Q = (double*)calloc(nk, sizeof(double)); /* Q = A P */
  double* V = (double*)calloc(nk, sizeof(double));
  double* Tmp = (double*)calloc(nk, sizeof(double));
  double* bs = (double*)calloc((size_t)n, sizeof(double));
  double* Sigma = (double*)calloc(kk, sizeof(double));
  double* G = (double*)calloc(kk, sizeof(double));
  double* Z = (double*)calloc(kk, sizeof(double));
  double* Xi = (double*)calloc(kk, sizeof(double));
  double* T = (double*)calloc(kk, sizeof(double));
  double* S2 = (double*)calloc(kk, sizeof(double));
  double* nu = (double*)calloc((size_t)k, sizeof(double));
  double* c = (double*)calloc((size_t)k, sizeof(double));
  memset(res, 0, sizeof(*res));
  res->best_col = 0;
  res->status = ORC_NOT_CONVERGED;

  const double bnorm = sqrt(dot(n, rhs, rhs));
  for (int32_t i = 0; i < n; ++i) bs[i] = d[i] * rhs[i]; /* scaled right-hand side D^{-1} b */

  /* X0 = (||B||_F / ||A U||_F) U, with B = [b ... b] (k copies) */
  mat_block(As, k, U, Tmp); /* Tmp = A U */
  const double normB = sqrt((double)k) * sqrt(dot(n, bs, bs));
  const double normAU = sqrt(dot((int32_t)nk, Tmp, Tmp));
  const double scale = (normAU > 0.0) ? normB / normAU : 0.0;
  for (size_t q = 0; q < nk; ++q) X0[q] = scale * U[q];
  /* B~ = B - A X0 = B - scale * A U;  X~0 = O;  R0 = B~ */
  for (int32_t j = 0; j < k; ++j)
    for (int32_t i = 0; i < n; ++i) R[i + (size_t)j * n] = bs[i] - scale * Tmp[i + (size_t)j * n];
  /* W0, Sigma0 = qr(R0);  P0 = W0 */
  int st = cholesky_qr(n, k, R, W, Sigma);
  if (st == ORC_OK) {
    memcpy(P, W, sizeof(double) * nk);
    if (cb && force_iters < 0) cb(user, 0, 0, restart, X0, Xt, R, W, P, Sigma);
  }

  int32_t it = 0;
  int exiting = 0;
  while (st == ORC_OK) {
    if (force_iters >= 0 && it == force_iters) break;
    if (force_iters < 0 && it >= maxit) break;
    ++it;
    /* Xi = (P^T A P)^{-1}, applied through the Cholesky factor of P^T A P (Section 3) */
    mat_block(As, k, P, Q);
    gram(n, k, k, P, Q, G);
    st = chol_upper(k, G, Z);
    if (st != ORC_OK) { --it; break; }
    spd_inverse_from_chol(k, Z, Xi);
    small_times_small(k, Xi, Sigma, T); /* T = Xi Sigma */
    /* X~ = X~ + P Xi Sigma;  R = R - A P Xi Sigma */
    block_times_small(n, k, P, T, Tmp);
    ORC_PAR
    for (size_t q = 0; q < nk; ++q) Xt[q] += Tmp[q];
    block_times_small(n, k, Q, T, Tmp);
    ORC_PAR
    for (size_t q = 0; q < nk; ++q) R[q] -= Tmp[q];
    if (force_iters < 0) {
      /* h = argmin_j ||R_j|| / ||b||, measured on the original-system residual D R (Section 1) */
      ORC_PAR
      for (int32_t j = 0; j < k; ++j) {
        double s = 0.0;
        for (int32_t i = 0; i < n; ++i) {
          const double r = R[i + (size_t)j * n] / d[i];
          s += r * r;
        }
        nu[j] = sqrt(s);
      }
      int32_t h = 0;
      for (int32_t j = 1; j < k; ++j)
        if (nu[j] < nu[h]) h = j;
      res->best_col = h;
      res->relres_recurrence = (bnorm > 0.0) ? nu[h] / bnorm : 0.0;
      if (nu[h] < tol * bnorm) {
        /* Bhat = B - R, c = argmin ||b - Bhat c||, r = b - Bhat c (original metric) */
        double* M = (double*)malloc(sizeof(double) * nk);
        for (int32_t j = 0; j < k; ++j)
          for (int32_t i = 0; i < n; ++i) M[i + (size_t)j * n] = rhs[i] - R[i + (size_t)j * n] / d[i];
        int fail = householder_lstsq(n, k, M, rhs, c);
        double rl = 0.0;
        if (!fail) {
          for (int32_t i = 0; i < n; ++i) {
            double s = rhs[i];
            for (int32_t j = 0; j < k; ++j) s -= (rhs[i] - R[i + (size_t)j * n] / d[i]) * c[j];
            rl += s * s;
          }
          rl = sqrt(rl);
        }
        /* fall back to the best column when the least-squares step is not usable (Section 2) */
        int finite = !fail && isfinite(rl);
        for (int32_t j = 0; j < k && finite; ++j) finite = isfinite(c[j]);
        if (!finite || rl > nu[h]) {
          for (int32_t j = 0; j < k; ++j) c[j] = (j == h) ? 1.0 : 0.0;
          rl = nu[h];
          res->ls_fallback = 1;
        } else {
          res->ls_fallback = 0;
        }
        free(M);
        res->relres_ls = (bnorm > 0.0) ? rl / bnorm : 0.0;
        if (rl < tol * bnorm) { /* convergence tolerance (set equal to the initial one) */
          exiting = 1;
          if (cb) cb(user, it, 1, restart, X0, Xt, R, W, P, Sigma);
          break;
        }
      }
    }
    /* W, zeta = qr(W - A P Xi);  P = W + P zeta^T;  Sigma = zeta Sigma */
    block_times_small(n, k, Q, Xi, Tmp);
    ORC_PAR
    for (size_t q = 0; q < nk; ++q) V[q] = W[q] - Tmp[q];
    st = cholesky_qr(n, k, V, W, Z);
    if (st != ORC_OK) break;
    ORC_PAR
    for (int32_t j = 0; j < k; ++j)
      for (int32_t i = 0; i < n; ++i) {
        double s = W[i + (size_t)j * n];
        for (int32_t l = j; l < k; ++l) s += P[i + (size_t)l * n] * Z[j + l * k]; /* (P zeta^T)_ij */
        Tmp[i + (size_t)j * n] = s;
      }
    memcpy(P, Tmp, sizeof(double) * nk);
    small_times_small(k, Z, Sigma, S2);
    memcpy(Sigma, S2, sizeof(double) * kk);
    if (cb && force_iters < 0) cb(user, it, 0, restart, X0, Xt, R, W, P, Sigma);
  }
  res->iterations = it;

  if (force_iters >= 0) {
    res->status = st;
    memcpy(st_X0, X0, sizeof(double) * nk);
    memcpy(st_Xt, Xt, sizeof(double) * nk);
    memcpy(st_R, R, sizeof(double) * nk);
    memcpy(st_W, W, sizeof(double) * nk);
    memcpy(st_P, P, sizeof(double) * nk);
    memcpy(st_Sigma, Sigma, sizeof(double) * kk);
  } else {
    if (exiting) res->status = ORC_OK;
    else {
      res->status = (st != ORC_OK) ? ORC_BREAKDOWN : ORC_NOT_CONVERGED;
      /* best iterate without an exit test: the best column of the current recurrence residual */
      int32_t h = 0;
      for (int32_t j = 0; j < k; ++j) {
        double s = 0.0;
        for (int32_t i = 0; i < n; ++i) {
          const double r = R[i + (size_t)j * n] / d[i];
          s += r * r;
        }
        nu[j] = sqrt(s);
        if (nu[j] < nu[h]) h = j;
      }
      for (int32_t j = 0; j < k; ++j) c[j] = (j == h) ? 1.0 : 0.0;
      res->best_col = h;
      res->relres_recurrence = (bnorm > 0.0) ? nu[h] / bnorm : 0.0;
      res->relres_ls = res->relres_recurrence;
      res->ls_fallback = 1;
    }
    /* X = X~ + X0;  x = X c;  back to the original variables x = D^{-1} xbar */
    for (int32_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int32_t j = 0; j < k; ++j) s += (Xt[i + (size_t)j * n] + X0[i + (size_t)j * n]) * c[j];
      delta[i] = d[i] * s;
    }
    if (c_out) memcpy(c_out, c, sizeof(double) * (size_t)k);
  }
  free(X0); free(Xt); free(R); free(W); free(P); free(Q); free(V); free(Tmp); free(bs);
  free(Sigma); free(G); free(Z); free(Xi); free(T); free(S2); free(nu); free(c);
}

/* ------------------------------------------------------- Chronopoulos-Gear CG (one solve) */

/* Chronopoulos & Gear (1989) single-reduction CG on the scaled matrix As with zero start:
 * per iteration one product w = A u, the two inner products (r,u) and (w,u) together, then
 * alpha, beta and the updates of p, s = A p, x and r. Test on ||D r|| / ||b||. */
static void cgear_core(const orc_mat* As, const double* d, const double* rhs, double tol, int32_t maxit,
                       double* delta, core_result* res) {
  const int32_t n = As->n;
  double* x = (double*)calloc((size_t)n, sizeof(double));
  double* r = (double*)calloc((size_t)n, sizeof(double));
  double* u = (double*)calloc((size_t)n, sizeof(double));
  double* w = (double*)calloc((size_t)n, sizeof(double));
  double* p = (double*)calloc((size_t)n, sizeof(double));
  double* s = (double*)calloc((size_t)n, sizeof(double));
  memset(res, 0, sizeof(*res));
  const double bnorm = sqrt(dot(n, rhs, rhs));
  for (int32_t i = 0; i < n; ++i) r[i] = d[i] * rhs[i];
  double gamma_old = 0.0, alpha_old = 0.0;
  int32_t it = 0;
  int converged = 0;
  for (;;) {
    memcpy(u, r, sizeof(double) * (size_t)n); /* u = M^{-1} r with M = I on the scaled system */
    mat_block(As, 1, u, w);
    const double gamma = dot(n, r, u), delta_ = dot(n, w, u);
    double nr = 0.0;
    for (int32_t i = 0; i < n; ++i) nr += (r[i] / d[i]) * (r[i] / d[i]);
    res->relres_recurrence = (bnorm > 0.0) ? sqrt(nr) / bnorm : 0.0;
    if (sqrt(nr) < tol * bnorm) { converged = 1; break; }
    if (it >= maxit) break;
    double alpha, beta;
    if (it == 0) {
      beta = 0.0;
      alpha = gamma / delta_;
    } else {
      beta = gamma / gamma_old;
      alpha = gamma / (delta_ - beta * gamma / alpha_old);
    }
    if (!isfinite(alpha) || !(alpha > 0.0)) { res->status = ORC_BREAKDOWN; break; }
    for (int32_t i = 0; i < n; ++i) {
      p[i] = u[i] + beta * p[i];
      s[i] = w[i] + beta * s[i];
      x[i] += alpha * p[i];
      r[i] -= alpha * s[i];
    }
    gamma_old = gamma;
    alpha_old = alpha;
    ++it;
  }
  res->iterations = it;
  if (converged) res->status = ORC_OK;
  else if (res->status != ORC_BREAKDOWN) res->status = ORC_NOT_CONVERGED;
  res->relres_ls = res->relres_recurrence;
  for (int32_t i = 0; i < n; ++i) delta[i] = d[i] * x[i];
  free(x); free(r); free(u); free(w); free(p); free(s);
}

/* ------------------------------------------- true-residual check and restart (both solvers) */

/* Recompute r = b - A x from the original A after each solve; while ||r||/||b|| > tol, solve the
 * correction system A e = r to 0.5 tol ||b|| / ||r|| and set x += e (at most max_restarts). */
static int solve_with_restarts(const orc_mat* A, const double* b, const double* U, int32_t k, int32_t precond,
                               double tol, int32_t maxit, int32_t max_restarts, int use_cg, double* x,
                               double* c_out, orc_info* info, orc_iter_cb cb, void* user) {
  const int32_t n = A->n;
  memset(info, 0, sizeof(*info));
  int st = validate(A, use_cg ? 1 : k);
  if (st == ORC_OK && !(tol > 0.0)) st = ORC_INVALID;
  if (st != ORC_OK) { info->status = st; return st; }
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  double *val_s = NULL, *dense_s = NULL;
  st = scale_system(A, precond, d, &val_s, &dense_s);
  if (st != ORC_OK) { free(d); info->status = st; return st; }
  orc_mat As = *A;
  if (A->dense) As.dense = dense_s; else As.val = val_s;

  double* rhs = (double*)malloc(sizeof(double) * (size_t)n);
  double* e = (double*)malloc(sizeof(double) * (size_t)n);
  double* Ax = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(rhs, b, sizeof(double) * (size_t)n);
  for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
  const double bnorm = sqrt(dot(n, b, b));
  double tol_inner = tol;
  int32_t total = 0, restarts = 0;
  core_result res;
  for (;;) {
    if (use_cg) cgear_core(&As, d, rhs, tol_inner, maxit - total, e, &res);
    else mbpcg_core(&As, d, rhs, U, k, tol_inner, maxit - total, restarts, e, c_out, &res, cb, user, -1,
                    NULL, NULL, NULL, NULL, NULL, NULL);
    total += res.iterations;
    for (int32_t i = 0; i < n; ++i) x[i] += e[i];
    mat_block(A, 1, x, Ax);
    double rr = 0.0;
    for (int32_t i = 0; i < n; ++i) {
      rhs[i] = b[i] - Ax[i];
      rr += rhs[i] * rhs[i];
    }
    const double relres = (bnorm > 0.0) ? sqrt(rr) / bnorm : 0.0;
    info->relres_true = relres;
    info->relres_recurrence = res.relres_recurrence;
    info->relres_ls = res.relres_ls;
    info->best_col = res.best_col;
    info->ls_fallback = res.ls_fallback;
    if (relres <= tol) { st = ORC_OK; break; }
    if (restarts >= max_restarts || total >= maxit || res.status == ORC_NOT_CONVERGED) {
      st = (res.status == ORC_OK) ? ORC_NOT_CONVERGED : res.status;
      break;
    }
    ++restarts;
    tol_inner = 0.5 * tol * bnorm / sqrt(rr);
  }
  info->iterations = total;
  info->restarts = restarts;
  info->status = st;
  free(rhs); free(e); free(Ax); free(d); free(val_s); free(dense_s);
  return st;
}

/* ------------------------------------------------------------------------------- public API */

int orc_matmat(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
               const double* dense, int32_t k, const double* X, double* Y) {
  orc_mat A = {n, row_ptr, col_idx, val, dense};
  if (validate(&A, k) != ORC_OK) return ORC_INVALID;
  mat_block(&A, k, X, Y);
  return ORC_OK;
}

int orc_mbpcg(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
              const double* dense, const double* b, const double* U, int32_t k, int32_t precond,
              double tol, int32_t maxit, int32_t max_restarts, double* x_out, double* c_out,
              orc_info* info, orc_iter_cb cb, void* user) {
  orc_mat A = {n, row_ptr, col_idx, val, dense};
  return solve_with_restarts(&A, b, U, k, precond, tol, maxit, max_restarts, 0, x_out, c_out, info, cb, user);
}

int orc_cg_cgear(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                 const double* dense, const double* b, int32_t precond, double tol, int32_t maxit,
                 int32_t max_restarts, double* x_out, orc_info* info) {
  orc_mat A = {n, row_ptr, col_idx, val, dense};
  return solve_with_restarts(&A, b, NULL, 1, precond, tol, maxit, max_restarts, 1, x_out, NULL, info, NULL, NULL);
}

int orc_mbpcg_state(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                    const double* dense, const double* b, const double* U, int32_t k,
                    int32_t precond, int32_t iters, double* X0, double* Xt, double* R, double* W,
                    double* P, double* Sigma) {
  orc_mat A = {n, row_ptr, col_idx, val, dense};
  int st = validate(&A, k);
  if (st != ORC_OK || iters < 0) return ORC_INVALID;
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  double *val_s = NULL, *dense_s = NULL;
  st = scale_system(&A, precond, d, &val_s, &dense_s);
  if (st == ORC_OK) {
    orc_mat As = A;
    if (dense) As.dense = dense_s; else As.val = val_s;
    double* delta = (double*)malloc(sizeof(double) * (size_t)n);
    core_result res;
    mbpcg_core(&As, d, b, U, k, 0.0, iters, 0, delta, NULL, &res, NULL, NULL, iters,
               X0, Xt, R, W, P, Sigma);
    st = res.status;
    free(delta);
  }
  free(d); free(val_s); free(dense_s);
  return st;
}
