// k x k steps of Algorithm 1, the fixed-order reductions, and the vector kernels of set-up, exit
// and the Chronopoulos-Gear CG baseline.
#include "kernels.h"
#include "small_kernels.cuh"

namespace mbpcg {

// One CTA of kReduceThreads per entry: thread t sums the partials p = t, t + kReduceThreads, ...,
// each warp combines its lanes by a butterfly, and thread 0 adds the warp sums in warp order
// (a fixed order: the same bits on every run).
__global__ void __launch_bounds__(kReduceThreads)
k_reduce(const double* __restrict__ part, int nparts, int pstride, double* __restrict__ out, int nent,
         const SolveState* __restrict__ st) {
  __shared__ double ws[kReduceThreads / 32];
  const int e = blockIdx.x, tid = threadIdx.x;
  if (e >= nent) return;
  // batches of kB partials per thread, all loads of a batch in flight together; the first batch
  // is loaded with the solve state (a skipped launch discards it), so the two L2 round trips
  // overlap. The adds keep the partials' order.
  constexpr int kB = 4;
  double v[kB];
  auto load = [&](int p0) {
#pragma unroll
    for (int b = 0; b < kB; ++b) {
      const int p = p0 + b * kReduceThreads;
      v[b] = p < nparts ? part[(size_t)p * pstride + e] : 0.0;
    }
  };
  load(tid);
  if (st != nullptr && st->done) return;
  double a = 0.0;
  for (int p0 = tid; p0 < nparts; p0 += kB * kReduceThreads) {
    if (p0 != tid) load(p0);
#pragma unroll
    for (int b = 0; b < kB; ++b)
      if (p0 + b * kReduceThreads < nparts) a += v[b];
  }
  for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
  if ((tid & 31) == 0) ws[tid >> 5] = a;
  __syncthreads();
  if (tid == 0) {
    double t = ws[0];
    for (int w = 1; w < kReduceThreads / 32; ++w) t += ws[w];
    out[e] = t;
  }
}

void launch_reduce(cudaStream_t s, const double* part, int nparts, int pstride, double* out, int nent,
                   const SolveState* st) {
  k_reduce<<<nent, kReduceThreads, 0, s>>>(part, nparts, pstride, out, nent, st);
}

__global__ void k_params(SolveState* st, double tol_rel, int maxit, int no_test, int restart, int s, int stag) {
  st->tol_rel = tol_rel;
  st->maxit = maxit;
  st->no_test = no_test;
  st->restart = restart;
  st->s = s;
  st->kerr = 0;
  st->stag_check = stag;
}

// Set-up scalars: ||rhs||, X0 = (||B||_F / ||A U||_F) U with ||B||_F = sqrt(s) ||D^{-1} rhs||.
__global__ void k_small_setup(SolveState* st, const double* __restrict__ red) {
  const double rn = sqrt(red[0]), bsn = sqrt(red[1]), aun = sqrt(red[2]);
  st->rhs_norm = rn;
  if (st->restart == 0) st->b_norm = rn;
  st->scale = (aun > 0.0) ? sqrt((double)st->s) * bsn / aun : 0.0;
  st->tol_abs = st->tol_rel * rn;
  st->it = 0;
  st->done = 0;
  st->r_from_v = 0;
  st->nu_ref = INFINITY;
  st->it_ref = 0;
  st->stagnated = 0;
  st->pw_skip = 0;
  st->status = 0;
  st->converged = 0;
  st->ls_fallback = 0;
  st->best_col = 0;
  st->nu_h = 0.0;
  st->ls_res = 0.0;
}

// Exit combination (Section 2): c = argmin ||rhs - Bhat c||, Bhat = B - R (Proposition 1), in the
// original metric. Written as min ||[rhs | D R] y|| subject to sum(y) = 1 with y = (1 - 1^T c, c)
// (the same minimiser), solved on the column-equilibrated (s+1) x (s+1) Gram:
//   y = G^{-1} 1 / (1^T G^{-1} 1),  ||residual||^2 = 1 / (1^T G^{-1} 1).
// Falls back to c = e_h when the Gram is not numerically positive definite, a value is not
// finite, or the combination is no better than column h. Without convergence (breakdown or
// maxit) the exit is the best column of the current residual block.
__global__ void __launch_bounds__(kSmallThreads)
k_small_ls(SolveState* st, const double* __restrict__ Mg, int kp, double* __restrict__ c_out) {
  constexpr int LD = kMaxKP + 1;
  __shared__ double A[LD * LD], sc[LD], y[LD], z[LD];
  __shared__ int flag, fallback;
  const int s = st->s, m = s + 1;
  const int np = npack(kp);
  if (!st->converged) {
    if (threadIdx.x == 0) {
      int h = 0;
      for (int j = 1; j < s; ++j)
        if (Mg[pidx(j, j)] < Mg[pidx(h, h)]) h = j;
      st->best_col = h;
      st->nu_h = sqrt(Mg[pidx(h, h)]);
      st->ls_res = st->nu_h;
      st->ls_fallback = 1;
      for (int j = 0; j < kp; ++j) c_out[j] = (j == h) ? 1.0 : 0.0;
    }
    return;
  }
  // G over index 0 = rhs, 1 + j = (D R)_j ; column-major, ld LD
  for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
    const int a = q % m, b = q / m;
    double v;
    if (a == 0 && b == 0) v = Mg[np + kp];
    else if (a == 0) v = Mg[np + b - 1];
    else if (b == 0) v = Mg[np + a - 1];
    else v = (a <= b) ? Mg[pidx(a - 1, b - 1)] : Mg[pidx(b - 1, a - 1)];
    A[a + b * LD] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    fallback = 0;
    for (int a = 0; a < m; ++a) {
      const double g = A[a + a * LD];
      if (!(g > 0.0) || !isfinite(g)) fallback = 1;
      sc[a] = 1.0 / sqrt(g);
    }
  }
  __syncthreads();
  if (!fallback) {
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
      const int a = q % m, b = q / m;
      A[a + b * LD] *= sc[a] * sc[b];
    }
    __syncthreads();
    if (cta_cholesky(m, LD, A, &flag)) fallback = 1;  // uniform: every thread sees the same flag
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double rl = 0.0;
    if (!fallback) {
      // Z^T y = sc (forward), Z z = y (back); denom = sc^T z
      for (int i = 0; i < m; ++i) {
        double v = sc[i];
        for (int l = 0; l < i; ++l) v = fma(-A[l + i * LD], y[l], v);
        y[i] = v / A[i + i * LD];
      }
      for (int i = m - 1; i >= 0; --i) {
        double v = y[i];
        for (int l = i + 1; l < m; ++l) v = fma(-A[i + l * LD], z[l], v);
        z[i] = v / A[i + i * LD];
      }
      double denom = 0.0;
      for (int i = 0; i < m; ++i) denom = fma(sc[i], z[i], denom);
      rl = sqrt(1.0 / denom);
      if (!(denom > 0.0) || !isfinite(denom) || !isfinite(rl) || rl > st->nu_h) fallback = 1;
      for (int j = 0; j < s && !fallback; ++j) {
        const double cj = sc[j + 1] * z[j + 1] / denom;
        if (!isfinite(cj)) fallback = 1;
      }
    }
    const int h = st->best_col;
    if (fallback) {
      for (int j = 0; j < kp; ++j) c_out[j] = (j == h) ? 1.0 : 0.0;
      st->ls_res = st->nu_h;
      st->ls_fallback = 1;
    } else {
      double denom = 0.0;
      for (int i = 0; i < m; ++i) denom = fma(sc[i], z[i], denom);
      for (int j = 0; j < kp; ++j) c_out[j] = (j < s) ? sc[j + 1] * z[j + 1] / denom : 0.0;
      st->ls_res = rl;
      st->ls_fallback = 0;
    }
  }
}

__global__ void k_small_true(SolveState* st, const double* __restrict__ rr) {
  st->true_res = sqrt(rr[0]);
}

// ------------------------------------------------------------------ Chronopoulos-Gear CG scalars

__global__ void k_small_cg_setup(SolveState* st, const double* __restrict__ red) {
  const double rn = sqrt(red[0]);
  st->rhs_norm = rn;
  if (st->restart == 0) st->b_norm = rn;
  st->tol_abs = st->tol_rel * rn;
  st->it = 0;
  st->done = 0;
  st->pw_skip = 1;
  st->status = 0;
  st->converged = 0;
  st->ls_fallback = 0;
  st->best_col = 0;
  st->cg_gamma_old = 0.0;
  st->cg_alpha_old = 0.0;
  st->cg_alpha = 0.0;
  st->cg_beta = 0.0;
  st->ls_res = 0.0;
  st->nu_h = 0.0;
}

// gamma = (r, u), delta = (w, u) with u = r and w = A u; test ||D r|| < tol ||rhs||; then
// beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old) (first step:
// beta = 0, alpha = gamma / delta). Sets the WHILE condition (use_cond = 0 outside a graph).
__global__ void k_small_cg(SolveState* st, const double* __restrict__ red, cudaGraphConditionalHandle cond,
                           int use_cond) {
  if (st->done) {
    if (use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  const double gamma = red[0], delta = red[1], nu = sqrt(red[2]);
  st->nu_h = nu;
  st->ls_res = nu;
  if (nu < st->tol_abs) {
    st->converged = 1;
    st->done = 1;
    st->status = 0;
    if (use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  if (st->it >= st->maxit) {
    st->done = 1;
    st->status = 5;
    if (use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  double alpha, beta;
  if (st->it == 0) {
    beta = 0.0;
    alpha = gamma / delta;
  } else {
    beta = gamma / st->cg_gamma_old;
    alpha = gamma / (delta - beta * gamma / st->cg_alpha_old);
  }
  if (!isfinite(alpha) || !(alpha > 0.0)) {
    st->done = 1;
    st->status = 6;
    if (use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  st->cg_alpha = alpha;
  st->cg_beta = beta;
  st->cg_gamma_old = gamma;
  st->cg_alpha_old = alpha;
  st->it += 1;
  if (use_cond) cudaGraphSetConditional(cond, 1);
}

// ------------------------------------------------------------------ vector kernels

// CSR structure check: row_ptr[0] = 0, monotone, row_ptr[n] = nnz, 0 <= col < n  (flag |= 1).
__global__ void k_validate_csr(int n, long long nnz, const int* __restrict__ rp, const int* __restrict__ ci,
                               int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && (rp[0] != 0 || (long long)rp[n] != nnz)) atomicOr(flag, 1);
  if (i < n) {
    const int a = rp[i], b = rp[i + 1];
    if (b < a || a < 0 || (long long)b > nnz) {
      atomicOr(flag, 1);
      return;
    }
    for (int p = a; p < b; ++p) {
      const int c = ci[p];
      if (c < 0 || c >= n) {
        atomicOr(flag, 1);
        return;
      }
    }
  }
}

// diag_i = sum of the entries (i, i) of row i; flag |= 2 if not positive and finite.
__global__ void k_diag_csr(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ av,
                           double* __restrict__ diag, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) a += av[p];
  diag[i] = a;
  if (!(a > 0.0) || !isfinite(a)) atomicOr(flag, 2);
}

__global__ void k_diag_dense(int n, const double* __restrict__ A, double* __restrict__ diag, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = A[(size_t)i * n + i];
  diag[i] = a;
  if (!(a > 0.0) || !isfinite(a)) atomicOr(flag, 2);
}

// flag |= 4 if any of the count values is NaN or infinite (grid-stride; one atomic per warp).
__global__ void k_check_finite(long long count, const double* __restrict__ v, int* __restrict__ flag) {
  bool bad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    bad |= !isfinite(v[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 4);
}

// d = 1/sqrt(diag) (= D^{-1} of Section 1), sqd = sqrt(diag) (= D), wdiag = diag (= D^2).
__global__ void k_make_scaling(int n, const double* __restrict__ diag, double* __restrict__ d,
                               double* __restrict__ sqd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = sqrt(diag[i]);
  sqd[i] = r;
  d[i] = 1.0 / r;
}

// In-place D^{-1} A D^{-1}.
__global__ void k_scale_csr(int n, const int* __restrict__ rp, const int* __restrict__ ci, double* __restrict__ av,
                            const double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double di = d[i];
  for (int p = rp[i]; p < rp[i + 1]; ++p) av[p] = di * av[p] * d[ci[p]];
}

__global__ void k_scale_dense(int n, double* __restrict__ A, const double* __restrict__ d) {
  const size_t total = (size_t)n * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const size_t l = q / n, i = q % n;  // column l, row i
    A[q] = d[i] * A[q] * d[l];
  }
}

// True residual r = b - A x on the original A, reconstructed from the scaled matrix:
// (A x)_i = D_i sum_j Abar_ij D_j x_j  (sqd = D, or NULL without scaling). CTA partials of ||r||^2.
__global__ void __launch_bounds__(kThreads)
k_resid_csr(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ av,
            const double* __restrict__ sqd, const double* __restrict__ b, const double* __restrict__ x,
            double* __restrict__ r, double* __restrict__ part, int pstride) {
  __shared__ double red[kThreads];
  int r0, r1;
  row_range(n, r0, r1);
  double acc = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += kThreads) {
    double a = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int c = ci[p];
      const double xc = (sqd != nullptr) ? sqd[c] * x[c] : x[c];
      a = fma(av[p], xc, a);
    }
    const double ri = (sqd != nullptr) ? fma(-sqd[i], a, b[i]) : b[i] - a;
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  red[threadIdx.x] = acc;
  cta_tree_sum(red, kThreads, 1);
  if (threadIdx.x == 0) part[(size_t)blockIdx.x * pstride] = red[0];
}

// Dense version: one warp per row, lanes over the reduction index.
__global__ void __launch_bounds__(kThreads)
k_resid_dense(int n, const double* __restrict__ A, const double* __restrict__ sqd, const double* __restrict__ b,
              const double* __restrict__ x, double* __restrict__ r, double* __restrict__ part, int pstride) {
  __shared__ double red[kThreads / 32];
  int r0, r1;
  row_range(n, r0, r1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int i = r0 + warp; i < r1; i += kThreads / 32) {
    const double* ai = A + (size_t)i * n;
    double a = 0.0;
    for (int l = lane; l < n; l += 32) {
      const double xl = (sqd != nullptr) ? sqd[l] * x[l] : x[l];
      a = fma(ai[l], xl, a);
    }
    for (int off = 16; off >= 1; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    const double ri = (sqd != nullptr) ? fma(-sqd[i], a, b[i]) : b[i] - a;
    if (lane == 0) {
      r[i] = ri;
      acc = fma(ri, ri, acc);
    }
  }
  if (lane == 0) red[warp] = acc;
  cta_tree_sum(red, kThreads / 32, 1);
  if (threadIdx.x == 0) part[(size_t)blockIdx.x * pstride] = red[0];
}

// CG set-up on the scaled system: r = D^{-1} rhs, x = p = s = 0; CTA partial of ||rhs||^2.
__global__ void __launch_bounds__(kThreads)
k_cg_init(int n, const double* __restrict__ rhs, const double* __restrict__ d, double* __restrict__ r,
          double* __restrict__ x, double* __restrict__ p, double* __restrict__ sv, double* __restrict__ part,
          int pstride) {
  __shared__ double red[kThreads];
  int r0, r1;
  row_range(n, r0, r1);
  double acc = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const double bi = rhs[i];
    r[i] = (d != nullptr) ? d[i] * bi : bi;
    x[i] = p[i] = sv[i] = 0.0;
    acc = fma(bi, bi, acc);
  }
  red[threadIdx.x] = acc;
  cta_tree_sum(red, kThreads, 1);
  if (threadIdx.x == 0) part[(size_t)blockIdx.x * pstride] = red[0];
}

// CTA partials of (r, r), (w, r) and ||D r||^2 (wdiag = D^2 or NULL).
__global__ void __launch_bounds__(kThreads)
k_cg_dots(int n, const double* __restrict__ r, const double* __restrict__ w, const double* __restrict__ wdiag,
          double* __restrict__ part, int pstride, const SolveState* __restrict__ st) {
  if (st->done) return;
  __shared__ double red[3 * kThreads];
  int r0, r1;
  row_range(n, r0, r1);
  double g = 0.0, dl = 0.0, nu = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const double ri = r[i];
    g = fma(ri, ri, g);
    dl = fma(w[i], ri, dl);
    nu = (wdiag != nullptr) ? fma(ri * wdiag[i], ri, nu) : fma(ri, ri, nu);
  }
  red[threadIdx.x * 3] = g;
  red[threadIdx.x * 3 + 1] = dl;
  red[threadIdx.x * 3 + 2] = nu;
  cta_tree_sum(red, kThreads, 3);
  if (threadIdx.x < 3) part[(size_t)blockIdx.x * pstride + threadIdx.x] = red[threadIdx.x];
}

// p = u + beta p;  s = w + beta s (s = A p);  x += alpha p;  r -= alpha s.
__global__ void __launch_bounds__(kThreads)
k_cg_update(int n, double* __restrict__ r, const double* __restrict__ w, double* __restrict__ x,
            double* __restrict__ p, double* __restrict__ sv, const SolveState* __restrict__ st) {
  if (st->done) return;
  const double alpha = st->cg_alpha, beta = st->cg_beta;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
    const double ri = r[i];
    const double pi = fma(beta, p[i], ri);
    const double si = fma(beta, sv[i], w[i]);
    p[i] = pi;
    sv[i] = si;
    x[i] = fma(alpha, pi, x[i]);
    r[i] = fma(-alpha, si, ri);
  }
}

// x_total += D^{-1} xbar.
__global__ void k_cg_finish(int n, const double* __restrict__ xbar, const double* __restrict__ d,
                            double* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] += (d != nullptr) ? d[i] * xbar[i] : xbar[i];
}

// dst = FP32 rounding of src (the mixed-precision copies of the scaled matrix values and diag A).
__global__ void k_to_f32(long long n, const double* __restrict__ src, float* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// Implicit-residual mode: nu_j = sigma_j^T G sigma_j for the columns j < s, into red[npack(kp) + j],
// where G (packed upper triangle at red[goff ...)) is V^T V, or V^T D^2 V with scaling, and sigma_j
// is column j of Sigma (upper triangular): the column norms of the new residual block V Sigma in
// the original metric. One warp per column; lane a forms (G sigma_j)_a.
__global__ void k_small_nu(SolveState* st, double* __restrict__ red, const double* __restrict__ Sigma, int kp,
                           int goff) {
  if (st->done) return;
  const int j = blockIdx.x, a = threadIdx.x, s = st->s;
  if (j >= s) return;
  double t = 0.0;
  if (a < s) {
    for (int b = 0; b <= j; ++b) {
      const double g = (a <= b) ? red[goff + pidx(a, b)] : red[goff + pidx(b, a)];
      t = fma(g, Sigma[b + j * kp], t);
    }
  }
  double v = (a <= j && a < s) ? Sigma[a + j * kp] * t : 0.0;
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (a == 0) red[npack(kp) + j] = v;
}

}  // namespace mbpcg
