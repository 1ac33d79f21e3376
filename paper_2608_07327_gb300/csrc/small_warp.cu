// The k x k steps of Algorithm 1 inside the iteration loop. For KP <= 8 one warp, lane j owning
// column j (k = s <= KP). On GB300 these are bound by FP64 latency, not throughput, so the algorithms
// are chosen for short dependency chains: a right-looking Cholesky with shuffles (no block-wide
// barriers), triangular solves in column (axpy) order, where each step is one multiply plus
// independent FMAs, and products that read their left factor from shared memory by broadcast.
//
// Padding: rows/columns s..KP-1 are factored as the identity and written back as zeros, so the row
// kernels keep the padded columns of every block at exactly zero.
#include <cfloat>

#include "kernels.h"

namespace mbpcg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Loads the symmetric s x s matrix whose upper triangle is packed in `packed` into column j = lane:
// a[i] = G[i][j] (i <= j), identity outside the leading s x s block.
template <int KP>
__device__ __forceinline__ void load_packed_column(const double* __restrict__ packed, int s, int j,
                                                   double (&a)[KP]) {
#pragma unroll
  for (int i = 0; i < KP; ++i) {
    double v = 0.0;
    if (i <= j) {
      if (j < s) v = packed[pidx(i, j)];
      else v = (i == j) ? 1.0 : 0.0;
    }
    a[i] = v;
  }
}

// In-register upper Cholesky G = Z^T Z: on return a[i] = Z[i][j] for i <= j (lane j).
// Returns false (uniformly) when a pivot of the leading s x s block is not finite or not above
// 64 eps max_{j<s} G_jj.
template <int KP>
__device__ __forceinline__ bool warp_cholesky(double (&a)[KP], int s, int j) {
  double dj = (j < s) ? a[j] : 0.0;
#pragma unroll
  for (int off = 16; off; off >>= 1) dj = fmax(dj, __shfl_xor_sync(kFull, dj, off));
  const double thresh = 64.0 * DBL_EPSILON * dj;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const double piv = __shfl_sync(kFull, a[k], k);
    if (k < s && (!isfinite(piv) || !(piv > thresh))) ok = false;
    const double zkk = sqrt(piv);
    const double rz = 1.0 / zkk;
    const double zkj = (j == k) ? zkk : a[k] * rz;  // Z[k][j] for j >= k
    if (j >= k) a[k] = zkj;
#pragma unroll
    for (int i = k + 1; i < KP; ++i) {
      const double zki = __shfl_sync(kFull, zkj, i);
      if (i <= j && j > k) a[i] = fma(-zki, zkj, a[i]);
    }
  }
  return ok;
}

// Zs[i*KP + l] = Z[i][l] (upper, zeros below) from the lanes' columns.
template <int KP>
__device__ __forceinline__ void store_columns(const double (&a)[KP], int j, double* Zs) {
  if (j >= KP) return;
#pragma unroll
  for (int i = 0; i < KP; ++i) Zs[i * KP + j] = (i <= j) ? a[i] : 0.0;
}

// Column j of Z^{-1} (upper triangular) by back substitution in column order:
// for l = KP-1..0: x_l = b_l / Z_ll; b_i -= Z_il x_l (i < l).  b = e_j.
// The column is written to Zt[j*KP + l] (lanes j < KP).
template <int KP>
__device__ __forceinline__ void upper_inverse_column(const double* Zs, const double* rdiag, int j, double* Zt) {
  double b[KP];
#pragma unroll
  for (int i = 0; i < KP; ++i) b[i] = (i == j) ? 1.0 : 0.0;
#pragma unroll
  for (int l = KP - 1; l >= 0; --l) {
    const double xl = b[l] * rdiag[l];
    if (j < KP) Zt[j * KP + l] = xl;
#pragma unroll
    for (int i = 0; i < l; ++i) b[i] = fma(-Zs[i * KP + l], xl, b[i]);
  }
}

// out (column-major, ld KP) column j from the transposed shared copy Zt[j*KP + i], zero padded.
template <int KP>
__device__ __forceinline__ void write_col_from_t(double* __restrict__ out, const double* Zt, int j, int s) {
  if (j >= KP) return;
#pragma unroll
  for (int i = 0; i < KP; ++i) out[i + j * KP] = (i < s && j < s) ? Zt[j * KP + i] : 0.0;
}

// out column j from the row-major shared copy Zs[i*KP + j], zero padded.
template <int KP>
__device__ __forceinline__ void write_col_from_s(double* __restrict__ out, const double* Zs, int j, int s) {
  if (j >= KP) return;
#pragma unroll
  for (int i = 0; i < KP; ++i) out[i + j * KP] = (i < s && j < s) ? Zs[i * KP + j] : 0.0;
}

}  // namespace

// W^0, Sigma^0 = qr(R^0): Sigma = chol(R^T R), SigmaInv = Sigma^{-1}.
template <int KP>
__global__ void __launch_bounds__(32)
k_small_sigma_w(SolveState* st, const double* __restrict__ Gp, double* __restrict__ Sigma,
                double* __restrict__ SigmaInv) {
  __shared__ double Zs[KP * KP], Zt[KP * KP], rd[KP];
  const int j = threadIdx.x, s = st->s;
  bool ok;
  {
    double a[KP];
    load_packed_column<KP>(Gp, s, j, a);
    ok = warp_cholesky<KP>(a, s, j);
    store_columns<KP>(a, j, Zs);
    if (j < KP) rd[j] = 1.0 / a[j < KP ? j : 0];
  }
  __syncwarp();
  if (!ok) {
    if (j == 0) {
      st->done = 1;
      st->pw_skip = 1;
      st->status = 6;
    }
    if (j < KP)
      for (int i = 0; i < KP; ++i) Sigma[i + j * KP] = SigmaInv[i + j * KP] = 0.0;
    return;
  }
  upper_inverse_column<KP>(Zs, rd, j, Zt);
  __syncwarp();
  write_col_from_s<KP>(Sigma, Zs, j, s);
  write_col_from_t<KP>(SigmaInv, Zt, j, s);
  if (j == 0 && st->maxit <= 0) {
    st->done = 1;
    st->pw_skip = 1;
  }
}

// Xi = (P^T A P)^{-1} = Z^{-1} Z^{-T} from the Cholesky factor of P^T A P (Section 3); T = Xi Sigma.
template <int KP>
__global__ void __launch_bounds__(32)
k_small_xi_w(SolveState* st, const double* __restrict__ G1p, const double* __restrict__ Sigma,
             double* __restrict__ Xi, double* __restrict__ T) {
  if (st->done) return;
  __shared__ double Zs[KP * KP], Zt[KP * KP], Xs[KP * KP], rd[KP];
  const int j = threadIdx.x, s = st->s;
  bool ok;
  {
    double a[KP];
    load_packed_column<KP>(G1p, s, j, a);
    ok = warp_cholesky<KP>(a, s, j);
    store_columns<KP>(a, j, Zs);
    if (j < KP) rd[j] = 1.0 / a[j < KP ? j : 0];
  }
  if (!ok) {
    if (j == 0) {
      st->done = 1;
      st->pw_skip = 1;
      st->status = 6;
    }
    return;
  }
  __syncwarp();
  upper_inverse_column<KP>(Zs, rd, j, Zt);  // Zt[b*KP + a] = Zinv[a][b]
  __syncwarp();
  // Xi[i][j] = sum_{l >= max(i, j)} Zinv[i][l] Zinv[j][l]
  if (j < KP) {
#pragma unroll 4
    for (int i = 0; i < KP; ++i) {
      double v = 0.0;
      for (int l = (i > j ? i : j); l < KP; ++l) v = fma(Zt[l * KP + i], Zt[l * KP + j], v);
      v = (i < s && j < s) ? v : 0.0;
      Xs[i * KP + j] = v;
      Xi[i + j * KP] = v;
    }
  }
  __syncwarp();
  // T[i][j] = sum_{l <= j} Xi[i][l] Sigma[l][j]
  if (j < KP) {
    double sg[KP];
#pragma unroll
    for (int l = 0; l < KP; ++l) sg[l] = Sigma[l + j * KP];
#pragma unroll 4
    for (int i = 0; i < KP; ++i) {
      double v = 0.0;
#pragma unroll
      for (int l = 0; l < KP; ++l)
        if (l <= j) v = fma(Xs[i * KP + l], sg[l], v);
      T[i + j * KP] = (i < s && j < s) ? v : 0.0;
    }
  }
  if (j == 0) st->it += 1;
}

// Best-basis test, zeta = chol(V^T V), zeta^{-1}, Sigma = zeta Sigma; sets the WHILE condition.
template <int KP>
__global__ void __launch_bounds__(32)
k_small_zeta_w(SolveState* st, const double* __restrict__ G2nu, double* __restrict__ Sigma,
               double* __restrict__ Zeta, double* __restrict__ ZetaInv, cudaGraphConditionalHandle cond,
               int use_cond) {
  __shared__ double Zs[KP * KP], Zt[KP * KP], rd[KP];
  const int j = threadIdx.x, s = st->s;
  if (st->done) {
    if (j == 0 && use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  // h = argmin_j nu_j, lowest index on ties (butterfly on (value, index): every lane gets the same)
  double nv = (j < s) ? G2nu[npack(KP) + j] : __longlong_as_double(0x7ff0000000000000ll);
  int h = j;
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const double ov = __shfl_xor_sync(kFull, nv, off);
    const int oh = __shfl_xor_sync(kFull, h, off);
    if (ov < nv || (ov == nv && oh < h)) {
      nv = ov;
      h = oh;
    }
  }
  const double nh = sqrt(nv);
  if (!st->no_test && nh < st->tol_abs) {
    if (j == 0) {
      st->best_col = h;
      st->nu_h = nh;
      st->converged = 1;
      st->done = 1;
      st->pw_skip = 1;
      st->status = 0;
      if (use_cond) cudaGraphSetConditional(cond, 0);
    }
    return;
  }
  bool ok;
  {
    double a[KP];
    load_packed_column<KP>(G2nu, s, j, a);
    ok = warp_cholesky<KP>(a, s, j);
    store_columns<KP>(a, j, Zs);
    if (j < KP) rd[j] = 1.0 / a[j < KP ? j : 0];
  }
  if (!ok) {
    if (j == 0) {
      st->best_col = h;
      st->nu_h = nh;
      st->done = 1;
      st->pw_skip = 1;
      st->status = 6;
      if (use_cond) cudaGraphSetConditional(cond, 0);
    }
    return;
  }
  __syncwarp();
  upper_inverse_column<KP>(Zs, rd, j, Zt);
  // Sigma[i][j] <- sum_{l=i..j} zeta[i][l] Sigma[l][j]  (lane j owns column j)
  if (j < KP) {
    double sg[KP];
#pragma unroll
    for (int l = 0; l < KP; ++l) sg[l] = Sigma[l + j * KP];
#pragma unroll 4
    for (int i = 0; i < KP; ++i) {
      double v = 0.0;
#pragma unroll
      for (int l = 0; l < KP; ++l)
        if (l >= i && l <= j) v = fma(Zs[i * KP + l], sg[l], v);
      Sigma[i + j * KP] = (i < s && j < s) ? v : 0.0;
    }
  }
  __syncwarp();
  write_col_from_s<KP>(Zeta, Zs, j, s);
  write_col_from_t<KP>(ZetaInv, Zt, j, s);
  if (j == 0) {
    st->best_col = h;
    st->nu_h = nh;
    int done = 0;
    if (st->it >= st->maxit) {
      done = 1;
      st->done = 1;
      st->pw_skip = 0;  // the last iteration still completes its W, P update
      st->status = st->no_test ? 0 : 5;
    }
    if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
  }
}

// ------------------------------------------------------------------------------------------------
// KP >= 16: one CTA of 256 threads. At s = 32 each of these steps is ~20-60 thousand FP64 FMAs, so
// the work is spread over all 8 warps of the SM; the sequential depth is kept short: a right-looking
// Cholesky with one barrier per column, and a blocked triangular inverse of logarithmic depth
// (inverse of [[Z11, Z12], [0, Z22]] has off-diagonal block -Z11^{-1} Z12 Z22^{-1}).

namespace {

constexpr int kCtaSmall = 256;

template <int KP>
struct SmallLd {
  static constexpr int LD = KP + 1;  // padded row stride of the shared k x k matrices
};

// (l, m) with 0 <= l <= m from the packed upper index q = m (m+1) / 2 + l.
__device__ __forceinline__ void unpack_upper(int q, int& l, int& m) {
  m = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
  while ((m + 1) * (m + 2) / 2 <= q) ++m;
  while (m * (m + 1) / 2 > q) --m;
  l = q - m * (m + 1) / 2;
}

// A (row-major, ld KP+1) holds the symmetric matrix with the identity outside s x s; on return Z
// holds its upper Cholesky factor (zeros below). Returns false when a pivot of the leading s x s
// block is not finite or not above 64 eps max_{j<s} G_jj. All threads must call it.
// FP64 instructions are scarce on this part (a full-warp FP64 instruction holds the SM's FP64
// unit for ~16 cycles), so each pivot's square root and reciprocal is computed once, by the thread
// that finishes updating that pivot one step earlier (look-ahead), and read by all from shared
// memory: one barrier per column.
template <int KP>
__device__ bool cta_chol(double* A, double* Z, int s) {
  constexpr int LD = SmallLd<KP>::LD;
  __shared__ double maxd, zd[KP], rzd[KP], ipd[KP];  // sqrt(pivot), 1/sqrt(pivot), 1/pivot
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (int q = tid; q < KP * LD; q += kCtaSmall) Z[q] = 0.0;
  if (tid == 0) {
    double m = 0.0;
    for (int j = 0; j < s; ++j) m = fmax(m, A[j * LD + j]);
    maxd = m;
    const double piv = A[0];
    bad = (s > 0 && (!isfinite(piv) || !(piv > 64.0 * DBL_EPSILON * m))) ? 1 : 0;
    const double r = rsqrt(piv);
    zd[0] = piv * r;
    rzd[0] = r;
    ipd[0] = r * r;
  }
  __syncthreads();
  for (int k = 0; k < KP; ++k) {
    const double zkk = zd[k], rz = rzd[k], ip = ipd[k];
    const int t = KP - k, cnt = t * (t + 1) / 2;
    for (int q = tid; q < cnt; q += kCtaSmall) {
      int l, m;
      unpack_upper(q, l, m);
      l += k;
      m += k;
      if (l == k) {
        Z[k * LD + m] = (m == k) ? zkk : A[k * LD + m] * rz;
      } else {  // A[l][m] -= Z[k][l] Z[k][m] = A[k][l] A[k][m] / pivot
        const double v = fma(-A[k * LD + l], A[k * LD + m] * ip, A[l * LD + m]);
        A[l * LD + m] = v;
        if (l == k + 1 && m == k + 1) {  // the next pivot is final now
          if (k + 1 < s && (!isfinite(v) || !(v > 64.0 * DBL_EPSILON * maxd))) bad = 1;
          const double r = rsqrt(v);
          zd[k + 1] = v * r;
          rzd[k + 1] = r;
          ipd[k + 1] = r * r;
        }
      }
    }
    __syncthreads();
  }
  return bad == 0;
}

// Zi = Z^{-1} for the upper triangular Z (ld KP+1), by doubling the size of inverted diagonal
// blocks: Zi12 = -Zi11 (Z12 Zi22). Tmp is scratch of the same shape.
template <int KP>
__device__ void cta_tri_inv(const double* Z, double* Zi, double* Tmp) {
  constexpr int LD = SmallLd<KP>::LD;
  const int tid = threadIdx.x;
  for (int q = tid; q < KP * KP; q += kCtaSmall) {
    const int i = q / KP, j = q % KP;
    Zi[i * LD + j] = (i == j) ? 1.0 / Z[i * LD + i] : 0.0;
  }
  __syncthreads();
  for (int b = 1; b < KP; b *= 2) {
    const int pairs = KP / (2 * b), work = pairs * b * b;
    for (int q = tid; q < work; q += kCtaSmall) {  // M = Z12 Zi22  (Zi22 upper: x <= c)
      const int pr = q / (b * b), r = (q / b) % b, c = q % b, p = pr * 2 * b;
      double v = 0.0;
      for (int x = 0; x <= c; ++x) v = fma(Z[(p + r) * LD + p + b + x], Zi[(p + b + x) * LD + p + b + c], v);
      Tmp[(p + r) * LD + p + b + c] = v;
    }
    __syncthreads();
    for (int q = tid; q < work; q += kCtaSmall) {  // Zi12 = -Zi11 M  (Zi11 upper: x >= r)
      const int pr = q / (b * b), r = (q / b) % b, c = q % b, p = pr * 2 * b;
      double v = 0.0;
      for (int x = r; x < b; ++x) v = fma(Zi[(p + r) * LD + p + x], Tmp[(p + x) * LD + p + b + c], v);
      Zi[(p + r) * LD + p + b + c] = -v;
    }
    __syncthreads();
  }
}

template <int KP>
__device__ void cta_load_packed(const double* __restrict__ packed, int s, double* A) {
  constexpr int LD = SmallLd<KP>::LD;
  for (int q = threadIdx.x; q < KP * KP; q += kCtaSmall) {
    const int i = q / KP, j = q % KP;
    double v;
    if (i < s && j < s) v = (i <= j) ? packed[pidx(i, j)] : packed[pidx(j, i)];
    else v = (i == j) ? 1.0 : 0.0;
    A[i * LD + j] = v;
  }
  __syncthreads();
}

template <int KP>
__device__ void cta_store(double* __restrict__ out, const double* M, int s) {
  constexpr int LD = SmallLd<KP>::LD;
  for (int q = threadIdx.x; q < KP * KP; q += kCtaSmall) {
    const int i = q % KP, j = q / KP;  // column-major out
    out[q] = (i < s && j < s) ? M[i * LD + j] : 0.0;
  }
}

}  // namespace

template <int KP>
__global__ void __launch_bounds__(kCtaSmall)
k_small_sigma_c(SolveState* st, const double* __restrict__ Gp, double* __restrict__ Sigma,
                double* __restrict__ SigmaInv) {
  constexpr int LD = SmallLd<KP>::LD;
  __shared__ double A[KP * LD], Z[KP * LD], Zi[KP * LD], Tmp[KP * LD];
  const int s = st->s;
  cta_load_packed<KP>(Gp, s, A);
  if (!cta_chol<KP>(A, Z, s)) {
    if (threadIdx.x == 0) {
      st->done = 1;
      st->pw_skip = 1;
      st->status = 6;
    }
    for (int q = threadIdx.x; q < KP * KP; q += kCtaSmall) Sigma[q] = SigmaInv[q] = 0.0;
    return;
  }
  cta_tri_inv<KP>(Z, Zi, Tmp);
  cta_store<KP>(Sigma, Z, s);
  cta_store<KP>(SigmaInv, Zi, s);
  if (threadIdx.x == 0 && st->maxit <= 0) {
    st->done = 1;
    st->pw_skip = 1;
  }
}

template <int KP>
__global__ void __launch_bounds__(kCtaSmall)
k_small_xi_c(SolveState* st, const double* __restrict__ G1p, const double* __restrict__ Sigma,
             double* __restrict__ Xi, double* __restrict__ T) {
  constexpr int LD = SmallLd<KP>::LD;
  if (st->done) return;
  __shared__ double A[KP * LD], Z[KP * LD], Zi[KP * LD], Tmp[KP * LD];
  const int s = st->s, tid = threadIdx.x;
  cta_load_packed<KP>(G1p, s, A);
  if (!cta_chol<KP>(A, Z, s)) {
    if (tid == 0) {
      st->done = 1;
      st->pw_skip = 1;
      st->status = 6;
    }
    return;
  }
  cta_tri_inv<KP>(Z, Zi, Tmp);
  // Xi = Zi Zi^T (into A; upper half computed, mirrored), Sigma (into Tmp)
  for (int q = tid; q < KP * (KP + 1) / 2; q += kCtaSmall) {
    int a, b;
    unpack_upper(q, a, b);  // a <= b
    double v = 0.0;
    for (int l = b; l < KP; ++l) v = fma(Zi[a * LD + l], Zi[b * LD + l], v);
    v = (b < s) ? v : 0.0;
    A[a * LD + b] = v;
    A[b * LD + a] = v;
  }
  for (int q = tid; q < KP * KP; q += kCtaSmall) {
    const int a = q / KP, b = q % KP;
    Tmp[a * LD + b] = Sigma[a + b * KP];
  }
  __syncthreads();
  cta_store<KP>(Xi, A, s);
  {  // T = Xi Sigma (Sigma upper: l <= b); each thread interleaves its R outputs
    constexpr int R = KP * KP / kCtaSmall > 0 ? KP * KP / kCtaSmall : 1;
    const int a = tid % KP;
    int b[R];
    double v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      b[r] = (tid + r * kCtaSmall) / KP;
      v[r] = 0.0;
    }
    if (tid + (R - 1) * kCtaSmall < KP * KP) {
      for (int l = 0; l <= b[R - 1]; ++l) {
        const double xa = A[a * LD + l];
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (l <= b[r]) v[r] = fma(xa, Tmp[l * LD + b[r]], v[r]);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) T[a + b[r] * KP] = (a < s && b[r] < s) ? v[r] : 0.0;
    }
  }
  if (tid == 0) st->it += 1;
}

template <int KP>
__global__ void __launch_bounds__(kCtaSmall)
k_small_zeta_c(SolveState* st, const double* __restrict__ G2nu, double* __restrict__ Sigma,
               double* __restrict__ Zeta, double* __restrict__ ZetaInv, cudaGraphConditionalHandle cond,
               int use_cond) {
  constexpr int LD = SmallLd<KP>::LD;
  __shared__ double A[KP * LD], Z[KP * LD], Zi[KP * LD], Tmp[KP * LD];
  __shared__ int stop;
  const int s = st->s, tid = threadIdx.x;
  if (st->done) {
    if (tid == 0 && use_cond) cudaGraphSetConditional(cond, 0);
    return;
  }
  if (tid < 32) {  // h = argmin_j nu_j, lowest index on ties
    const int j = tid;
    double nv = (j < s) ? G2nu[npack(KP) + j] : __longlong_as_double(0x7ff0000000000000ll);
    int h = j;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const double ov = __shfl_xor_sync(kFull, nv, off);
      const int oh = __shfl_xor_sync(kFull, h, off);
      if (ov < nv || (ov == nv && oh < h)) {
        nv = ov;
        h = oh;
      }
    }
    if (tid == 0) {
      const double nh = sqrt(nv);
      st->best_col = h;
      st->nu_h = nh;
      stop = 0;
      if (!st->no_test && nh < st->tol_abs) {
        st->converged = 1;
        st->done = 1;
        st->pw_skip = 1;
        st->status = 0;
        stop = 1;
        if (use_cond) cudaGraphSetConditional(cond, 0);
      }
    }
  }
  __syncthreads();
  if (stop) return;
  cta_load_packed<KP>(G2nu, s, A);
  if (!cta_chol<KP>(A, Z, s)) {
    if (tid == 0) {
      st->done = 1;
      st->pw_skip = 1;
      st->status = 6;
      if (use_cond) cudaGraphSetConditional(cond, 0);
    }
    return;
  }
  cta_tri_inv<KP>(Z, Zi, Tmp);
  for (int q = tid; q < KP * KP; q += kCtaSmall) {
    const int a = q / KP, b = q % KP;
    Tmp[a * LD + b] = Sigma[a + b * KP];
  }
  __syncthreads();
  {  // Sigma = zeta Sigma (both upper: a <= l <= b); R interleaved outputs per thread
    constexpr int R = KP * KP / kCtaSmall > 0 ? KP * KP / kCtaSmall : 1;
    const int a = tid % KP;
    int b[R];
    double v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      b[r] = (tid + r * kCtaSmall) / KP;
      v[r] = 0.0;
    }
    if (tid + (R - 1) * kCtaSmall < KP * KP) {
      for (int l = a; l <= b[R - 1]; ++l) {
        const double za = Z[a * LD + l];
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (l <= b[r]) v[r] = fma(za, Tmp[l * LD + b[r]], v[r]);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) Sigma[a + b[r] * KP] = (a < s && b[r] < s) ? v[r] : 0.0;
    }
  }
  cta_store<KP>(Zeta, Z, s);
  cta_store<KP>(ZetaInv, Zi, s);
  if (tid == 0) {
    int done = 0;
    if (st->it >= st->maxit) {
      done = 1;
      st->done = 1;
      st->pw_skip = 0;  // the last iteration still completes its W, P update
      st->status = st->no_test ? 0 : 5;
    }
    if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
  }
}

// ------------------------------------------------------------------------------------ launchers

// KP <= 8: one warp; KP >= 16: one CTA of 256 threads.
#define MBPCG_SMALL_SWITCH(kp, WARP, CTA) \
  switch (kp) {                           \
    case 1: WARP(1); break;               \
    case 2: WARP(2); break;               \
    case 4: WARP(4); break;               \
    case 8: WARP(8); break;               \
    case 16: CTA(16); break;              \
    default: CTA(32); break;              \
  }

void launch_small_sigma(cudaStream_t s, int kp, SolveState* st, const double* Gp, double* Sigma, double* SigmaInv) {
#define WARP(K) k_small_sigma_w<K><<<1, 32, 0, s>>>(st, Gp, Sigma, SigmaInv)
#define CTA(K) k_small_sigma_c<K><<<1, kCtaSmall, 0, s>>>(st, Gp, Sigma, SigmaInv)
  MBPCG_SMALL_SWITCH(kp, WARP, CTA)
#undef WARP
#undef CTA
}
void launch_small_xi(cudaStream_t s, int kp, SolveState* st, const double* G1p, const double* Sigma, double* Xi,
                     double* T) {
#define WARP(K) k_small_xi_w<K><<<1, 32, 0, s>>>(st, G1p, Sigma, Xi, T)
#define CTA(K) k_small_xi_c<K><<<1, kCtaSmall, 0, s>>>(st, G1p, Sigma, Xi, T)
  MBPCG_SMALL_SWITCH(kp, WARP, CTA)
#undef WARP
#undef CTA
}
void launch_small_zeta(cudaStream_t s, int kp, SolveState* st, const double* G2nu, double* Sigma, double* Zeta,
                       double* ZetaInv, cudaGraphConditionalHandle cond, int use_cond) {
#define WARP(K) k_small_zeta_w<K><<<1, 32, 0, s>>>(st, G2nu, Sigma, Zeta, ZetaInv, cond, use_cond)
#define CTA(K) k_small_zeta_c<K><<<1, kCtaSmall, 0, s>>>(st, G2nu, Sigma, Zeta, ZetaInv, cond, use_cond)
  MBPCG_SMALL_SWITCH(kp, WARP, CTA)
#undef WARP
#undef CTA
}

}  // namespace mbpcg
