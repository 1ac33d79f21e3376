// The k x k steps of Algorithm 1: the set-up Cholesky QR factor (one warp for KP <= 8, lane j
// owning column j, or one CTA) and the two steps of every iteration (a thread-block cluster, see
// below). On GB300 these are bound by FP64 latency, not throughput, so the algorithms are chosen
// for short dependency chains.
//
// Padding: rows/columns s..KP-1 are factored as the identity and written back as zeros, so the row
// kernels keep the padded columns of every block at exactly zero.
#include <cfloat>

#include <cooperative_groups.h>

#include "kernels.h"

namespace mbpcg {
namespace {

constexpr unsigned kFull = 0xffffffffu;
namespace cg = cooperative_groups;

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
template <int KP, int NT = kCtaSmall>
__device__ bool cta_chol(double* A, double* Z, int s, const double** rz_out = nullptr) {
  constexpr int LD = SmallLd<KP>::LD;
  __shared__ double maxd, zd[KP], rzd[KP], ipd[KP];  // sqrt(pivot), 1/sqrt(pivot), 1/pivot
  if (rz_out != nullptr) *rz_out = rzd;
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (int q = tid; q < KP * LD; q += NT) Z[q] = 0.0;
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
    for (int q = tid; q < cnt; q += NT) {
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

template <int KP, int NT = kCtaSmall>
__device__ void cta_load_packed(const double* __restrict__ packed, int s, double* A) {
  constexpr int LD = SmallLd<KP>::LD;
  for (int q = threadIdx.x; q < KP * KP; q += NT) {
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

// ------------------------------------------------------------------------------------------------
// KP >= 16 inside the loop: a cluster of CS CTAs of 128 threads.
//
// Cost model of this part: an FP64 instruction holds its SM sub-partition's FP64 unit for 64 cycles
// whatever the number of active lanes, and its result is ready 64 cycles later (four independent
// chains in one warp take four times as long as one). So the factorisation is organised around its
// serial chain of pivots, and every other FP64 operation is packed into full warps and spread over
// the sub-partitions and the CTAs of the cluster.
//
// Factorisation (every CTA of the cluster, redundantly): symmetric Gaussian elimination
// G = L D L^T. Warp 0 (the pivot warp) carries the chain: pivot d_k -> 1/d_k -> row k+1 updated by
// step k -> d_{k+1}; warps 1-3 and, at KP = 32, 5-7 (two per sub-partition, so that one hides the
// other's latencies; warp 4 stays idle to leave the pivot warp's sub-partition to it) apply step k
// to the rest of the trailing matrix while the pivot warp already works on step k+1 (two named
// barriers per step hand rows over). Nothing else is on that chain: afterwards each CTA forms only
// the columns or rows of L^{-1} it needs, by triangular solves with one KP-lane shuffle segment per
// column. Z = D^{1/2} L^T, Z^{-1} = L^{-T} D^{-1/2}, Xi = G^{-1} = L^{-T} D^{-1} L^{-1}.
//
// After it, each CTA owns CPC = 128 / KP columns b = c + CS r (r < CPC; c = rank in the cluster) of
// every result; columns computed elsewhere are read from the owner's shared memory (distributed
// shared memory) after a cluster barrier.

template <int KP>
struct ClusterCfg {
  static constexpr int NT = 128;       // threads of the column phases (thread = (column r, row a))
  static constexpr int NF = KP >= 32 ? 256 : 128;  // threads of the CTA (all take part in the factorisation)
  static constexpr int NB = NF > 128 ? NF - 64 : NF - 32;  // bulk threads (warp 0 and, if present, 4 excluded)
  static constexpr int IDLE = NF > 128 ? 4 : 3;             // warp free before the factorisation's bulk work
  static constexpr int CPC = NT / KP;  // columns per CTA: 4 (KP = 32), 8 (KP = 16)
  static constexpr int CS = KP / CPC;  // CTAs per cluster: 8, 2
};

// 1/d for a positive normal d below 2^1000, within about an ulp: the hardware approximation
// (rcp.approx.f32) of d's leading 23 significand bits, rescaled by d's exponent with integer
// operations, then one third-order Newton step y = y0 (1 + e + e^2), e = 1 - d y0 (the truncated
// series of 1 / (1 - e)); the seed's relative error is below 2^-22, so e^3 is below 2^-66.
__device__ __forceinline__ double rcp_pos(double d) {
  const long long bits = __double_as_longlong(d);
  const int e = (int)(bits >> 52) & 0x7FF;
  const float f = __int_as_float(0x3F800000 | (int)((bits >> 29) & 0x7FFFFF));  // in [1, 2)
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));  // in (0.5, 1]
  const int rb = __float_as_int(r);
  const long long ex = (long long)(((rb >> 23) & 0xFF) - 127 + 2046 - e);
  const double y0 = __longlong_as_double((ex << 52) | ((long long)(rb & 0x7FFFFF) << 29));
  const double eps = fma(-d, y0, 1.0);
  const double e2 = fma(eps, eps, eps);
  return fma(y0, e2, y0);
}

// 1/sqrt(d) for a positive normal d, within about an ulp: rsqrt.approx.f32 of the leading
// significand bits with the exponent's parity folded in (argument in [1, 4)), then one third-order
// Newton step y = y0 (1 + e/2 + 3 e^2/8), e = 1 - d y0^2 (the series of (1 - e)^{-1/2}).
__device__ __forceinline__ double rsqrt_pos(double d) {
  const long long bits = __double_as_longlong(d);
  const int E = ((int)(bits >> 52) & 0x7FF) - 1023;
  const int odd = E & 1;
  const float f = __int_as_float(((127 + odd) << 23) | (int)((bits >> 29) & 0x7FFFFF));  // in [1, 4)
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));  // in (0.5, 1]
  const int rb = __float_as_int(r);
  const int half = (E - odd) / 2;
  const long long ex = (long long)(((rb >> 23) & 0xFF) - 127 - half + 1023);
  const double y0 = __longlong_as_double((ex << 52) | ((long long)(rb & 0x7FFFFF) << 29));
  const double t = d * y0;
  const double eps = fma(-t, y0, 1.0);
  const double q = eps * fma(eps, 0.375, 0.5);
  return fma(y0, q, y0);
}

__device__ __forceinline__ void named_bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// A cluster barrier split in two: every thread of every CTA arrives once, then waits once; work
// between the two overlaps the barrier's latency.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Shared working set of the factorisation (matrices row-major with ld KP+1).
template <int KP>
struct LdlWork {
  static constexpr int LD = KP + 1;
  static constexpr int OU = KP * LD, OL = 2 * KP * LD, OR = 3 * KP * LD;  // offsets of U, Lt, R from S
  double S[KP * LD];   // in: G (identity outside s x s); then the trailing matrices; later reused
  double U[KP * LD];   // row k of D L^T: U[k][m] = d_k L[m][k] (m >= k)
  double Lt[KP * LD];  // Lt[k][m] = L[m][k] (m > k)
  double R[KP * LD];   // L^{-1}, unit lower triangular (the Xi step fills it column by column)
  double d[KP], inv[KP];
  unsigned short tri[KP * (KP + 1) / 2];  // packed index q = m (m+1)/2 + l (l <= m) -> l | m << 8
  int bad;
};

// The entries of the packed Gram that this thread's share of ldl_init uses. The buffer holds the
// triangle of the handle's padded width KL (<= KP; s <= KL), whatever s is, so the loads need no
// solve state: issued before the state is read, their L2 round trip overlaps its own. Entries past
// KL are not read (zero here; ldl_init replaces them by the identity).
template <int KP, int KL>
__device__ __forceinline__ void ldl_load(const double* __restrict__ packed, double (&g)[KP * KP / ClusterCfg<KP>::NF]) {
  constexpr int NT = ClusterCfg<KP>::NF, NI = KP * KP / NT;
#pragma unroll
  for (int i = 0; i < NI; ++i) {  // all loads in flight at once
    const int q = threadIdx.x + NT * i, r = q / KP, c = q % KP;
    g[i] = (r < KL && c < KL) ? ((r <= c) ? packed[pidx(r, c)] : packed[pidx(c, r)]) : 0.0;
  }
}

template <int KP>
__device__ void ldl_init(LdlWork<KP>& W, const double (&g)[KP * KP / ClusterCfg<KP>::NF], int s) {
  constexpr int LD = LdlWork<KP>::LD, NT = ClusterCfg<KP>::NF, NI = KP * KP / NT;
  double v[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int q = threadIdx.x + NT * i, r = q / KP, c = q % KP;
    v[i] = (r < s && c < s) ? g[i] : (r == c ? 1.0 : 0.0);
  }
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int q = threadIdx.x + NT * i, r = q / KP, c = q % KP;
    W.S[r * LD + c] = v[i];
    W.R[r * LD + c] = (r == c) ? 1.0 : 0.0;
    if (r >= s) W.U[r * LD + c] = (r == c) ? 1.0 : 0.0;
  }
  for (int m = 0, q0 = 0; m < KP; q0 += ++m)
    for (int l = threadIdx.x; l <= m; l += NT) W.tri[q0 + l] = (unsigned short)(l | (m << 8));
  if (threadIdx.x < KP && threadIdx.x >= s) W.d[threadIdx.x] = W.inv[threadIdx.x] = 1.0;
  __syncthreads();
}

// G = L D L^T (see above). Sets W.bad when a pivot of the leading s x s block is not a
// finite number above 64 eps max_j G_jj (or not below 2^1000). All NF threads call it; it ends with
// a block-wide barrier.
template <int KP>
__device__ void ldl_factor(LdlWork<KP>& W, int s) {
  using LW = LdlWork<KP>;
  constexpr int LD = LW::LD, NB = ClusterCfg<KP>::NB, NBAR = 32 + NB;  // threads on the named barriers
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {  // pivot warp; lane j holds column j of the current pivot row
    const int j = tid;
    long long mb = (j < s) ? __double_as_longlong(W.S[j * LD + j]) : 0;  // bit order = value order for x >= 0
#pragma unroll
    for (int off = 16; off; off >>= 1) mb = max(mb, __shfl_xor_sync(kFull, mb, off));
    const long long thr_b = __double_as_longlong(64.0 * DBL_EPSILON * __longlong_as_double(mb));
    double row = (j < KP) ? W.S[j] : 0.0;
    bool bad = false;
    for (int k = 0; k < s; ++k) {
      const double dk = __shfl_sync(kFull, row, k);
      const double a = __shfl_sync(kFull, row, (k + 1 < KP) ? k + 1 : k);
      const long long db = __double_as_longlong(dk);
      bad |= !(db > thr_b && db < 0x7E70000000000000LL);  // thr < d_k < 2^1000 (NaN fails)
      const double inv = rcp_pos(dk);
      const double w = row * inv;
      if (j >= k && j < KP) W.U[k * LD + j] = row;
      if (j > k && j < KP) W.Lt[k * LD + j] = w;
      if (j == 0) {
        W.d[k] = dk;
        W.inv[k] = inv;
      }
      // The bulk warps must have finished step k-1 before step k is published: otherwise their
      // step-k arrivals on barrier 2 could complete the phase meant for step k-1 without this warp.
      if (k >= 1) named_bar_sync(2, NBAR);  // the bulk warps finished step k-1
      named_bar_arrive(1, NBAR);            // step k published
      if (k + 1 < s) {
        const double nxt = (j < KP) ? W.S[(k + 1) * LD + j] : 0.0;  // row k+1 after step k-1
        row = fma(-a, w, nxt);
      }
    }
    named_bar_sync(2, NBAR);
    if (j == 0) W.bad = bad ? 1 : 0;
  } else if (warp != 4) {  // bulk: step k on rows k+2.. of the trailing matrix
    static_assert(ClusterCfg<KP>::NF == 128 || ClusterCfg<KP>::NF == 256, "bulk thread numbering");
    const int bt = tid - (warp < 4 ? 32 : 64);
    double* base = W.S;
    for (int k = 0; k < s; ++k) {
      named_bar_sync(1, NBAR);
      const int t = s - k - 2, cnt = t > 0 ? t * (t + 1) / 2 : 0;
      for (int q = bt; q < cnt; q += NB) {  // S[l][m] -= S[k][l] S[k][m] / d_k
        const int pk = W.tri[q], l = k + 2 + (pk & 0xFF), m = k + 2 + (pk >> 8);
        base[l * LD + m] = fma(-base[LW::OU + k * LD + l], base[LW::OL + k * LD + m], base[l * LD + m]);
      }
      named_bar_arrive(2, NBAR);
    }
  }
  __syncthreads();
}

// Column b of L^{-1} (L unit lower triangular, L[l][k] = Lt[k][l]) by forward substitution
// L x = e_b; the thread holds row a of the column, a KP-lane shuffle segment holds the column, bmin
// is the smallest b of the calling warp (steps before it leave x exactly as it is).
template <int KP>
__device__ double ldl_inv_column(const LdlWork<KP>& W, int a, int b, int bmin, int s) {
  constexpr int LD = LdlWork<KP>::LD;
  double x = (a == b) ? 1.0 : 0.0;
  for (int k = bmin; k < s - 1; ++k) {
    const double xk = __shfl_sync(kFull, x, k, KP);
    if (a > k && a < s) x = fma(-W.Lt[k * LD + a], xk, x);
  }
  return x;
}

// Row b of L^{-1}, i.e. x with L^T x = e_b (x_a = 0 for a > b), by back substitution; bmax is the
// largest b of the calling warp.
template <int KP>
__device__ double ldl_inv_row(const LdlWork<KP>& W, int a, int b, int bmax) {
  constexpr int LD = LdlWork<KP>::LD;
  double x = (a == b) ? 1.0 : 0.0;
  for (int l = bmax; l >= 1; --l) {
    const double xl = __shfl_sync(kFull, x, l, KP);
    if (a < l && l <= b) x = fma(-W.Lt[a * LD + l], xl, x);  // x_l = 0 for l > b
  }
  return x;
}

// Copies the columns of M (ld KP+1) owned by the other CTAs of the cluster into this CTA's M
// (upper triangle a <= b only when upper is set).
template <int KP>
__device__ void cluster_gather_columns(double* M, int c, bool upper) {
  using CC = ClusterCfg<KP>;
  constexpr int LD = KP + 1;
  cg::cluster_group cluster = cg::this_cluster();
  for (int q = threadIdx.x; q < KP * KP; q += CC::NF) {
    const int a = q / KP, b = q % KP, owner = b % CC::CS;
    if (owner != c && (!upper || a <= b)) {
      const double* rm = cluster.map_shared_rank(M, owner);
      M[a * LD + b] = rm[a * LD + b];
    }
  }
}

// Xi = (P^T A P)^{-1} from the packed Gram G1p and T = Xi Sigma, both column-major KL x KL with zeros
// outside s x s; the step counter advances. KL (<= KP) is the padded width of the k x k matrices in
// global memory; a narrower system is computed inside KP x KP with the identity outside s x s.
template <int KP, int KL>
__global__ void __launch_bounds__(ClusterCfg<KP>::NF) __cluster_dims__(ClusterCfg<KP>::CS, 1, 1)
k_small_xi_x(SolveState* st, const double* __restrict__ G1p, const double* __restrict__ Sigma,
             double* __restrict__ Xi, double* __restrict__ T) {
  using CC = ClusterCfg<KP>;
  constexpr int LD = KP + 1;
  __shared__ LdlWork<KP> W;
  __shared__ double Sg[KP * CC::CPC], V[KP * CC::CPC];
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x, c = (int)cluster.block_rank();
  const bool ct = tid < CC::NT;  // column-phase thread: column b = c + CS r, row a
  const int r = tid / KP, a = tid % KP, b = c + CC::CS * r;
  // the Gram and Sigma first: a launch that returns discards them, the others overlap the round
  // trips of these loads and of the solve state
  double gv[KP * KP / CC::NF];
  ldl_load<KP, KL>(G1p, gv);
  const double sg = (ct && a < KL && b < KL) ? Sigma[a + b * KL] : 0.0;  // own columns (upper)
  if (st->done) return;
  const int s = st->s;
  if (ct) Sg[a * CC::CPC + r] = sg;
  ldl_init<KP>(W, gv, s);
  ldl_factor<KP>(W, s);
  if (W.bad) {  // every CTA reaches the same verdict
    if (c == 0 && tid == 0) {
      st->done = 1;
      st->pw_skip = 1;
      st->status = 6;
    }
    return;
  }
  // own columns of L^{-1}, then the others' through distributed shared memory
  if (ct) W.R[a * LD + b] = ldl_inv_column<KP>(W, a, b, c + CC::CS * ((32 * (tid >> 5)) / KP), s);
  cluster.sync();
  cluster_gather_columns<KP>(W.R, c, false);
  __syncthreads();
  // Xi[a][b] = sum_{j >= b} L^{-1}[j][a] (L^{-1}[j][b] / d_j) for a <= b, into W.S (upper part)
  double* X = W.S;
  if (ct) {
    V[a * CC::CPC + r] = W.inv[a] * W.R[a * LD + b];
    __syncwarp();
    double v = 0.0;
    for (int j = b; j < s; ++j) v = fma(W.R[j * LD + a], V[j * CC::CPC + r], v);
    if (a <= b) X[a * LD + b] = v;
  }
  cluster.sync();  // also: every CTA has finished reading the L^{-1} columns of the others
  cluster_gather_columns<KP>(X, c, true);
  __syncthreads();
  cluster_arrive();  // this CTA reads no other CTA's shared memory from here on
  if (ct) {
    const bool in = (a < s && b < s);
    double v = 0.0;  // T[a][b] = sum_{l <= b} Xi[a][l] Sigma[l][b]
    for (int l = 0; l <= b; ++l) v = fma(X[min(a, l) * LD + max(a, l)], Sg[l * CC::CPC + r], v);
    if (a < KL && b < KL) {
      Xi[a + b * KL] = in ? X[min(a, b) * LD + max(a, b)] : 0.0;
      T[a + b * KL] = in ? v : 0.0;
    }
  }
  cluster_wait();  // no CTA leaves while another may still read its shared memory
  if (c == 0 && tid == 0) st->it += 1;
}

// zeta from the packed Gram V^T V (Z = D^{1/2} L^T), zeta^{-1}, Sigma <- zeta Sigma, after the
// stopping test on nu (argmin over the columns, lowest index on ties); sets the loop's conditional.
// The factorisation starts before the stopping test is decided and is discarded if it stops.
// KL: padded width of the k x k matrices in global memory, as for k_small_xi_x.
template <int KP, int KL>
__global__ void __launch_bounds__(ClusterCfg<KP>::NF) __cluster_dims__(ClusterCfg<KP>::CS, 1, 1)
k_small_zeta_x(SolveState* st, const double* __restrict__ G2nu, double* __restrict__ Sigma,
               double* __restrict__ Zeta, double* __restrict__ ZetaInv, cudaGraphConditionalHandle cond,
               int use_cond) {
  using CC = ClusterCfg<KP>;
  constexpr int LD = KP + 1;
  __shared__ LdlWork<KP> W;
  __shared__ double Sg[KP * CC::CPC];
  __shared__ double nh_s;
  __shared__ int h_s, stop_s;
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x, c = (int)cluster.block_rank();
  const bool lead = (c == 0 && tid == 0);
  const bool ct = tid < CC::NT;
  const int r = tid / KP, a = tid % KP, b = c + CC::CS * r;
  // the Gram, Sigma and the norms first, as in k_small_xi_x
  double gv[KP * KP / CC::NF];
  ldl_load<KP, KL>(G2nu, gv);
  const double sg = (ct && a < KL && b < KL) ? Sigma[a + b * KL] : 0.0;
  const int jn = tid & 31;
  const long long nvb = ((tid >> 5) == CC::IDLE && jn < KL) ? __double_as_longlong(G2nu[npack(KL) + jn]) : 0;
  const int s = st->s;
  if (st->done) {  // the solve stopped in an earlier iteration: no W, P update in this one
    if (lead) {
      st->pw_skip = 1;
      if (use_cond) cudaGraphSetConditional(cond, 0);
    }
    return;
  }
  if (ct) Sg[a * CC::CPC + r] = sg;
  ldl_init<KP>(W, gv, s);
  if ((tid >> 5) == CC::IDLE) {  // a warp without early factorisation work decides the stopping test
    const int j = jn;  // h = argmin_j nu_j, lowest index on ties (nu >= 0: bit order = value order)
    long long nv = (j < s) ? nvb : 0x7FF0000000000000LL;
    int h = j;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const long long ov = __shfl_xor_sync(kFull, nv, off);
      const int oh = __shfl_xor_sync(kFull, h, off);
      if (ov < nv || (ov == nv && oh < h)) {
        nv = ov;
        h = oh;
      }
    }
    if (j == 0) {
      nh_s = sqrt(__longlong_as_double(nv));
      h_s = h;
      stop_s = (!st->no_test && nh_s < st->tol_abs) ? 1 : 0;
    }
  }
  ldl_factor<KP>(W, s);
  const double nh = nh_s;
  const int h = h_s;
  if (stop_s) {  // late CTAs may then find done set and return early: nothing of theirs is used
    if (lead) {
      st->best_col = h;
      st->nu_h = nh;
      st->converged = 1;
      st->done = 1;
      st->pw_skip = 1;
      st->status = 0;
      st->r_from_v = 1;
      if (use_cond) cudaGraphSetConditional(cond, 0);
    }
    return;
  }
  if (W.bad) {
    if (lead) {
      st->best_col = h;
      st->nu_h = nh;
      st->done = 1;
      st->pw_skip = 1;
      st->status = 6;
      st->r_from_v = 1;
      if (use_cond) cudaGraphSetConditional(cond, 0);
    }
    return;
  }
  cluster_arrive();  // this CTA has read all of the solve state it uses
  if (ct) {
    const double ra = rsqrt_pos(W.d[a]);              // d_a^{-1/2}
    const double rb = __shfl_sync(kFull, ra, b, KP);  // d_b^{-1/2} (lane b of this column's segment)
    double v = 0.0;  // (zeta Sigma)[a][b] = d_a^{-1/2} sum_{l = a..b} U[a][l] Sigma[l][b]
    for (int l = a; l <= b; ++l) v = fma(W.U[a * LD + l], Sg[l * CC::CPC + r], v);
    const bool in = (a < s && b < s), up = in && a <= b;
    const int bmax = c + CC::CS * ((32 * ((tid >> 5) + 1)) / KP - 1);
    const double lr = ldl_inv_row<KP>(W, a, b, bmax);  // L^{-1}[b][a]; every lane takes part in the shuffles
    if (a < KL && b < KL) {
      Sigma[a + b * KL] = in ? v * ra : 0.0;
      Zeta[a + b * KL] = up ? W.U[a * LD + b] * ra : 0.0;
      ZetaInv[a + b * KL] = up ? lr * rb : 0.0;
    }
  }
  cluster_wait();  // every CTA has read the state before the leader updates it
  if (lead) {
    st->best_col = h;
    st->nu_h = nh;
    st->r_from_v = 0;
    int done = 0;
    if (st->it >= st->maxit) {
      done = 1;
      st->done = 1;
      st->pw_skip = 0;  // the last iteration still completes its W, P update
      st->status = st->no_test ? 0 : 5;
    } else if (st->stag_check) {
      // A mixed-precision inner solve whose residual estimate has stopped falling has delivered
      // what FP32 can: end it (the exit combination and the FP64 true residual follow) so that the
      // refinement loop restarts from the FP64 residual instead of iterating on.
      if (nh < 0.9 * st->nu_ref) {
        st->nu_ref = nh;
        st->it_ref = st->it;
      } else if (st->it - st->it_ref > max(256, 2 * st->it_ref)) {
        done = 1;
        st->done = 1;
        st->pw_skip = 0;
        st->status = 0;
        st->stagnated = 1;  // not converged: the exit takes column h (the least-squares combination
                            // of drifted FP32 residuals is not to be trusted)
      }
    }
    if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
  }
}

// 1/d and 1/sqrt(d) exactly as the k x k steps take them of their pivots, one value per thread
// (grid-stride), for the component entry that checks them against their error bounds.
__global__ void k_pivot_recips(long long n, const double* __restrict__ d, double* __restrict__ inv,
                               double* __restrict__ rsq) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v = d[i];
    inv[i] = rcp_pos(v);
    rsq[i] = rsqrt_pos(v);
  }
}

// ------------------------------------------------------------------------------------ launchers

void launch_pivot_recips(cudaStream_t s, int n, const double* d, double* inv, double* rsq) {
  const int nb = n / 256 + 1 < 1024 ? n / 256 + 1 : 1024;
  k_pivot_recips<<<nb, 256, 0, s>>>(n, d, inv, rsq);
}

// Set-up: one warp (KP <= 8) or one CTA of 256 threads. Loop: a cluster of CTAs, computed 16 wide for
// KP <= 8 (the identity outside s x s) and stored at the handle's width.
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
#define WARP(K) k_small_xi_x<16, K><<<ClusterCfg<16>::CS, ClusterCfg<16>::NF, 0, s>>>(st, G1p, Sigma, Xi, T)
#define CTA(K) k_small_xi_x<K, K><<<ClusterCfg<K>::CS, ClusterCfg<K>::NF, 0, s>>>(st, G1p, Sigma, Xi, T)
  MBPCG_SMALL_SWITCH(kp, WARP, CTA)
#undef WARP
#undef CTA
}
void launch_small_zeta(cudaStream_t s, int kp, SolveState* st, const double* G2nu, double* Sigma, double* Zeta,
                       double* ZetaInv, cudaGraphConditionalHandle cond, int use_cond) {
#define WARP(K)                                                                                    \
  k_small_zeta_x<16, K><<<ClusterCfg<16>::CS, ClusterCfg<16>::NF, 0, s>>>(st, G2nu, Sigma, Zeta, ZetaInv, cond, \
                                                                        use_cond)
#define CTA(K) \
  k_small_zeta_x<K, K><<<ClusterCfg<K>::CS, ClusterCfg<K>::NF, 0, s>>>(st, G2nu, Sigma, Zeta, ZetaInv, cond, use_cond)
  MBPCG_SMALL_SWITCH(kp, WARP, CTA)
#undef WARP
#undef CTA
}

}  // namespace mbpcg
