// k x k (k = s <= 32) steps of Algorithm 1 and the reductions that feed them. These run on one CTA
// between the row passes; matrices are column-major KP x KP in global memory with every entry
// outside the leading s x s block kept at zero (so the row kernels can run at width KP).
#pragma once
#include <cfloat>

#include "mbpcg_device.cuh"

namespace mbpcg {

constexpr int kSmallThreads = 256;

constexpr int kReduceThreads = 128;  // threads per entry in k_reduce

// out[e] = sum over p < nparts of part[p * pstride + e] for e < nent, in a fixed order.
__global__ void k_reduce(const double* __restrict__ part, int nparts, int pstride, double* __restrict__ out, int nent,
                         const SolveState* __restrict__ st);

// Right-looking Cholesky G = Z^T Z of the leading s x s block of A (shared memory, column-major,
// leading dimension KP); on return the upper triangle of A holds Z and the rest is zero.
// Breakdown (returns 1) when a pivot is not finite or not above 64 eps max_j G_jj.
__device__ inline int cta_cholesky(int s, int KP, double* A, int* flag) {
  const int tid = threadIdx.x;
  __shared__ double maxd;
  if (tid == 0) {
    double m = 0.0;
    for (int j = 0; j < s; ++j) m = fmax(m, fabs(A[j + j * KP]));
    maxd = m;
    *flag = 0;
  }
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (tid == 0) {
      const double piv = A[j + j * KP];
      if (!isfinite(piv) || !(piv > 64.0 * DBL_EPSILON * maxd)) *flag = 1;
      else A[j + j * KP] = sqrt(piv);
    }
    __syncthreads();
    if (*flag) return 1;
    const double inv = 1.0 / A[j + j * KP];
    for (int m = j + 1 + tid; m < s; m += blockDim.x) A[j + m * KP] *= inv;
    __syncthreads();
    // trailing update of the upper triangle: A[l][m] -= Z[j][l] Z[j][m], j < l <= m < s
    const int t = s - j - 1;
    for (int q = tid; q < t * t; q += blockDim.x) {
      const int l = j + 1 + q % t, m = j + 1 + q / t;
      if (l <= m) A[l + m * KP] = fma(-A[j + l * KP], A[j + m * KP], A[l + m * KP]);
    }
    __syncthreads();
  }
  for (int q = tid; q < KP * KP; q += blockDim.x) {
    const int l = q % KP, m = q / KP;
    if (l > m || l >= s || m >= s) A[q] = 0.0;
  }
  __syncthreads();
  return 0;
}

// Zi = Z^{-1} for upper triangular Z (leading s x s, column-major, ld KP); thread j solves column j
// by back substitution with precomputed reciprocals of the diagonal. Zi is zero outside s x s.
__device__ inline void cta_tri_inv_upper(int s, int KP, const double* Z, double* Zi, double* rdiag) {
  const int tid = threadIdx.x;
  for (int q = tid; q < KP * KP; q += blockDim.x) Zi[q] = 0.0;
  if (tid < s) rdiag[tid] = 1.0 / Z[tid + tid * KP];
  __syncthreads();
  if (tid < s) {
    const int j = tid;
    Zi[j + j * KP] = rdiag[j];
    for (int i = j - 1; i >= 0; --i) {
      double a = 0.0;
      for (int l = i + 1; l <= j; ++l) a = fma(Z[i + l * KP], Zi[l + j * KP], a);
      Zi[i + j * KP] = -a * rdiag[i];
    }
  }
  __syncthreads();
}

// Unpack a packed upper triangle (length KP(KP+1)/2) into a full symmetric KP x KP column-major
// matrix restricted to the leading s x s block (zeros elsewhere).
__device__ inline void cta_unpack_sym(int s, int KP, const double* packed, double* A) {
  for (int q = threadIdx.x; q < KP * KP; q += blockDim.x) {
    const int l = q % KP, m = q / KP;
    double v = 0.0;
    if (l < s && m < s) v = (l <= m) ? packed[pidx(l, m)] : packed[pidx(m, l)];
    A[q] = v;
  }
  __syncthreads();
}

}  // namespace mbpcg
