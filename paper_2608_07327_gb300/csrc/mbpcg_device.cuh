// Device-side building blocks shared by every kernel of the MBPCG library (sm_103a).
//
// Layout in HBM: an n x s block of the method (X0, X~, R, W, P, A P, V of Algorithm 1) is stored
// row-major with the row width KP = s rounded up to a power of two (1..32). Columns s..KP-1 are
// kept at exactly zero by construction (the k x k kernels zero the padded rows/columns of every
// small matrix), so the padded lanes never change the result.
//
// FP64 cost model: on GB300 double precision runs at ~1.2 TFLOP/s against ~70 TFLOP/s FP32 and
// 6.6 TB/s HBM, so every k x k contraction on the per-row path is bound by the FP64 pipe. The
// kernels therefore count DFMAs: Gram matrices accumulate only the upper triangle, triangular
// products pair columns (j, KP-1-j) so that every lane runs the same trip count, and additions
// are folded into FMAs.
//
// Reductions are deterministic: every CTA writes its partial sums to its own slot and slots are
// summed in a fixed tree order, so repeated solves are bit-identical.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mbpcg {

constexpr int kThreads = 256;  // threads per CTA of every row kernel
constexpr int kMaxKP = 32;

// Control block of one solve, in device memory. Written only by single-CTA kernels; every other
// kernel reads it after a kernel boundary.
struct SolveState {
  int32_t it;          // iterations of the current inner solve
  int32_t maxit;       // cap of the current inner solve
  int32_t status;      // 0 ok, 5 not converged, 6 breakdown
  int32_t done;        // 1: the iteration loop stops (read by every loop kernel)
  int32_t pw_skip;     // 1: the W/P update of this iteration is not needed
  int32_t best_col;    // h
  int32_t ls_fallback; // exit used column h
  int32_t converged;   // exit test passed
  int32_t no_test;     // diagnostic mode: run exactly maxit iterations
  int32_t s;           // number of copies
  int32_t restart;     // index of the current inner solve (0 = the user's right-hand side)
  int32_t kerr;        // 1: a kernel's bounded wait timed out (the solve returns MBPCG_ERR_TIMEOUT)
  int32_t r_from_v;    // implicit-residual mode: 1 if the current residual block is V Sigma, 0 if W Sigma
  double tol_rel;      // tolerance of the current inner solve, relative to ||rhs||
  double tol_abs;      // tol_rel * ||rhs||
  double rhs_norm;     // ||rhs|| of the current inner solve (original metric)
  double b_norm;       // ||b|| of the user's right-hand side
  double scale;        // X0 = scale * U
  double nu_h;         // ||R_h|| at the last test (original metric)
  double ls_res;       // ||rhs - Bhat c|| of the exit combination
  double true_res;     // ||b - A x||
  // Chronopoulos-Gear CG scalars
  double cg_gamma_old, cg_alpha_old, cg_alpha, cg_beta;
  // stagnation exit of the mixed-precision inner solves (stag_check = 1): the inner solve ends when
  // nu_h has not fallen below 0.9 nu_ref for more than max(256, 2 it_ref) iterations
  double nu_ref;       // last nu_h that was 10 % below the one before
  int32_t it_ref;      // iteration of nu_ref
  int32_t stag_check;  // 1: the rule is on (mixed precision, not in diagnostic mode)
  int32_t stagnated;   // 1: the current inner solve ended by the rule
  int32_t pad_;
};

// Per-KP launch shape of the row kernels: a thread owns CPT consecutive columns of one row
// (CPT = KP for KP <= 4, else 2), TPR threads share a row, a tile holds ROWS rows.
template <int KP>
struct Cfg {
  static constexpr int CPT = (KP <= 4) ? KP : 2;
  static constexpr int TPR = KP / CPT;
  static constexpr int ROWS = kThreads / TPR;
  static constexpr int NPACK = KP * (KP + 1) / 2;
};

__host__ __device__ constexpr int npack(int kp) { return kp * (kp + 1) / 2; }
// packed index of entry (l, j), l <= j, of a symmetric KP x KP matrix (upper triangle, by column)
__host__ __device__ inline int pidx(int l, int j) { return j * (j + 1) / 2 + l; }
__device__ inline void punpack(int e, int& l, int& j) {
  // j = floor((sqrt(8e + 1) - 1) / 2) from an FP32 square root, then made exact by one step each way
  j = (int)((sqrtf((float)(8 * e + 1)) - 1.f) * 0.5f);
  if ((j + 1) * (j + 2) / 2 <= e) ++j;
  if (j * (j + 1) / 2 > e) --j;
  l = e - j * (j + 1) / 2;
}

// Balanced contiguous row range of this CTA.
__device__ inline void row_range(int n, int& r0, int& r1) {
  r0 = (int)(((long long)n * blockIdx.x) / gridDim.x);
  r1 = (int)(((long long)n * (blockIdx.x + 1)) / gridDim.x);
}

__host__ __device__ constexpr int pow2_ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Vector load/store of C consecutive doubles; the address is 16-byte aligned whenever C >= 2
// (rows are KP*8 bytes, chunks start at even columns, buffers are 256-byte aligned).
template <int C>
__device__ __forceinline__ void ldv(const double* __restrict__ p, double (&v)[C]) {
  if constexpr (C == 1) {
    v[0] = __ldg(p);
  } else {
#pragma unroll
    for (int c = 0; c < C; c += 2) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(p + c));
      v[c] = t.x;
      v[c + 1] = t.y;
    }
  }
}
template <int C>
__device__ __forceinline__ void ldv_plain(const double* p, double (&v)[C]) {
  if constexpr (C == 1) {
    v[0] = *p;
  } else {
#pragma unroll
    for (int c = 0; c < C; c += 2) {
      const double2 t = *reinterpret_cast<const double2*>(p + c);
      v[c] = t.x;
      v[c + 1] = t.y;
    }
  }
}
template <int C>
__device__ __forceinline__ void stv(double* p, const double (&v)[C]) {
  if constexpr (C == 1) {
    *p = v[0];
  } else {
#pragma unroll
    for (int c = 0; c < C; c += 2) *reinterpret_cast<double2*>(p + c) = make_double2(v[c], v[c + 1]);
  }
}

// Deterministic in-CTA tree sum over the leading dimension of buf[m][e] (m rows of e entries,
// row-major in shared memory); the result is left in buf[0][0..e). All threads must call it.
__device__ inline void cta_tree_sum(double* buf, int m, int e) {
  for (int half = pow2_ceil(m) / 2; half >= 1; half >>= 1) {
    __syncthreads();
    for (int q = threadIdx.x; q < half * e; q += blockDim.x) {
      const int s = q / e, r = q - s * e;
      if (s + half < m) buf[s * e + r] += buf[(s + half) * e + r];
    }
  }
  __syncthreads();
}

// Upper triangle of X^T Y over the rows of a tile staged in shared memory (row stride KP).
// Threads own 2x2 blocks (bl <= bj) of the KP x KP result and a residue class of rows, so every
// thread issues the same number of FMAs. KP = 1 degenerates to one scalar per thread.
template <int KP>
struct GramTile {
  static constexpr int NB2 = (KP + 1) / 2;
  static constexpr int NBLK = NB2 * (NB2 + 1) / 2;
  static constexpr int RS = kThreads / NBLK;  // row classes
  static constexpr int RED = RS * NBLK * 4;   // doubles of shared scratch for finish()
  int bl, bj, blk, split;
  bool active;
  double a00, a01, a10, a11;

  __device__ __forceinline__ void init(int tid) {
    active = tid < NBLK * RS;
    blk = tid % NBLK;
    split = tid / NBLK;
    bj = 0;
    while ((bj + 1) * (bj + 2) / 2 <= blk) ++bj;
    bl = blk - bj * (bj + 1) / 2;
    a00 = a01 = a10 = a11 = 0.0;
  }
  __device__ __forceinline__ void accumulate(const double* Xs, const double* Ys, int nrows) {
    if (!active) return;
    if constexpr (KP == 1) {
      for (int r = split; r < nrows; r += RS) a00 = fma(Xs[r], Ys[r], a00);
    } else {
      for (int r = split; r < nrows; r += RS) {
        const double2 x = *reinterpret_cast<const double2*>(Xs + r * KP + 2 * bl);
        const double2 y = *reinterpret_cast<const double2*>(Ys + r * KP + 2 * bj);
        a00 = fma(x.x, y.x, a00);
        a01 = fma(x.x, y.y, a01);
        a10 = fma(x.y, y.x, a10);
        a11 = fma(x.y, y.y, a11);
      }
    }
  }
  // Sums the row classes in a fixed tree and writes the packed upper triangle to out[0..NPACK).
  __device__ void finish(double* red, double* out) {
    __syncthreads();
    if (active) {
      const int o = (split * NBLK + blk) * 4;
      red[o] = a00;
      red[o + 1] = a01;
      red[o + 2] = a10;
      red[o + 3] = a11;
    }
    cta_tree_sum(red, RS, NBLK * 4);
    for (int e = threadIdx.x; e < KP * (KP + 1) / 2; e += blockDim.x) {
      int l, j;
      punpack(e, l, j);
      const int b = (j / 2) * (j / 2 + 1) / 2 + l / 2;
      out[e] = red[b * 4 + (l & 1) * 2 + (j & 1)];
    }
    __syncthreads();
  }
};

// SplitMix64 (Steele, Lea & Flood 2014) in counter-based form, for the U == NULL option.
__host__ __device__ inline uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline double splitmix_uniform01(uint64_t seed, uint64_t stream, uint64_t index) {
  const uint64_t g = 0x9E3779B97F4A7C15ull;
  const uint64_t key = splitmix_mix(seed + (stream + 1) * g);
  const uint64_t w = splitmix_mix(key + (index + 1) * g);
  return (double)(w >> 11) * 0x1.0p-53;
}

}  // namespace mbpcg
