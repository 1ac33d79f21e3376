// FP64-accurate products Y = X M of an n x K block X by a K x K matrix M (K = 32 or 16, the padded
// width) on the FP16 tensor cores (tcgen05), by the exact digit splitting of ozaki_digits.cuh: X
// split row by row (scale of the row), M column by column; a digit is exact in FP16. These are the k x k-row products of the block update and of the W/P
// update of Algorithm 1 (P T, (AP) T, (AP) Xi; V zeta^{-1}, P zeta^T), which on the FP64 pipe of
// this GPU (2 FMA per clock per SM) cost more than the A P product's digit stream.
//
// Exactness. The reduction index has K <= 32 values, so a level sum S_L = sum_{t+u=L} sum_l x^t_il m^u_lj
// is at most 8 * 32 * 127^2 < 2^22: every level of the FP32 accumulator is an exact integer. Levels
// 0..4 are combined in int64 (exact), levels 5..7 in FP32 (rounding below 2^-56 of the scales),
// levels above 7 are dropped (below 2^-56 of the scales), as in the dense A P product:
//     Y_ij = 2^(e_i + f_j - 2044) * sum_{L=0..7} S_L 2^(-14 - 7L);
// the two parts meet in one int64 below 2^62, converted to FP64 once (its only rounding).
//
// One CTA of 256 threads per (128-row tile, product, 16 output columns: K / 16 CTAs): M is staged
// in shared memory by one coalesced load; two threads per row write the 8 digits of their K / 2
// values of X into shared memory (K-major, no swizzle: 8 tiles of 128 x K FP16; 16-byte stores of 8
// consecutive digits; the row scale is combined by one shuffle), 2 K threads the 8 digits of the
// CTA's 16 columns of M (128 x K: row 16 u + j holds digit u of column j); one thread issues
// 8 K / 16 MMAs (digit t of X against digits 0..7-t of M, N = 16 (8 - t), into TMEM columns
// 16 t .. 127), and each warp drains 8 columns of its 32 rows (warps w and w + 4 share a TMEM lane
// quarter): 8 loads, the combination above, and one FP64 scaling per value. Two CTAs fit on an SM (81 KB of
// shared memory at K = 32, 128 TMEM columns each), so one phase of a CTA overlaps another's.
#include "kernels.h"
#include "ozaki_digits.cuh"
#include "tcgen05.cuh"

namespace mbpcg {

namespace {

constexpr int kRpRows = 128;                        // rows per CTA (= TMEM lanes)
constexpr int kRpN = 16;                            // output columns per CTA
constexpr int kRpThreads = 256;
constexpr uint32_t kRpTmemCols = kOzDigits * kRpN;  // 8 levels x 16 columns

// K = 32 or 16: columns of X, order of M (the padded width of the blocks)
template <int K>
struct RpCfg {
  static constexpr uint32_t ATile = kRpRows * K * 2;            // one digit of the X tile: 8 / 4 KB
  static constexpr uint32_t BBytes = kOzDigits * kRpN * K * 2;  // the digits of 16 columns of M
  static constexpr size_t Smem = 1024 + (size_t)kOzDigits * ATile + BBytes + K * K * sizeof(double);
  static constexpr uint32_t Sbo = (K / 8) * 128;                // 8-row groups of a K-wide tile
  static constexpr int Xh = K / 2;                              // values of a row per thread
  static constexpr int Halves = K / kRpN;                       // CTAs per (tile, product)
  static_assert(K == 16 || K == 32, "width");
};

// v 2^k for an integer k: an integer add to the exponent field while the result stays a normal
// number (no rounding: the FP64 pipe of this GPU is slow), else ldexp
__device__ __forceinline__ double scale2(double v, int k) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF) + k;
  if (v == 0.0) return v;
  return (e >= 1 && e <= 2046 && ((b >> 52) & 0x7FF) != 0) ? __longlong_as_double(b + (long long)k * (1LL << 52))
                                                            : ldexp(v, k);
}

// 8 FP16 digits (16 bytes) for 8 consecutive values of the reduction index
__device__ __forceinline__ uint4 pack8(const int (&d)[8]) {
  uint4 v;
  v.x = oz_f16_pair_of_ints(d[0], d[1]);
  v.y = oz_f16_pair_of_ints(d[2], d[3]);
  v.z = oz_f16_pair_of_ints(d[4], d[5]);
  v.w = oz_f16_pair_of_ints(d[6], d[7]);
  return v;
}

}  // namespace

template <int K>
__global__ void __launch_bounds__(kRpThreads)
k_rowprod_tc(int n, RowProdJobs jobs, const SolveState* __restrict__ st, int skip_on_pw, int* __restrict__ err) {
  using C = RpCfg<K>;
  if (st != nullptr && (skip_on_pw ? st->pw_skip : st->done)) return;
  extern __shared__ __align__(1024) uint8_t rsm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(rsm);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(rsm + 8);
  int* fexp = reinterpret_cast<int*>(rsm + 16);    // scales of this CTA's 16 columns of M
  int* erows = reinterpret_cast<int*>(rsm + 128);  // row scales of the X tile (128 ints)
  uint8_t* As = rsm + 1024;
  uint8_t* Bs = As + (size_t)kOzDigits * C::ATile;
  double* Ms = reinterpret_cast<double*>(Bs + C::BBytes);  // M as stored (column-major K x K)
  const RowProdJob J = jobs.j[blockIdx.y / C::Halves];
  const int jb = kRpN * (blockIdx.y % C::Halves);  // first output column of this CTA
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = tid >> 1, hx = tid & 1;  // digit phase: row r of the tile, values 16 hx .. 16 hx + 15
  const int row = blockIdx.x * kRpRows + r;

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, kRpTmemCols);
#pragma unroll
  for (int i = 0; i < K * K / kRpThreads; ++i) Ms[tid + kRpThreads * i] = J.M[tid + kRpThreads * i];
  // this thread's K / 2 values of its row of X (zeros past n)
  constexpr int kXh = C::Xh;
  double x[kXh];
  if (row < n) {
    const double2* xr = reinterpret_cast<const double2*>(J.X + (size_t)row * K + kXh * hx);
#pragma unroll
    for (int c = 0; c < kXh / 2; ++c) {
      const double2 v = xr[c];
      x[2 * c] = v.x;
      x[2 * c + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < kXh; ++c) x[c] = 0.0;
  }
  __syncthreads();  // M staged
  // element (l, j) of the matrix used: M, or M^T with transM
  auto mu = [&](int l, int j) { return J.transM ? Ms[j + l * K] : Ms[l + j * K]; };
  if (tid < kRpN) {
    int m = 0;
#pragma unroll 8
    for (int l = 0; l < K; ++l) m = max(m, biased_exponent(mu(l, jb + tid)));
    fexp[tid] = m;
  }
  int erow = 0;
#pragma unroll
  for (int c = 0; c < kXh; ++c) erow = max(erow, biased_exponent(x[c]));
  erow = max(erow, __shfl_xor_sync(0xffffffffu, erow, 1));  // the other half of the row
  if (hx == 0) erows[r] = erow;
#pragma unroll
  for (int c8 = 0; c8 < kXh; c8 += 8) {  // digits of x[c8 .. c8+7]: one 16-byte store per digit
    int d[8][kOzDigits];
#pragma unroll
    for (int e = 0; e < 8; ++e) ozaki_digits(x[c8 + e], erow, d[e]);
    const uint32_t off = umma_kmajor_offset(r, kXh * hx + c8, K);
#pragma unroll
    for (int t = 0; t < kOzDigits; ++t) {
      const int dt[8] = {d[0][t], d[1][t], d[2][t], d[3][t], d[4][t], d[5][t], d[6][t], d[7][t]};
      *reinterpret_cast<uint4*>(As + (size_t)t * C::ATile + off) = pack8(dt);
    }
  }
  __syncthreads();  // column and row scales ready
  if (tid < kRpN * (K / 8)) {  // column jj, values 8 g .. 8 g + 7 of l
    const int jj = tid % kRpN, g = tid / kRpN;
    int d[8][kOzDigits];
#pragma unroll
    for (int e = 0; e < 8; ++e) ozaki_digits(mu(8 * g + e, jb + jj), fexp[jj], d[e]);
#pragma unroll
    for (int u = 0; u < kOzDigits; ++u) {
      const int du[8] = {d[0][u], d[1][u], d[2][u], d[3][u], d[4][u], d[5][u], d[6][u], d[7][u]};
      *reinterpret_cast<uint4*>(Bs + umma_kmajor_offset(kRpN * u + jj, 8 * g, K)) = pack8(du);
    }
  }
  // the digits were written by ordinary stores; the MMAs read shared memory through the async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
#pragma unroll
    for (int t = 0; t < kOzDigits; ++t) {
      const uint32_t idesc = umma_idesc_f16_f32(kRpRows, kRpN * (kOzDigits - t));
#pragma unroll
      for (int k = 0; k < K / 16; ++k)
        umma_ss(tmem + (uint32_t)(kRpN * t), umma_smem_desc(a0 + (uint32_t)t * C::ATile + 256u * k, 128, C::Sbo),
                  umma_smem_desc(b0 + 256u * k, 128, C::Sbo), idesc, (t == 0 && k == 0) ? 0u : 1u);
    }
    umma_commit(bar);
  }
  const bool ok = mbar_wait_bounded(bar, 0);
  tc_fence_after_sync();
  if (ok) {
    // warp w: TMEM lane quarter w % 4 (rows 32 (w % 4) + lane), columns 8 (w / 4) .. + 7 of the 16
    constexpr int kDn = kRpN / 2;
    const int q4 = warp & 3, c0 = kDn * (warp >> 2), dr = 32 * q4 + lane;
    long long acc_i[kDn];
    float acc_f[kDn];
#pragma unroll
    for (int j = 0; j < kDn; ++j) {
      acc_i[j] = 0;
      acc_f[j] = 0.f;
    }
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q4) << 16);
    uint32_t rv[kOzDigits][kDn];  // all levels' loads in flight together, one wait
#pragma unroll
    for (int L = 0; L < kOzDigits; ++L) tmem_ld8(lane_base + (uint32_t)(kRpN * L + c0), rv[L]);
    tmem_wait_ld();
#pragma unroll
    for (int L = 0; L < kOzDigits; ++L) {
      if (L < 5) {
        const int sh = 7 * (4 - L);
#pragma unroll
        for (int j = 0; j < kDn; ++j) acc_i[j] += (long long)__float2int_rn(__uint_as_float(rv[L][j])) << sh;
      } else {
        const float sc = (L == 5) ? 1.f : (L == 6) ? 0x1p-7f : 0x1p-14f;
#pragma unroll
        for (int j = 0; j < kDn; ++j) acc_f[j] = fmaf(__uint_as_float(rv[L][j]), sc, acc_f[j]);
      }
    }
    // Y = 2^(e + f - 2100) (acc_i 2^14 + round(acc_f 2^7)): exact in int64 (|acc_i| < 2^48; the
    // rounding drops less than 2^-56 of the scales), one conversion to FP64, the scale by exponent
    const int orow = blockIdx.x * kRpRows + dr, er = erows[dr];
    if (orow < n) {
      double* yr = J.Y + (size_t)orow * K + jb + c0;
#pragma unroll
      for (int j = 0; j < kDn; j += 2) {
        double2 v;
        const long long t0 = (acc_i[j] << 14) + __float2ll_rn(acc_f[j] * 0x1p7f);
        const long long t1 = (acc_i[j + 1] << 14) + __float2ll_rn(acc_f[j + 1] * 0x1p7f);
        v.x = scale2((double)t0, er + fexp[c0 + j] - 2100);
        v.y = scale2((double)t1, er + fexp[c0 + j + 1] - 2100);
        *reinterpret_cast<double2*>(yr + j) = v;
      }
    }
  } else if (err != nullptr) {
    atomicExch(err, 1);
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, kRpTmemCols);
}

template <int K>
static void rowprod_tc_k(cudaStream_t s, int n, const RowProdJobs& jobs, int njobs, const SolveState* st,
                         int skip_on_pw, int* err) {
  using C = RpCfg<K>;
  ensure_dynamic_smem(k_rowprod_tc<K>, C::Smem);
  k_rowprod_tc<K><<<dim3((n + kRpRows - 1) / kRpRows, C::Halves * njobs), kRpThreads, C::Smem, s>>>(n, jobs, st,
                                                                                                    skip_on_pw, err);
}

void rowprod_tc(cudaStream_t s, int n, int kp, const RowProdJobs& jobs, int njobs, const SolveState* st,
                int skip_on_pw, int* err) {
  if (kp == 16) rowprod_tc_k<16>(s, n, jobs, njobs, st, skip_on_pw, err);
  else rowprod_tc_k<32>(s, n, jobs, njobs, st, skip_on_pw, err);
}

}  // namespace mbpcg
