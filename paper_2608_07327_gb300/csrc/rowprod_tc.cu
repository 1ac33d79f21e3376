// FP64-accurate products Y = X M of an n x K block X by a K x K matrix M (K = 32 or 16, the padded
// width) on the FP16 tensor cores (tcgen05), by the exact digit splitting of ozaki_digits.cuh: X
// split row by row (scale of the row), M column by column; a digit is exact in FP16. These are the
// k x k-row products of the block update and of the W/P update of Algorithm 1 (P T, (AP) T, (AP) Xi;
// V zeta^{-1}, P zeta^T), which on the FP64 pipe of this GPU (2 FMA per clock per SM) cost more than
// the A P product's digit stream.
//
// Exactness. The reduction index has K <= 32 values, so a level sum S_L = sum_{t+u=L} sum_l x^t_il m^u_lj
// is at most 8 * 32 * 127^2 < 2^22: every level of the FP32 accumulator is an exact integer. Levels
// 0..4 are combined in int64 (exact), levels 5..7 in FP32 (rounding below 2^-56 of the scales),
// levels above 7 are dropped (below 2^-56 of the scales), as in the dense A P product:
//     Y_ij = 2^(e_i + f_j - 2044) * sum_{L=0..7} S_L 2^(-14 - 7L);
// the two parts meet in one int64 below 2^62, converted to FP64 once (its only rounding).
//
// One CTA of 512 threads per (128-row tile, product), all K output columns. The kernel is a chain of
// short phases, so each is spread over all 16 warps and kept off the FP64 pipe:
//  - digits of X: four threads per row, K / 4 values each (the 8 lanes of a quarter warp take 8
//    rows, so the 16-byte digit stores hit distinct banks); the row scale is a max over the four by
//    two shuffles; the digit bytes of each value are spread into two words once, and digit t of two
//    values becomes an FP16 pair by one byte permutation, an OR and one FP16 multiply-add;
//  - digits of M: read straight from global memory, warp w holding column w (and w + 16) with lane =
//    reduction index, so the column scale is one warp max (redux.sync);
//  - one thread issues 8 K / 16 MMAs (digit t of X against digits 0..7-t of M, N = K (8 - t), into
//    TMEM columns K t .. 8 K - 1: column K L + j accumulates level L of output column j);
//  - warp w drains K / 4 columns of its TMEM lane quarter (w % 4): 8 loads, the combination above
//    (the integer levels taken out of the FP32 accumulator by an add, int64 multiply-adds) and the
//    int64 -> FP64 rounding with the scale in integer operations (int_to_fp64.cuh): conversions on
//    the FP64 pipe made this phase the longest one; the products are staged in shared memory and
//    written out as whole 16-byte-coalesced rows of the tile (the TMEM layout gives a thread one row).
#include "int_to_fp64.cuh"
#include "kernels.h"
#include "ozaki_digits.cuh"
#include "tcgen05.cuh"

namespace mbpcg {

namespace {

constexpr int kRpRows = 128;  // rows per CTA (= TMEM lanes)
constexpr int kRpThreads = 512;

// K = 32 or 16: columns of X, order of M (the padded width of the blocks)
template <int K>
struct RpCfg {
  static constexpr uint32_t ATile = kRpRows * K * 2;          // one digit of the X tile: 8 / 4 KB
  static constexpr uint32_t BBytes = kOzDigits * K * K * 2;   // the digits of M: row K u + j = digit u of column j
  static constexpr size_t Smem = 1024 + (size_t)kOzDigits * ATile + BBytes;
  static constexpr uint32_t Sbo = (K / 8) * 128;              // 8-row groups of a K-wide tile
  static constexpr int Vpt = K / 4;                           // values of a row per thread
  static constexpr int Cpw = K / 16;                          // columns of M per warp
  static constexpr int Dn = K / 4;                            // output columns per drain warp
  static constexpr uint32_t TmemCols = kOzDigits * K;         // 8 levels x K columns
  static_assert(K == 16 || K == 32, "width");
};

// An FP32 accumulator level holding an integer below 2^22 in magnitude, as that integer: adding
// 1.5 2^23 puts it in the low bits of the significand (exactly), an integer subtract takes it out.
__device__ __forceinline__ int oz_level_int(uint32_t raw) {
  return (int)(__float_as_uint(__uint_as_float(raw) + 12582912.0f) - 0x4B400000u);
}

template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&v)[N]) {
  if constexpr (N == 8) tmem_ld8(taddr, v);
  else tmem_ld4(taddr, v);
}

}  // namespace

template <int K>
__global__ void __launch_bounds__(kRpThreads, 1)
k_rowprod_tc(int n, RowProdJobs jobs, const SolveState* __restrict__ st, int skip_on_pw, int* __restrict__ err) {
  using C = RpCfg<K>;
  extern __shared__ __align__(1024) uint8_t rsm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(rsm);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(rsm + 8);
  int* fexp = reinterpret_cast<int*>(rsm + 16);    // column scales of M (K ints)
  int* erows = reinterpret_cast<int*>(rsm + 256);  // row scales of the X tile (128 ints)
  uint8_t* As = rsm + 1024;
  uint8_t* Bs = As + (size_t)kOzDigits * C::ATile;
  const RowProdJob J = blockIdx.y == 0 ? jobs.j[0] : blockIdx.y == 1 ? jobs.j[1] : jobs.j[2];  // no local copy
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // loads first, before the solve state is read (a skipped launch discards them): this thread's
  // values of X (row r of the tile, values Vpt q .. Vpt q + Vpt - 1) and of M (reduction index
  // lane, columns warp + 16 c)
  const int r = 8 * warp + (lane & 7), q = lane >> 3;
  const int row = blockIdx.x * kRpRows + r;
  double x[C::Vpt];
  if (row < n) {
    const double2* xr = reinterpret_cast<const double2*>(J.X + (size_t)row * K + C::Vpt * q);
#pragma unroll
    for (int c = 0; c < C::Vpt / 2; ++c) {
      const double2 v = xr[c];
      x[2 * c] = v.x;
      x[2 * c + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < C::Vpt; ++c) x[c] = 0.0;
  }
  double mv[C::Cpw];
#pragma unroll
  for (int c = 0; c < C::Cpw; ++c) {
    const int j = warp + 16 * c;
    mv[c] = lane < K ? (J.transM ? J.M[j + lane * K] : J.M[lane + j * K]) : 0.0;
  }
  if (st != nullptr && (skip_on_pw ? st->pw_skip : st->done)) return;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, C::TmemCols);  // while the loads are in flight

  // digits of X
  int erow = 0;
#pragma unroll
  for (int c = 0; c < C::Vpt; ++c) erow = max(erow, biased_exponent(x[c]));
  erow = max(erow, __shfl_xor_sync(0xffffffffu, erow, 8));
  erow = max(erow, __shfl_xor_sync(0xffffffffu, erow, 16));
  if (q == 0) erows[r] = erow;
  {
    uint32_t wh[C::Vpt], wl[C::Vpt], s2[C::Vpt / 2], c2[C::Vpt / 2];
    int sg[C::Vpt];
#pragma unroll
    for (int c = 0; c < C::Vpt; ++c) oz_digit_bytes(ozaki_magnitude(x[c], erow, sg[c]), wh[c], wl[c]);
#pragma unroll
    for (int p = 0; p < C::Vpt / 2; ++p) oz_sign_pair(sg[2 * p], sg[2 * p + 1], s2[p], c2[p]);
    const uint32_t off = umma_kmajor_offset(r, C::Vpt * q, K);
#pragma unroll
    for (int t = 0; t < kOzDigits; ++t) {
      uint32_t w[C::Vpt / 2];
#pragma unroll
      for (int p = 0; p < C::Vpt / 2; ++p)
        w[p] = t < 4 ? oz_f16_digit_pair(wh[2 * p], wh[2 * p + 1], t, s2[p], c2[p])
                     : oz_f16_digit_pair(wl[2 * p], wl[2 * p + 1], t, s2[p], c2[p]);
      if constexpr (C::Vpt == 8) *reinterpret_cast<uint4*>(As + (size_t)t * C::ATile + off) = make_uint4(w[0], w[1], w[2], w[3]);
      else *reinterpret_cast<uint2*>(As + (size_t)t * C::ATile + off) = make_uint2(w[0], w[1]);
    }
  }

  // digits of M: column j = warp + 16 c, reduction index l = lane
#pragma unroll
  for (int c = 0; c < C::Cpw; ++c) {
    const int j = warp + 16 * c;
    const int f = (int)__reduce_max_sync(0xffffffffu, (unsigned)biased_exponent(mv[c]));
    if (lane == 0) fexp[j] = f;
    if (lane < K) {
      int d[kOzDigits];
      ozaki_digits(mv[c], f, d);
#pragma unroll
      for (int u = 0; u < kOzDigits; ++u)
        *reinterpret_cast<uint16_t*>(Bs + umma_kmajor_offset(K * u + j, lane, K)) =
            (uint16_t)(oz_f16_pair_of_ints(d[u], 0) & 0xFFFFu);
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
      const uint32_t idesc = umma_idesc_f16_f32(kRpRows, K * (kOzDigits - t));
#pragma unroll
      for (int k = 0; k < K / 16; ++k)
        umma_ss(tmem + (uint32_t)(K * t), umma_smem_desc(a0 + (uint32_t)t * C::ATile + 256u * k, 128, C::Sbo),
                umma_smem_desc(b0 + 256u * k, 128, C::Sbo), idesc, (t == 0 && k == 0) ? 0u : 1u);
    }
    umma_commit(bar);
  }
  const bool ok = mbar_wait_bounded(bar, 0);
  tc_fence_after_sync();
  // drain: warp w takes TMEM lane quarter w % 4 (tile rows 32 (w % 4) + lane) and output columns
  // Dn (w / 4) .. + Dn - 1. The products go to a staging tile in shared memory (the X digits' space,
  // which the finished MMAs no longer read), its 16-byte chunks XOR-swizzled by row so that these
  // row-wise writes and the coalesced copy-out below both hit distinct banks.
  constexpr int Dn = C::Dn, Ch = K / 2;  // Ch: 16-byte chunks per row
  double* stage = reinterpret_cast<double*>(As);
  if (ok) {
    const int q4 = warp & 3, c0 = Dn * (warp >> 2), dr = 32 * q4 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q4) << 16);
    uint32_t rv[kOzDigits][Dn];  // all levels' loads in flight together, one wait
#pragma unroll
    for (int L = 0; L < kOzDigits; ++L) tmem_ld_cols<Dn>(lane_base + (uint32_t)(K * L + c0), rv[L]);
    tmem_wait_ld();
    const int er = erows[dr] - 2100;
#pragma unroll
    for (int j = 0; j < Dn; j += 2) {
      double y[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jj = j + h;
        // Y = 2^(e + f - 2100) (S0 2^42 + S1 2^35 + S2 2^28 + S3 2^21 + S4 2^14 + round(F 2^7)), F the
        // FP32 sum S5 + S6 2^-7 + S7 2^-14: exact in int64 (|F 2^7| < 2^29 rounds into 32 bits), one
        // rounding to FP64, the scale by exponent
        float f = fmaf(__uint_as_float(rv[5][jj]), 1.f, 0.f);
        f = fmaf(__uint_as_float(rv[6][jj]), 0x1p-7f, f);
        f = fmaf(__uint_as_float(rv[7][jj]), 0x1p-14f, f);
        const int a = oz_level_int(rv[3][jj]) * 128 + oz_level_int(rv[4][jj]);
        const int b = oz_level_int(rv[1][jj]) * 128 + oz_level_int(rv[2][jj]);
        const long long t = (long long)oz_level_int(rv[0][jj]) * (1LL << 42) + (long long)b * (1LL << 28) +
                            (long long)a * (1LL << 14) + (long long)__float2int_rn(f * 0x1p7f);
        const int k = er + fexp[c0 + jj];
        bool normal;
        y[h] = ll_to_double_scaled_rn(t, k, normal);
        if (!normal) y[h] = ldexp(ll_to_double_rn(t), k);
      }
      const int ch = (c0 + j) / 2;
      *reinterpret_cast<double2*>(stage + dr * K + 2 * (ch ^ (dr & (Ch - 1)))) = make_double2(y[0], y[1]);
    }
  } else if (err != nullptr) {
    atomicExch(err, 1);
  }
  __syncthreads();
  if (ok) {
    const int rows = min(kRpRows, n - (int)blockIdx.x * kRpRows);
    double* yt = J.Y + (size_t)blockIdx.x * kRpRows * K;
    for (int g = tid; g < rows * Ch; g += kRpThreads) {
      const int rr = g / Ch, ch = g % Ch;
      *reinterpret_cast<double2*>(yt + (size_t)rr * K + 2 * ch) =
          *reinterpret_cast<const double2*>(stage + rr * K + 2 * (ch ^ (rr & (Ch - 1))));
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, C::TmemCols);
}

template <int K>
static void rowprod_tc_k(cudaStream_t s, int n, const RowProdJobs& jobs, int njobs, const SolveState* st,
                         int skip_on_pw, int* err) {
  using C = RpCfg<K>;
  ensure_dynamic_smem(k_rowprod_tc<K>, C::Smem);
  k_rowprod_tc<K><<<dim3((n + kRpRows - 1) / kRpRows, njobs), kRpThreads, C::Smem, s>>>(n, jobs, st, skip_on_pw,
                                                                                        err);
}

void rowprod_tc(cudaStream_t s, int n, int kp, const RowProdJobs& jobs, int njobs, const SolveState* st,
                int skip_on_pw, int* err) {
  if (kp == 16) rowprod_tc_k<16>(s, n, jobs, njobs, st, skip_on_pw, err);
  else rowprod_tc_k<32>(s, n, jobs, njobs, st, skip_on_pw, err);
}

}  // namespace mbpcg
