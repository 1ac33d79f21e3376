// FP64-accurate dense product Q = A P on the BF16 tensor cores (tcgen05), by exact splitting
// (Ozaki et al., "Error-free transformations of matrix multiplication by using fast routines of
// matrix multiplication and its applications", Numer. Algorithms 2012).
//
// Splitting. Each row i of A (A is symmetric, so row i = column i) is scaled by 2^-F_i, F_i the
// largest binary exponent in the row, and the magnitude of every entry is written as 8 base-128
// digits taken straight from its 53-bit significand (integer shifts, truncation below 2^-56 of the
// row scale). Columns of P are split the same way with their own scales G_j. A digit is an integer
// in [-127, 127], exact in BF16. Then
//     (A P)_ij = 2^(F_i + G_j) * sum_{L=2..16} 2^(-7L) * S_L,   S_L = sum_{t+u=L} sum_l a^t_il b^u_lj
// and the terms with t + u > 9 are below 2^-56 of the row/column scales and are dropped.
//
// Exactness. A product of two digits is < 2^14, so a level-L sum over a window of 128 values of l
// is at most (L-1) * 127^2 * 128 < 2^24 for L <= 6: the FP32 accumulator of the tensor core holds
// it exactly. Levels 2..6 are therefore drained from TMEM every 128 values of l and combined in
// int64 (exact); levels 7..9 are carried in FP32 (their rounding is below 2^-58 of the scale).
// The result has the accuracy of an FP64 product (error ~2^-53 |A||P|; an FP64 GEMM's bound is
// n 2^-53 |A||P|).
//
// Data movement. Digits are stored in global memory already in the tensor-core operand layout
// (K-major, no swizzle, 128 x 64 tiles of 16 KB for A, 8*KPT x 64 tiles for P), so whole tiles move
// with 1-D TMA bulk copies into shared memory: the digits of one (M tile, chunk) are adjacent, and
// one copy brings kOzDPS of them into a stage (5 stages of 32 KB, 2 P buffers). Fewer, larger
// stages matter: each stage hand-off is a round trip through two mbarriers and two threads. The MMA for digit t of A
// uses all needed digits of P at once (N = KPT * (9 - t)), writing levels t+1..9 of the
// accumulator. Producer, MMA issuer and drain run in separate warps; every wait is bounded.
#include "kernels.h"
#include "ozaki_digits.cuh"
#include "tcgen05.cuh"

namespace mbpcg {

namespace {

constexpr int kOzMT = 128;                             // rows per M tile (= TMEM lanes)
constexpr int kOzKC = 64;                              // reduction index per chunk
constexpr int kOzWin = 2;                              // chunks per exact window (128 values of l)
constexpr uint32_t kATileBytes = kOzMT * kOzKC * 2;    // 16 KB: one digit of one (M tile, chunk)
constexpr int kOzDPS = 2;                              // A digits per shared-memory stage
constexpr int kOzAStages = 5;                          // stages of kOzDPS digits (32 KB each)
constexpr int kOzPBufs = 2;
constexpr uint32_t kAStageBytes = kOzDPS * kATileBytes;
constexpr int kOzStagesPerChunk = kOzDigits / kOzDPS;
static_assert(kOzDigits % kOzDPS == 0, "a stage holds whole digits of one chunk");

}  // namespace

// emax[i] = largest biased exponent of row i of the column-major symmetric A (= column i).
__global__ void k_oz_rowexp(int n, const double* __restrict__ A, int* __restrict__ emax) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double* row = A + (size_t)warp * n;
  int m = 0;
  for (int l = lane; l < n; l += 32) m = max(m, biased_exponent(row[l]));
  for (int off = 16; off; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if (lane == 0) emax[warp] = m;
}

// Digits of A into tiles [mtile][kchunk][digit] of 128 x 64 bf16 (canonical K-major layout).
__global__ void k_oz_slice_a(int n, int nK, const double* __restrict__ A, const int* __restrict__ emax,
                             uint16_t* __restrict__ tiles) {
  const size_t total = (size_t)n * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / n), l = (int)(q % n);
    int d[kOzDigits];
    ozaki_digits(A[q], emax[i], d);  // A[i*n + l] = row i (symmetric)
    const size_t tile0 = ((size_t)(i / kOzMT) * nK + l / kOzKC) * kOzDigits;
    const uint32_t off = umma_kmajor_offset(i % kOzMT, l % kOzKC, kOzKC) / 2;
#pragma unroll
    for (int t = 0; t < kOzDigits; ++t) tiles[(tile0 + t) * (kATileBytes / 2) + off] = bf16_of_int(d[t]);
  }
}

// emaxP[j] = max over rows of the biased exponent of P[:, j] (atomicMax of integers: order-free).
// Element-parallel: the thread stride is a multiple of KP, so each thread stays on one column.
template <int KP>
__global__ void k_oz_colexp(int n, const double* __restrict__ P, int* __restrict__ emaxP,
                            const SolveState* __restrict__ st) {
  if (st != nullptr && st->done) return;
  __shared__ int m[KP];
  if (threadIdx.x < KP) m[threadIdx.x] = 0;
  __syncthreads();
  const size_t total = (size_t)n * KP, stride = (size_t)gridDim.x * blockDim.x;
  const size_t q0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  int loc = 0;
  for (size_t q = q0; q < total; q += stride) loc = max(loc, biased_exponent(P[q]));
  atomicMax(&m[q0 % KP], loc);
  __syncthreads();
  if (threadIdx.x < KP) atomicMax(&emaxP[threadIdx.x], m[threadIdx.x]);
}

// Digits of P into chunks [kchunk] of (8 * KPT) x 64 bf16, row index KPT * t + j (canonical
// K-major layout, so digit t of every column j is one contiguous N-range).
template <int KP, int KPT>
__global__ void k_oz_slice_p(int n, const double* __restrict__ P, const int* __restrict__ emaxP,
                             uint16_t* __restrict__ chunks, const SolveState* __restrict__ st) {
  if (st != nullptr && st->done) return;
  constexpr uint32_t kChunkElems = kOzDigits * KPT * kOzKC;
  const size_t total = (size_t)n * KP;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(q / KP), j = (int)(q % KP);
    int d[kOzDigits];
    ozaki_digits(P[q], emaxP[j], d);
    uint16_t* ch = chunks + (size_t)(l / kOzKC) * kChunkElems;
#pragma unroll
    for (int t = 0; t < kOzDigits; ++t) ch[umma_kmajor_offset(KPT * t + j, l % kOzKC, kOzKC) / 2] = bf16_of_int(d[t]);
  }
}

template <int KPT>
struct OzCfg {
  static constexpr uint32_t kPChunkBytes = kOzDigits * KPT * kOzKC * 2;
  static constexpr uint32_t kAccCols = 8 * KPT;                         // one accumulator set
  static constexpr uint32_t kTmemCols = (2 * kAccCols <= 256) ? 256 : 512;  // two sets (double buffer)
  static constexpr size_t kBarBytes = 1024;  // barriers + TMEM slot, keeps tiles 1024-aligned
  static constexpr size_t kSmem = kBarBytes + (size_t)kOzAStages * kAStageBytes + (size_t)kOzPBufs * kPChunkBytes;
};
static_assert(OzCfg<32>::kSmem <= 227 * 1024, "shared memory of one CTA");

constexpr int kOzDrainWarps = 4;                      // warps 0..3: TMEM lane quarters 0..3
constexpr int kOzProducerWarp = 4;                    // TMA issue
constexpr int kOzMmaWarp = 5;                         // MMA issue
constexpr int kOzTcThreads = 32 * 6;

// Work split (stream-K over windows). The product is nM row tiles x nW windows of wl chunks each
// (wl = 2: one exact window of 128 values of l; wl = 1 for small n). The U = nM nW windows, tile
// by tile, are cut into gridDim.x contiguous ranges of equal length (+-1), one per CTA, so the CTAs
// get the same work whatever nM is. A range that crosses a tile boundary is two (or more)
// segments; each segment of tile m writes its partial rows to slice (CTA - first CTA of tile m) of
// Qpart, and the split sum adds the slices of each tile in slice order (deterministic).
__host__ __device__ __forceinline__ int oz_cta_of(long long f, int G, long long U) {
  return (int)(((f + 1) * G + U - 1) / U) - 1;  // the CTA whose window range holds flat window f
}
__host__ __device__ __forceinline__ int oz_slices(int mt, int nW, int G, long long U) {
  return oz_cta_of((long long)(mt + 1) * nW - 1, G, U) - oz_cta_of((long long)mt * nW, G, U) + 1;
}

// Qpart[k][i][j] = the part of (A P)_ij over the K range of slice k of row i's tile, for j < KP.
// Warp-specialised: a producer thread streams A-digit tiles and P-digit chunks into shared memory
// (empty/full mbarriers), an MMA thread issues tcgen05.mma into one of two TMEM accumulator sets,
// alternating per window, and four drain warps read a finished set (levels 2..6 exact in int64,
// 7..9 in FP32) while the MMA thread fills the other.
template <int KPT>
__global__ void __launch_bounds__(kOzTcThreads, 1)
k_dense_tc(int n, int KP, int nK, int wl, int nW, const uint8_t* __restrict__ Atiles, const int* __restrict__ emaxA,
           const uint8_t* __restrict__ Pchunks, const int* __restrict__ emaxP, double* __restrict__ Qpart,
           int* __restrict__ err, const SolveState* __restrict__ st, int dir) {
  using C = OzCfg<KPT>;
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(1024) uint8_t osm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(osm);
  uint64_t* empty = full + kOzAStages;
  uint64_t* pfull = empty + kOzAStages;
  uint64_t* pempty = pfull + kOzPBufs;
  uint64_t* accf = pempty + kOzPBufs;  // [2] accumulator set ready for draining
  uint64_t* acce = accf + 2;           // [2] accumulator set drained
  uint64_t* fin = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  uint8_t* As = osm + C::kBarBytes;
  uint8_t* Ps = As + (size_t)kOzAStages * kAStageBytes;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, g = blockIdx.x;
  const long long U = (long long)((n + kOzMT - 1) / kOzMT) * nW;
  const long long f0 = U * g / G;
  const int nwin = (int)(U * (g + 1) / G - f0);
  // Window order: on odd iterations of a solve each CTA walks its range backwards, so that it starts
  // on the digits the previous product read last, the ones most likely still in L2 (A is read every
  // iteration).
  if (st != nullptr) dir ^= st->it & 1;

  if (tid == 0) {
    for (int q = 0; q < kOzAStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < kOzPBufs; ++q) {
      mbar_init(&pfull[q], 1);
      mbar_init(&pempty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], kOzDrainWarps);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, C::kTmemCols);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  int issued_a = 0, issued_p = 0;  // copies issued (producer thread only)

  if (warp == kOzProducerWarp) {
    if (lane == 0) {
      const uint64_t pol_stream = l2_policy_evict_first();  // A digits: 16 B per entry of A, read once
      bool ok = true;
      int cc = 0;  // chunks of this CTA so far
      for (int w = 0; w < nwin && ok; ++w) {
        const long long f = f0 + (dir ? nwin - 1 - w : w);
        const int mt = (int)(f / nW), c0 = (int)(f % nW) * wl, c1 = min(nK, c0 + wl);
        for (int c = c0; c < c1 && ok; ++c, ++cc) {
          const int b = cc % kOzPBufs;
          if (cc >= kOzPBufs) ok = mbar_wait_bounded(&pempty[b], (uint32_t)((cc / kOzPBufs - 1) & 1));
          if (!ok) break;
          mbar_arrive_expect_tx(&pfull[b], C::kPChunkBytes);
          tma_load_1d(Ps + (size_t)b * C::kPChunkBytes, Pchunks + (size_t)c * C::kPChunkBytes, C::kPChunkBytes,
                      &pfull[b]);
          issued_p = cc + 1;
          for (int u = 0; u < kOzStagesPerChunk && ok; ++u) {
            const int j = cc * kOzStagesPerChunk + u, q = j % kOzAStages;
            if (j >= kOzAStages) ok = mbar_wait_bounded(&empty[q], (uint32_t)((j / kOzAStages - 1) & 1));
            if (!ok) break;
            mbar_arrive_expect_tx(&full[q], kAStageBytes);
            tma_load_1d_hint(As + (size_t)q * kAStageBytes,
                             Atiles + (((size_t)mt * nK + c) * kOzDigits + u * kOzDPS) * kATileBytes, kAStageBytes,
                             &full[q], pol_stream);
            issued_a = j + 1;
          }
          if (*abort_flag) ok = false;
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (err != nullptr) atomicExch(err, 1);
      }
    }
  } else if (warp == kOzMmaWarp) {
    if (lane == 0) {
      bool ok = true;
      int cc = 0;
      for (int w = 0; w < nwin && ok; ++w) {
        const int ab = w & 1;
        if (w >= 2) ok = mbar_wait_bounded(&acce[ab], (uint32_t)((w / 2 - 1) & 1));
        tc_fence_after_sync();
        const long long f = f0 + (dir ? nwin - 1 - w : w);
        const int c0 = (int)(f % nW) * wl, nc = min(nK, c0 + wl) - c0, cc0 = cc;
        for (; cc < cc0 + nc && ok; ++cc) {
          const int b = cc % kOzPBufs;
          ok = mbar_wait_bounded(&pfull[b], (uint32_t)((cc / kOzPBufs) & 1));
          const uint32_t b_base = smem_addr(Ps + (size_t)b * C::kPChunkBytes);
          for (int u = 0; u < kOzStagesPerChunk && ok; ++u) {
            const int j = cc * kOzStagesPerChunk + u, q = j % kOzAStages;
            ok = mbar_wait_bounded(&full[q], (uint32_t)((j / kOzAStages) & 1));
            if (!ok) break;
#pragma unroll
            for (int dd = 0; dd < kOzDPS; ++dd) {
              const int t = u * kOzDPS + dd;
              const uint32_t a_base = smem_addr(As + (size_t)q * kAStageBytes + (size_t)dd * kATileBytes);
              const uint32_t idesc = umma_idesc_bf16_f32(kOzMT, KPT * (kOzDigits - t));
              const uint32_t d = tmem + (uint32_t)(ab * C::kAccCols + KPT * t);
#pragma unroll
              for (int k4 = 0; k4 < kOzKC / 16; ++k4) {
                const uint32_t first = (cc == cc0 && t == 0 && k4 == 0) ? 0u : 1u;
                umma_bf16(d, umma_smem_desc(a_base + 256u * k4, 128, 1024),
                          umma_smem_desc(b_base + 256u * k4, 128, 1024), idesc, first);
              }
            }
            umma_commit(&empty[q]);
          }
          if (ok) umma_commit(&pempty[b]);
          if (*abort_flag) ok = false;
        }
        if (!ok) *abort_flag = 1;  // before the commit, so the drain warps see it
        umma_commit(&accf[ab]);
      }
      if (!ok) {
        *abort_flag = 1;
        if (err != nullptr) atomicExch(err, 1);
      }
      umma_commit(fin);
      mbar_wait_bounded(fin, 0);
    }
  } else {
    // drain warps 0..3: warp w reads TMEM lanes 32w..32w+31 = rows of this M tile
    long long acc_i[KPT];
    float acc_f[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      acc_i[j] = 0;
      acc_f[j] = 0.f;
    }
    bool ok = true;
    for (int w = 0; w < nwin; ++w) {
      const int ab = w & 1;
      if (!mbar_wait_bounded(&accf[ab], (uint32_t)((w / 2) & 1))) ok = false;
      tc_fence_after_sync();
      if (!ok || *abort_flag) {
        ok = false;
        break;
      }
      const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(ab * C::kAccCols);
#pragma unroll
      for (int L = 0; L < kOzDigits; ++L) {
        float v[KPT];
        if constexpr (KPT == 32) {
          uint32_t r[32];
          tmem_ld32(lane_base + (uint32_t)(KPT * L), r);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
        } else {
          uint32_t r[16];
          tmem_ld16(lane_base + (uint32_t)(KPT * L), r);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
        }
        if (L < 5) {
          const int sh = 7 * (4 - L);
#pragma unroll
          for (int j = 0; j < KPT; ++j) acc_i[j] += (long long)__float2int_rn(v[j]) << sh;
        } else {
          const float sc = (L == 5) ? 1.f : (L == 6) ? 0x1p-7f : 0x1p-14f;
#pragma unroll
          for (int j = 0; j < KPT; ++j) acc_f[j] = fmaf(v[j], sc, acc_f[j]);
        }
      }
      tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[ab]);
      const long long f = f0 + (dir ? nwin - 1 - w : w);
      if (w == nwin - 1 || (dir ? f % nW == 0 : (f + 1) % nW == 0)) {  // end of a segment: its tile's rows
        const int mt = (int)(f / nW), row = mt * kOzMT + 32 * warp + lane;
        const int slice = g - oz_cta_of((long long)mt * nW, G, U);
        if (row < n) {
          const int fa = emaxA[row] - 1022;
          double* out = Qpart + ((size_t)slice * n + row) * KP;
#pragma unroll
          for (int j = 0; j < KPT; ++j) {
            if (j < KP) {
              const double v = (double)acc_i[j] * 0x1p-42 + (double)acc_f[j] * 0x1p-49;
              out[j] = ldexp(v, fa + emaxP[j] - 1022);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
          acc_i[j] = 0;
          acc_f[j] = 0.f;
        }
      }
    }
    if (!ok || *abort_flag) {
      *abort_flag = 1;
      if (err != nullptr) atomicExch(err, 1);
    }
  }
  __syncthreads();
  if (*abort_flag && tid == 32 * kOzProducerWarp) {
    // let the copies still in flight land before the shared memory is released (bounded waits);
    // only the last issue into each stage or buffer can still be pending
    for (int j = max(0, issued_a - kOzAStages); j < issued_a; ++j)
      mbar_wait_bounded(&full[j % kOzAStages], (uint32_t)((j / kOzAStages) & 1));  // stages of kOzDPS digits
    for (int cc = max(0, issued_p - kOzPBufs); cc < issued_p; ++cc)
      mbar_wait_bounded(&pfull[cc % kOzPBufs], (uint32_t)((cc / kOzPBufs) & 1));
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, C::kTmemCols);
}

// Q[i][j] = sum over the slices of row i's tile of Qpart[k][i][j], in slice order. Block 0 then
// clears the column exponents of P for the next product (they are rebuilt by the W/P update,
// which writes P).
template <int KP>
__global__ void k_oz_sum(int n, int nW, const double* __restrict__ Qpart, double* __restrict__ Q,
                         int* __restrict__ emaxP, const SolveState* __restrict__ st, int nctas) {
  if (st != nullptr && st->done) return;
  const size_t total = (size_t)n * KP;
  const long long U = (long long)((n + kOzMT - 1) / kOzMT) * nW;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int ns = oz_slices((int)(q / KP) / kOzMT, nW, nctas, U);
    double a = Qpart[q];
    for (int k = 1; k < ns; ++k) a += Qpart[(size_t)k * total + q];
    Q[q] = a;
  }
  if (blockIdx.x == 0 && threadIdx.x < KP) emaxP[threadIdx.x] = 0;
}

// The same split sum fused with the CTA partials of the upper triangle of P^T Q (the Gram of the
// Xi step of Algorithm 1), one pass over balanced row ranges (partials as k_gram writes them).
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_oz_sum_gram(int n, int nW, const double* __restrict__ Qpart, const double* __restrict__ P, double* __restrict__ Q,
              int* __restrict__ emaxP, double* __restrict__ part, int pstride, const SolveState* __restrict__ st, int nctas) {
  using C = Cfg<KP>;
  using G = GramTile<KP>;
  if (st != nullptr && st->done) return;
  __shared__ __align__(16) double Xs[C::ROWS * KP];
  __shared__ __align__(16) double Ys[C::ROWS * KP];
  __shared__ __align__(16) double red[G::RED];
  const size_t total = (size_t)n * KP;
  const long long U = (long long)((n + kOzMT - 1) / kOzMT) * nW;
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  G g;
  g.init(tid);
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    double xv[C::CPT], yv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) xv[c] = yv[c] = 0.0;
    if (i < r1) {
      const size_t o = (size_t)i * KP + j0;
      ldv<C::CPT>(P + o, xv);
      ldv<C::CPT>(Qpart + o, yv);
      const int ns = oz_slices(i / kOzMT, nW, nctas, U);
      for (int k = 1; k < ns; ++k) {
        double t[C::CPT];
        ldv<C::CPT>(Qpart + (size_t)k * total + o, t);
#pragma unroll
        for (int c = 0; c < C::CPT; ++c) yv[c] += t[c];
      }
      stv<C::CPT>(Q + o, yv);
    }
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) {
      Xs[rl * KP + j0 + c] = xv[c];
      Ys[rl * KP + j0 + c] = yv[c];
    }
    __syncthreads();
    g.accumulate(Xs, Ys, min(C::ROWS, r1 - base));
    __syncthreads();
  }
  g.finish(red, part + (size_t)blockIdx.x * pstride);
  if (blockIdx.x == 0 && tid < KP) emaxP[tid] = 0;
}

// ------------------------------------------------------------------------------------ launchers

size_t oz_a_tiles_bytes(int n) {
  const size_t nM = (n + kOzMT - 1) / kOzMT, nK = (n + kOzKC - 1) / kOzKC;
  return nM * nK * kOzDigits * kATileBytes;
}
size_t oz_p_chunks_bytes(int n, int kp) {
  const int kpt = kp < 16 ? 16 : kp;
  const size_t nK = (n + kOzKC - 1) / kOzKC;
  return nK * (size_t)kOzDigits * kpt * kOzKC * 2;
}
namespace {
// The work split of k_dense_tc for n rows on `sms` SMs: at most one CTA per SM and per window;
// windows of two chunks unless that leaves SMs idle. When the row tiles fit on the SMs, the CTA
// count is the largest multiple of the tile count, so that every CTA works on one tile: the
// product is bound by HBM reads, and at n = 4096 (32 tiles) 128 CTAs beat 152 by 8 %.
struct OzSplit {
  int nM, nK, wl, nW, G;
  long long U;
  OzSplit(int n, int sms) {
    nM = (n + kOzMT - 1) / kOzMT;
    nK = (n + kOzKC - 1) / kOzKC;
    wl = (long long)nM * ((nK + kOzWin - 1) / kOzWin) >= sms ? kOzWin : 1;
    nW = (nK + wl - 1) / wl;
    U = (long long)nM * nW;
    G = (int)(U < sms ? U : sms);
    if (nM <= G) G = nM * (G / nM);
  }
};
}  // namespace

// Slices of Qpart the split needs: the most CTAs that share one row tile.
int oz_ksplit(int n, int sms) {
  const OzSplit sp(n, sms > 0 ? sms : 1);
  int m = 1;
  for (int mt = 0; mt < sp.nM; ++mt) m = max(m, oz_slices(mt, sp.nW, sp.G, sp.U));
  return m;
}

void oz_prepare_a(cudaStream_t s, int n, const double* A, int* emaxA, uint8_t* Atiles) {
  cudaMemsetAsync(Atiles, 0, oz_a_tiles_bytes(n), s);
  k_oz_rowexp<<<(n * 32 + 255) / 256, 256, 0, s>>>(n, A, emaxA);
  const int nK = (n + kOzKC - 1) / kOzKC;
  k_oz_slice_a<<<4096, 256, 0, s>>>(n, nK, A, emaxA, reinterpret_cast<uint16_t*>(Atiles));
}

template <int KP, int KPT>
static void oz_product_kp(cudaStream_t s, int n, int sms, const uint8_t* Atiles, const int* emaxA, const double* P,
                          uint8_t* Pchunks, int* emaxP, double* Qpart, double* Q, int* err, const SolveState* st,
                          double* part, int pstride, int nb, int exp_ready) {
  using C = OzCfg<KPT>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dense_tc<KPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
    attr = true;
  }
  const OzSplit sp(n, sms > 0 ? sms : 1);
  const int g = (int)(((size_t)n * KP + 255) / 256);
  if (!exp_ready) {
    cudaMemsetAsync(emaxP, 0, sizeof(int) * KP, s);
    k_oz_colexp<KP><<<g < 1024 ? g : 1024, 256, 0, s>>>(n, P, emaxP, st);
  }
  k_oz_slice_p<KP, KPT><<<g < 4096 ? g : 4096, 256, 0, s>>>(n, P, emaxP, reinterpret_cast<uint16_t*>(Pchunks), st);
  k_dense_tc<KPT><<<sp.G, kOzTcThreads, C::kSmem, s>>>(n, KP, sp.nK, sp.wl, sp.nW, Atiles, emaxA, Pchunks, emaxP,
                                                       Qpart, err, st, 0);
  if (part != nullptr) k_oz_sum_gram<KP><<<nb, kThreads, 0, s>>>(n, sp.nW, Qpart, P, Q, emaxP, part, pstride, st, sp.G);
  else k_oz_sum<KP><<<g < 4096 ? g : 4096, 256, 0, s>>>(n, sp.nW, Qpart, Q, emaxP, st, sp.G);
}

template <int KPT>
static void oz_mma_kp(cudaStream_t s, int n, int KP, int sms, const uint8_t* Atiles, const int* emaxA,
                      const uint8_t* Pchunks, const int* emaxP, double* Qpart) {
  using C = OzCfg<KPT>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dense_tc<KPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
    attr = true;
  }
  const OzSplit sp(n, sms > 0 ? sms : 1);
  k_dense_tc<KPT><<<sp.G, kOzTcThreads, C::kSmem, s>>>(n, KP, sp.nK, sp.wl, sp.nW, Atiles, emaxA, Pchunks, emaxP,
                                                       Qpart, nullptr, nullptr, 0);
}

void oz_mma(cudaStream_t s, int n, int kp, int sms, const uint8_t* Atiles, const int* emaxA, const uint8_t* Pchunks,
            const int* emaxP, double* Qpart) {
  if (kp >= 32) oz_mma_kp<32>(s, n, kp, sms, Atiles, emaxA, Pchunks, emaxP, Qpart);
  else oz_mma_kp<16>(s, n, kp, sms, Atiles, emaxA, Pchunks, emaxP, Qpart);
}

void oz_product(cudaStream_t s, int n, int kp, int sms, const uint8_t* Atiles, const int* emaxA, const double* P,
                uint8_t* Pchunks, int* emaxP, double* Qpart, double* Q, int* err, const SolveState* st, double* part,
                int pstride, int nb, int exp_ready) {
#define OZ_ARGS s, n, sms, Atiles, emaxA, P, Pchunks, emaxP, Qpart, Q, err, st, part, pstride, nb, exp_ready
  switch (kp) {
    case 1: oz_product_kp<1, 16>(OZ_ARGS); break;
    case 2: oz_product_kp<2, 16>(OZ_ARGS); break;
    case 4: oz_product_kp<4, 16>(OZ_ARGS); break;
    case 8: oz_product_kp<8, 16>(OZ_ARGS); break;
    case 16: oz_product_kp<16, 16>(OZ_ARGS); break;
    default: oz_product_kp<32, 32>(OZ_ARGS); break;
  }
#undef OZ_ARGS
}

}  // namespace mbpcg
