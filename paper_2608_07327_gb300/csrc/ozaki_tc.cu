// FP64-accurate dense product Q = A P on the FP16 tensor cores (tcgen05), by exact splitting
// (Ozaki et al., "Error-free transformations of matrix multiplication by using fast routines of
// matrix multiplication and its applications", Numer. Algorithms 2012).
//
// Splitting. Each row i of A (A is symmetric, so row i = column i) is scaled by 2^-F_i, F_i the
// largest binary exponent in the row, and the magnitude of every entry is written as 8 base-128
// digits taken straight from its 53-bit significand (integer shifts; rounded to nearest below 2^-56
// of the row scale). Columns of P are split the same way with their own scales G_j. A digit is an
// integer in [-127, 127], exact in FP16. With level L = t + u of the digit pair (a^t, b^u),
//     (A P)_ij = 2^(F_i + G_j) * sum_L 2^(-7L - 14) * S_L,   S_L = sum_{t+u=L} sum_l a^t_il b^u_lj,
// and levels 0..8 are kept (43 of the 64 pairs; level 8 weighs 2^-70 of the scales per term).
// Dropping level 8 as well -- the first form of this product -- left an error of about 1.7e-14
// ||A P|| on the benchmark system, eight times an FP64 product's, and cost the solver 6 % more
// iterations than the FP64 oracle; with it the error is about 6e-16 ||A P|| (measured on an
// emulation of the split against an 80-bit product), below an FP64 product's.
//
// Exactness. A product of two digits is < 2^14, so a level-L sum over a window of 128 values of l
// is at most (L + 1) * 127^2 * 128 < 2^24 for L <= 4 (and 7 * 127^2 * 128 < 2^24 for L = 8): the
// FP32 accumulator of the tensor core holds it exactly. Levels 0..4 are therefore drained from
// TMEM every 128 values of l and combined in int64 (exact); levels 5..8 are carried in FP32
// (their rounding is below 2^-70 of the scale per window).
//
// Data movement. The digits of A are made once per matrix and stored as bytes (digit + 128), 8 bytes
// per entry of A -- as many as A itself in FP64 -- in blocks of 128 rows x 16 values of l (16 KB)
// that one 1-D TMA bulk copy moves into shared memory. Converter warps turn each block into the
// FP16 operand of the tensor cores and write it to tensor memory (tcgen05.st), where the MMA reads
// A from (the A-in-TMEM form of tcgen05.mma); the digits of P come from shared memory (canonical
// K-major tiles, 8*KPT x 64 per chunk of l, made by k_oz_slice_p every product). The MMA for digit
// t of A uses all needed digits of P at once (N = KPT * (9 - t), or 8 KPT for t = 0), writing
// levels t..min(t + 7, 8) of the accumulator. Producer, converters, MMA issuer and drain run in
// separate warps; every wait is bounded.
#include <cuda_fp16.h>

#include <type_traits>

#include "int_to_fp64.cuh"
#include "kernels.h"
#include "ozaki_digits.cuh"
#include "tcgen05.cuh"

namespace mbpcg {

namespace {

constexpr int kOzMT = 128;                             // rows per M tile (= TMEM lanes)
constexpr int kOzKC = 64;                              // reduction index per chunk (P digits)
constexpr int kOzWin = 2;                              // chunks per exact window (128 values of l)
constexpr int kOzSetK = 16;                            // reduction index per block of A digits (one MMA K step)
constexpr int kOzSetsPerChunk = kOzKC / kOzSetK;
constexpr uint32_t kASetBytes = kOzMT * kOzSetK * kOzDigits;  // 16 KB: 128 rows x 16 l x 8 digit bytes
constexpr int kOzAStages = 6;                          // A blocks in flight (shared memory)
constexpr int kOzPBufs = 4;                            // P digit chunks in flight
constexpr uint32_t kAColsPerSet = kOzDigits * kOzSetK / 2;  // TMEM columns of one converted block (64)
constexpr int kOzABufs = 3;  // converted A blocks in TMEM: a conversion has two MMA steps of slack
constexpr int kOzLevels = 9;                           // digit-pair levels t + u = 0..8 kept

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

// Byte offset of digit t of (row r, value k of l) inside a block of A digits: row r owns 128
// bytes, 16-byte slot t of them holding k = 0..15 of digit t; the slot is stored at position
// t ^ (r % 8), so that the 32 rows a converter warp reads at once fall on different shared-memory
// banks.
__host__ __device__ inline uint32_t oz_a8_offset(int r, int k, int t) {
  return (uint32_t)(r * 128 + ((t ^ (r & 7)) << 4) + k);
}

// Digits of A as bytes (digit + 128) into blocks [mtile][set][row][256 bytes] (see oz_a8_offset).
// The blocks are preset to 128 (digit 0) so that rows and values of l past n contribute nothing.
__global__ void k_oz_slice_a8(int n, int nS, const double* __restrict__ A, const int* __restrict__ emax,
                              uint8_t* __restrict__ blocks) {
  const size_t total = (size_t)n * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / n), l = (int)(q % n);
    int d[kOzDigits];
    ozaki_digits(A[q], emax[i], d);  // A[i*n + l] = row i (symmetric)
    uint8_t* blk = blocks + ((size_t)(i / kOzMT) * nS + l / kOzSetK) * kASetBytes;
#pragma unroll
    for (int t = 0; t < kOzDigits; ++t) blk[oz_a8_offset(i % kOzMT, l % kOzSetK, t)] = (uint8_t)(d[t] + 128);
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

// Digits of P into chunks [kchunk] of (8 * KPT) x 64 fp16, row index KPT * t + j (canonical
// K-major layout, so digit t of every column j is one contiguous N-range). One thread per value.
// (Forms with 16-byte stores -- a thread taking 8 consecutive values of a column, or digit t of
// them -- were slower: 8.4 against 5.5 us at n = 4096, KP = 32.)
template <int KP, int KPT>
__global__ void k_oz_slice_p(int n, const double* __restrict__ P, const int* __restrict__ emaxP,
                             uint16_t* __restrict__ chunks, const SolveState* __restrict__ st) {
  constexpr uint32_t kChunkElems = kOzDigits * KPT * kOzKC;
  const size_t total = (size_t)n * KP, stride = (size_t)gridDim.x * blockDim.x;
  size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  // the first value and its column scale are loaded with the solve state (a skipped launch discards
  // them), so the two L2 round trips overlap
  double pv = q < total ? P[q] : 0.0;
  int ev = q < total ? emaxP[q % KP] : 0;
  if (st != nullptr && st->done) return;
  for (; q < total; q += stride) {
    const int l = (int)(q / KP), j = (int)(q % KP);
    if (q >= stride) {  // (not the thread's first value)
      pv = P[q];
      ev = emaxP[j];
    }
    int d[kOzDigits];
    ozaki_digits(pv, ev, d);
    uint16_t* ch = chunks + (size_t)(l / kOzKC) * kChunkElems;
#pragma unroll
    for (int t = 0; t < kOzDigits; t += 2) {
      const uint32_t h2 = oz_f16_pair_of_ints(d[t], d[t + 1]);
      ch[umma_kmajor_offset(KPT * t + j, l % kOzKC, kOzKC) / 2] = (uint16_t)(h2 & 0xFFFFu);
      ch[umma_kmajor_offset(KPT * (t + 1) + j, l % kOzKC, kOzKC) / 2] = (uint16_t)(h2 >> 16);
    }
  }
}

template <int KPT>
struct OzCfg {
  static constexpr uint32_t kPChunkBytes = kOzDigits * KPT * kOzKC * 2;
  static constexpr uint32_t kAccCols = kOzLevels * KPT;   // the accumulator: 9 levels x KPT columns
  static constexpr uint32_t kTmemCols = 512;              // accumulator + kOzABufs converted A blocks
  static_assert(kAccCols + kOzABufs * kAColsPerSet <= kTmemCols, "tensor memory of one CTA");
  static constexpr size_t kBarBytes = 1024;  // barriers + TMEM slot, keeps the blocks 1024-aligned
  static constexpr size_t kSmem = kBarBytes + (size_t)kOzAStages * kASetBytes + (size_t)kOzPBufs * kPChunkBytes;
};
static_assert(OzCfg<32>::kSmem <= 227 * 1024, "shared memory of one CTA");

constexpr int kOzDrainGroups = 4;    // drain warps per TMEM lane quarter (each a quarter of the columns)
constexpr int kOzDrainWarps = 4 * kOzDrainGroups;  // warps 0..15: lane quarter w % 4, columns group w / 4
constexpr int kOzConvWarps = 4;      // warps 16..19: lane quarter w % 4, A digits -> FP16 in TMEM
constexpr int kOzProducerWarp = 20;  // TMA issue of the A digit blocks
constexpr int kOzMmaWarp = 21;       // MMA issue
constexpr int kOzPProducerWarp = 22; // TMA issue of the P digit chunks (its own thread, so that a
                                     // chunk is requested as soon as a buffer is free)
constexpr int kOzTcThreads = 32 * 23;

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

// Two digit bytes (digit + 128) of w, bytes j and j + 1, -> an FP16 pair (the lower k in the low
// half): each byte is placed under the exponent of 1024 (an FP16 1024 + u, exact for u < 1024) and
// 1024 + 128 is subtracted from both halves at once (exact: small integers).
__device__ __forceinline__ uint32_t oz_f16_pair(uint32_t w, uint32_t sel) {
  const uint32_t b = __byte_perm(w, 0x64646464u, sel);  // halves 0x64uu: 1024 + u
  const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&b), __half2half2(__ushort_as_half(0x6480)));
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Raw partial sums of one slice of the product: int64 levels 0..4 (units 2^-42 of the row and
// column scales) and FP32 levels 5..8 (units 2^-49), [slice][column][row] each, so that the 32
// rows of a drain warp store 32 consecutive values; the split sum turns them into FP64 once per
// output (FP64 instructions are scarce on this GPU: converting in the MMA kernel held its SMs'
// FP64 units for the last ~5 us of the product).
struct OzPart {
  long long* qi;
  float* qf;      // levels 5..8 carried in FP32 (the default rounding)
  long long* ql;  // levels 5..8 as exact integers in units of 2^-70 (rounded once: same storage)
};
__host__ __device__ inline OzPart oz_part(double* Qpart, int n, int kp, int ksplit) {
  OzPart p;
  p.qi = reinterpret_cast<long long*>(Qpart);
  p.ql = p.qi + (size_t)ksplit * n * kp;
  p.qf = reinterpret_cast<float*>(p.ql);
  return p;
}

// Raw partials of (A P)_ij over the K range of slice k of row i's tile (OzPart layout), for j < KP.
// Warp-specialised (23 warps), all waits bounded:
//   producers (one thread each): A digit blocks (16 KB: 128 rows x 16 values of l x 8 digit bytes)
//     into kOzAStages shared stages, and P digit chunks (64 values of l) into kOzPBufs buffers, by
//     1-D TMA bulk copies on mbarriers;
//   converters (4 warps, thread = row): a block's bytes -> FP16 digits in one of kOzABufs TMEM A
//     buffers (tcgen05.st);
//   MMA issuer (one thread): per block and digit t of A, one tcgen05.mma (K = 16) with A from TMEM
//     and all needed digits of P from shared memory into levels t..min(t + 7, 8) of the accumulator;
//   drain (16 warps, thread = row, a quarter of the columns each): after each window of 128 values
//     of l, the 9 levels are copied out of TMEM in two rounds and the accumulator is released to
//     the next window (one accumulator: the tensor memory also holds the A buffers); levels 0..4
//     are added exactly into int64, levels 5..8 in FP32 (or exactly into int64 with ONCE).
template <int KPT, bool ONCE>
__global__ void __launch_bounds__(kOzTcThreads, 1)
k_dense_tc(int n, int KP, int nK, int wl, int nW, const uint8_t* __restrict__ Ablocks, const int* __restrict__ emaxA,
           const uint8_t* __restrict__ Pchunks, int* __restrict__ emaxP, double* __restrict__ Qpart, int ksplit,
           int* __restrict__ err, const SolveState* __restrict__ st, int dir) {
  using C = OzCfg<KPT>;
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(1024) uint8_t osm[];
  uint64_t* sfull = reinterpret_cast<uint64_t*>(osm);  // [kOzAStages] A block landed
  uint64_t* sempty = sfull + kOzAStages;               // [kOzAStages] A block converted (stage free)
  uint64_t* pfull = sempty + kOzAStages;               // [kOzPBufs] P chunk landed
  uint64_t* pempty = pfull + kOzPBufs;                 // [kOzPBufs] P chunk used by its MMAs
  uint64_t* afull = pempty + kOzPBufs;                 // [kOzABufs] TMEM A buffer written
  uint64_t* aempty = afull + kOzABufs;                 // [kOzABufs] TMEM A buffer read by its MMAs
  uint64_t* accf = aempty + kOzABufs;                  // accumulator ready for draining
  uint64_t* acce = accf + 1;                           // accumulator drained
  uint64_t* fin = acce + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  uint8_t* As = osm + C::kBarBytes;
  uint8_t* Ps = As + (size_t)kOzAStages * kASetBytes;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, g = blockIdx.x;
  const int nS = nK * kOzSetsPerChunk;
  const long long U = (long long)((n + kOzMT - 1) / kOzMT) * nW;
  const long long f0 = U * g / G;
  const int nwin = (int)(U * (g + 1) / G - f0);
  // Window order: on odd iterations of a solve each CTA walks its range backwards, so that it starts
  // on the digits the previous product read last, the ones most likely still in L2 (A is read every
  // iteration).
  if (st != nullptr) dir ^= st->it & 1;

  if (tid == 0) {
    for (int q = 0; q < kOzAStages; ++q) {
      mbar_init(&sfull[q], 1);
      mbar_init(&sempty[q], kOzConvWarps);
    }
    for (int q = 0; q < kOzPBufs; ++q) {
      mbar_init(&pfull[q], 1);
      mbar_init(&pempty[q], 1);
    }
    for (int q = 0; q < kOzABufs; ++q) {
      mbar_init(&afull[q], kOzConvWarps);
      mbar_init(&aempty[q], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, kOzDrainWarps);  // every drain warp arrives once per window
    mbar_init(fin, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, C::kTmemCols);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t abuf0 = tmem + C::kAccCols;
  // the split sum scales with this copy of the column exponents of P (it clears the live ones)
  if (g == 0 && tid < KP) emaxP[kMaxKP + tid] = emaxP[tid];
  int issued_a = 0, issued_p = 0;  // copies issued (producer thread only)

  if (warp == kOzProducerWarp) {
    if (lane == 0) {
      const uint64_t pol_stream = l2_policy_evict_first();  // A digits: 8 B per entry of A, read once
      bool ok = true;
      int j = 0;  // A blocks of this CTA so far
      for (int w = 0; w < nwin && ok; ++w) {
        const long long f = f0 + (dir ? nwin - 1 - w : w);
        const int mt = (int)(f / nW), c0 = (int)(f % nW) * wl, c1 = min(nK, c0 + wl);
        for (int c = c0; c < c1 && ok; ++c) {
          for (int u = 0; u < kOzSetsPerChunk && ok; ++u, ++j) {
            const int q = j % kOzAStages;
            if (j >= kOzAStages) ok = mbar_wait_bounded(&sempty[q], (uint32_t)((j / kOzAStages - 1) & 1));
            if (!ok) break;
            mbar_arrive_expect_tx(&sfull[q], kASetBytes);
            tma_load_1d_hint(As + (size_t)q * kASetBytes,
                             Ablocks + ((size_t)mt * nS + (size_t)c * kOzSetsPerChunk + u) * kASetBytes, kASetBytes,
                             &sfull[q], pol_stream);
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
  } else if (warp == kOzPProducerWarp) {
    if (lane == 0) {
      bool ok = true;
      int cc = 0;  // chunks of this CTA so far
      for (int w = 0; w < nwin && ok; ++w) {
        const long long f = f0 + (dir ? nwin - 1 - w : w);
        const int c0 = (int)(f % nW) * wl, c1 = min(nK, c0 + wl);
        for (int c = c0; c < c1 && ok; ++c, ++cc) {
          const int b = cc % kOzPBufs;
          if (cc >= kOzPBufs) ok = mbar_wait_bounded(&pempty[b], (uint32_t)((cc / kOzPBufs - 1) & 1));
          if (!ok) break;
          mbar_arrive_expect_tx(&pfull[b], C::kPChunkBytes);
          tma_load_1d(Ps + (size_t)b * C::kPChunkBytes, Pchunks + (size_t)c * C::kPChunkBytes, C::kPChunkBytes,
                      &pfull[b]);
          issued_p = cc + 1;
          if (*abort_flag) ok = false;
        }
      }
      if (!ok) {
        *abort_flag = 1;
        if (err != nullptr) atomicExch(err, 1);
      }
    }
  } else if (warp >= kOzDrainWarps && warp < kOzDrainWarps + kOzConvWarps) {
    // converters: thread = row 32 (warp % 4) + lane of the M tile (warps 16..19: quarters 0..3)
    const int r = 32 * (warp & 3) + lane;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    bool ok = true;
    int j = 0;
    for (int w = 0; w < nwin && ok; ++w) {
      const long long f = f0 + (dir ? nwin - 1 - w : w);
      const int c0 = (int)(f % nW) * wl, nsets = (min(nK, c0 + wl) - c0) * kOzSetsPerChunk;
      for (int u = 0; u < nsets && ok; ++u, ++j) {
        const int q = j % kOzAStages, ab = j % kOzABufs;
        ok = mbar_wait_bounded(&sfull[q], (uint32_t)((j / kOzAStages) & 1));
        if (ok && j >= kOzABufs) ok = mbar_wait_bounded(&aempty[ab], (uint32_t)((j / kOzABufs - 1) & 1));
        ok = __all_sync(0xffffffffu, ok && !*abort_flag);  // tcgen05.st needs the whole warp
        if (!ok) break;
        tc_fence_after_sync();
        const uint8_t* row = As + (size_t)q * kASetBytes + r * 128;
        const uint32_t dst = abuf0 + (uint32_t)ab * kAColsPerSet + lane_off;
#pragma unroll
        for (int t = 0; t < kOzDigits; ++t) {
          const uint4 w4 = *reinterpret_cast<const uint4*>(row + ((t ^ (r & 7)) << 4));
          uint32_t v[8];
          const uint32_t wd[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
          for (int q2 = 0; q2 < 4; ++q2) {
            v[2 * q2] = oz_f16_pair(wd[q2], 0x4140u);      // bytes 0, 1
            v[2 * q2 + 1] = oz_f16_pair(wd[q2], 0x4342u);  // bytes 2, 3
          }
          tmem_st8(dst + (uint32_t)(8 * t), v);  // digit t: columns 8 t .. 8 t + 7 (k pairs 0..7)
        }
        tmem_wait_st();
        tc_fence_before_sync();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&afull[ab]);
          mbar_arrive(&sempty[q]);
        }
      }
    }
    if (!ok) {
      *abort_flag = 1;
      if (err != nullptr) atomicExch(err, 1);
    }
  } else if (warp == kOzMmaWarp) {
    if (lane == 0) {
      bool ok = true;
      int cc = 0, j = 0;
      for (int w = 0; w < nwin && ok; ++w) {
        if (w >= 1) ok = mbar_wait_bounded(acce, (uint32_t)((w - 1) & 1));  // the previous window drained
        tc_fence_after_sync();
        const long long f = f0 + (dir ? nwin - 1 - w : w);
        const int c0 = (int)(f % nW) * wl, nc = min(nK, c0 + wl) - c0, cc0 = cc;
        for (; cc < cc0 + nc && ok; ++cc) {
          const int b = cc % kOzPBufs;
          ok = mbar_wait_bounded(&pfull[b], (uint32_t)((cc / kOzPBufs) & 1));
          const uint32_t b_base = smem_addr(Ps + (size_t)b * C::kPChunkBytes);
          for (int u = 0; u < kOzSetsPerChunk && ok; ++u, ++j) {
            const int ab = j % kOzABufs;
            ok = mbar_wait_bounded(&afull[ab], (uint32_t)((j / kOzABufs) & 1));
            if (!ok) break;
            tc_fence_after_sync();
            const uint32_t a_base = abuf0 + (uint32_t)ab * kAColsPerSet;
            const uint32_t bk = b_base + 256u * u;  // K step u of the P chunk
            const uint64_t bdesc = umma_smem_desc(bk, 128, 1024);
            // digit t of A with digits 0 .. min(7, 8 - t) of P: levels t .. min(t + 7, 8). The first
            // K step of a window overwrites every level: digit 1 (levels 1..8) first, then digit 0
            // alone into level 0, then digit 0 accumulating into levels 1..7 (digits 1..7 of P, rows
            // KPT.. of the chunk: KPT/8 core-matrix groups further).
            const bool first = (cc == cc0 && u == 0);
#pragma unroll
            for (int t = 0; t < kOzDigits; ++t) {
              const int nu = (t == 0) ? kOzDigits : kOzLevels - t;
              if (first && t == 0) {
                umma_tmem_a(tmem + (uint32_t)KPT, a_base + 8u, bdesc, umma_idesc_f16_f32(kOzMT, KPT * (kOzLevels - 1)),
                            0u);
                umma_tmem_a(tmem, a_base, bdesc, umma_idesc_f16_f32(kOzMT, KPT), 0u);
                umma_tmem_a(tmem + (uint32_t)KPT, a_base, umma_smem_desc(bk + 1024u * (KPT / 8), 128, 1024),
                            umma_idesc_f16_f32(kOzMT, KPT * (kOzDigits - 1)), 1u);
              } else if (!(first && t == 1)) {
                umma_tmem_a(tmem + (uint32_t)(KPT * t), a_base + (uint32_t)(8 * t), bdesc,
                            umma_idesc_f16_f32(kOzMT, KPT * nu), 1u);
              }
            }
            umma_commit(&aempty[ab]);
          }
          if (ok) umma_commit(&pempty[b]);
          if (*abort_flag) ok = false;
        }
        if (!ok) *abort_flag = 1;  // before the commit, so the drain warps see it
        umma_commit(accf);
      }
      if (!ok) {
        *abort_flag = 1;
        if (err != nullptr) atomicExch(err, 1);
      }
      umma_commit(fin);
      mbar_wait_bounded(fin, 0);
    }
  } else if (warp < kOzDrainWarps) {
    // drain warps 0..7: warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of this M tile) and the
    // column half w / 4 (DC = KPT / 2 columns) of every level
    constexpr int DC = KPT / kOzDrainGroups;
    const int half = warp >> 2;  // column group of this warp
    long long acc_i[DC];
    using Lo = typename std::conditional<ONCE, long long, float>::type;
    Lo acc_f[DC];
#pragma unroll
    for (int jj = 0; jj < DC; ++jj) {
      acc_i[jj] = 0;
      acc_f[jj] = 0;
    }
    bool ok = true;
    for (int w = 0; w < nwin; ++w) {
      if (!mbar_wait_bounded(accf, (uint32_t)(w & 1))) ok = false;
      tc_fence_after_sync();
      ok = __all_sync(0xffffffffu, ok && !*abort_flag);  // tcgen05.ld needs the whole warp
      if (!ok) break;
      const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(DC * half);
      // two rounds (levels 5..8, then 0..4): the loads of a round are in flight together (one wait
      // each); the accumulator is released as soon as the second round is in registers. Levels
      // 5..8 go first because their adds are FP32 FMAs; the 40 integer conversions of levels 0..4
      // (a slow unit: 16 per clock per SM) then run after the release, beside the next MMAs.
#pragma unroll
      for (int rd = 0; rd < 2; ++rd) {
        constexpr int kR = 5;
        const int L0 = rd == 0 ? kR : 0, nl = rd == 0 ? kOzLevels - kR : kR;
        uint32_t rr[kR][DC];
#pragma unroll
        for (int q = 0; q < kR; ++q) {
          if (q < nl) {
            if constexpr (DC == 16) tmem_ld16(lane_base + (uint32_t)(KPT * (L0 + q)), rr[q]);
            else if constexpr (DC == 8) tmem_ld8(lane_base + (uint32_t)(KPT * (L0 + q)), rr[q]);
            else tmem_ld4(lane_base + (uint32_t)(KPT * (L0 + q)), rr[q]);
          }
        }
        tmem_wait_ld();
        if (rd == 1) {
          tc_fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(acce);
        }
#pragma unroll
        for (int q = 0; q < kR; ++q) {
          const int L = L0 + q;
          if (L < 5) {
            const int sh = 7 * (4 - L);
#pragma unroll
            for (int jj = 0; jj < DC; ++jj) acc_i[jj] += (long long)__float2int_rn(__uint_as_float(rr[q][jj])) << sh;
          } else if (L < kOzLevels) {
            if constexpr (ONCE) {  // exact: a window's level sum is an integer below 2^24
              const int sh = 7 * (kOzLevels - 1 - L);
#pragma unroll
              for (int jj = 0; jj < DC; ++jj) acc_f[jj] += (long long)__float2int_rn(__uint_as_float(rr[q][jj])) << sh;
            } else {
              const float sc = (L == 5) ? 1.f : (L == 6) ? 0x1p-7f : (L == 7) ? 0x1p-14f : 0x1p-21f;
#pragma unroll
              for (int jj = 0; jj < DC; ++jj) acc_f[jj] = fmaf(__uint_as_float(rr[q][jj]), sc, acc_f[jj]);
            }
          }
        }
      }
      const long long f = f0 + (dir ? nwin - 1 - w : w);
      if (w == nwin - 1 || (dir ? f % nW == 0 : (f + 1) % nW == 0)) {  // end of a segment: its tile's rows
        const int mt = (int)(f / nW), row = mt * kOzMT + 32 * (warp & 3) + lane;
        const int slice = g - oz_cta_of((long long)mt * nW, G, U);
        if (row < n) {
          const OzPart qp = oz_part(Qpart, n, KP, ksplit);
#pragma unroll
          for (int jj = 0; jj < DC; ++jj) {
            const int j = DC * half + jj;
            if (j < KP) {
              const size_t o = ((size_t)slice * KP + j) * n + row;
              qp.qi[o] = acc_i[jj];
              if constexpr (ONCE) qp.ql[o] = acc_f[jj];
              else qp.qf[o] = acc_f[jj];
            }
          }
        }
#pragma unroll
        for (int jj = 0; jj < DC; ++jj) {
          acc_i[jj] = 0;
          acc_f[jj] = 0;
        }
      }
    }
    if (!ok || *abort_flag) {
      *abort_flag = 1;
      if (err != nullptr) atomicExch(err, 1);
    }
  }
  __syncthreads();
  // after an abort, let the copies still in flight land before the shared memory is released
  // (bounded waits); only the last issue into each stage or buffer can still be pending
  if (*abort_flag && tid == 32 * kOzProducerWarp)
    for (int j = max(0, issued_a - kOzAStages); j < issued_a; ++j)
      mbar_wait_bounded(&sfull[j % kOzAStages], (uint32_t)((j / kOzAStages) & 1));
  if (*abort_flag && tid == 32 * kOzPProducerWarp)
    for (int cc = max(0, issued_p - kOzPBufs); cc < issued_p; ++cc)
      mbar_wait_bounded(&pfull[cc % kOzPBufs], (uint32_t)((cc / kOzPBufs) & 1));
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem, C::kTmemCols);
}

// An FP32 value as FP64 (exact) with integer operations, zeros as +0 (the sums below start from +0,
// so the sign of a zero term never shows); subnormal, infinite and NaN inputs take the conversion
// instruction, which on this GPU runs on the FP64 pipe.
__device__ __forceinline__ double oz_f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  if ((b << 1) == 0) return 0.0;
  if (e == 0 || e == 0xFFu) return (double)f;
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                          ((unsigned long long)(e + 896u) << 52) |
                                          ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// Sums of the raw partials of output o over the ns slices of its tile (slice stride `stride`
// entries): the int64 parts exactly; the levels 5..8 parts exactly too when they are integers
// (ONCE), else FP32 values summed in FP64 in slice order. The first kOzSliceBatch slices are loaded
// at once, as many as the buffer holds (ksplit) whatever ns is, so that the loads need not wait for
// ns (two 64-bit divisions): slices past ns are read and left out of the sums. Returns the product
// before its scale. The conversions to FP64 and the scalings by powers of two are integer
// operations (int_to_fp64.cuh): the FP64 pipe keeps only the adds of the FP32 parts and the final
// multiply-add.
constexpr int kOzSliceBatch = 8;
template <bool ONCE>
__device__ __forceinline__ double oz_slice_value(const OzPart& qp, size_t o, size_t stride, int ns, int ksplit) {
  long long vi[kOzSliceBatch];
  typename std::conditional<ONCE, long long, float>::type vf[kOzSliceBatch];
#pragma unroll
  for (int k = 0; k < kOzSliceBatch; ++k) {
    vi[k] = 0;
    vf[k] = 0;
    if (k < ksplit) {
      vi[k] = qp.qi[(size_t)k * stride + o];
      if constexpr (ONCE) vf[k] = qp.ql[(size_t)k * stride + o];
      else vf[k] = qp.qf[(size_t)k * stride + o];
    }
  }
  long long si = 0;
  typename std::conditional<ONCE, long long, double>::type sf = 0;
#pragma unroll
  for (int k = 0; k < kOzSliceBatch; ++k) {
    if (k >= ns) break;
    si += vi[k];
    if constexpr (ONCE) sf += vf[k];
    else if (k == 0) sf = oz_f32_to_f64(vf[0]);  // = 0 + vf[0]
    else sf += oz_f32_to_f64(vf[k]);
  }
  for (int k = kOzSliceBatch; k < ns; ++k) {
    si += qp.qi[(size_t)k * stride + o];
    if constexpr (ONCE) sf += qp.ql[(size_t)k * stride + o];
    else sf += oz_f32_to_f64(qp.qf[(size_t)k * stride + o]);
  }
  // levels 0..4 in units of 2^-42, levels 5..8 in units of 2^-49 (FP32 carry) or 2^-70 (exact);
  // si 2^-42 is a normal number or zero, so the scaled conversion never leaves the normal range
  bool normal;
  const double hi = ll_to_double_scaled_rn(si, -42, normal);
  if constexpr (ONCE) return fma(ll_to_double_rn(sf), 0x1p-70, hi);
  else return fma(sf, 0x1p-49, hi);
}

// v 2^e: an integer add to the exponent field when v and the result are normal numbers (the same
// bits as the product), else a product by a power of two (exact wherever ldexp is), else ldexp.
__device__ __forceinline__ double oz_scale(double v, int e) {
  const long long b = __double_as_longlong(v);
  const int ev = (int)((b >> 52) & 0x7FF);
  if (ev != 0 && ev + e >= 1 && ev + e <= 2046) return __longlong_as_double(b + (long long)e * (1LL << 52));
  if (e >= -1022 && e <= 1023) return v * __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(v, e);
}

// Q[i][j] = the product from the slices of row i's tile (in slice order). Block 0 then clears the
// column exponents of P for the next product (they are rebuilt by the W/P update, which writes
// P); the scaling reads the copy the MMA kernel made of them.
template <int KP, bool ONCE>
__global__ void k_oz_sum(int n, int nW, const double* __restrict__ Qpart, double* __restrict__ Q,
                         const int* __restrict__ emaxA, int* __restrict__ emaxP, const SolveState* __restrict__ st,
                         int nctas, int ksplit) {
  if (st != nullptr && st->done) return;
  const OzPart qp = oz_part(const_cast<double*>(Qpart), n, KP, ksplit);
  const size_t total = (size_t)n * KP;
  const long long U = (long long)((n + kOzMT - 1) / kOzMT) * nW;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / n), i = (int)(q % n);  // consecutive threads: consecutive rows of column j
    const int ns = oz_slices(i / kOzMT, nW, nctas, U);
    Q[(size_t)i * KP + j] =
        oz_scale(oz_slice_value<ONCE>(qp, q, total, ns, ksplit), emaxA[i] - 1022 + emaxP[kMaxKP + j] - 1022);
  }
  if (blockIdx.x == 0 && threadIdx.x < KP) emaxP[threadIdx.x] = 0;
}

// The same split sum fused with the CTA partials of the upper triangle of P^T Q (the Gram of the
// Xi step of Algorithm 1), one pass over balanced row ranges (partials as k_gram writes them).
template <int KP, bool ONCE>
__global__ void __launch_bounds__(kThreads)
k_oz_sum_gram(int n, int nW, const double* __restrict__ Qpart, const double* __restrict__ P, double* __restrict__ Q,
              const int* __restrict__ emaxA, int* __restrict__ emaxP, double* __restrict__ part, int pstride,
              const SolveState* __restrict__ st, int nctas, int ksplit) {
  using C = Cfg<KP>;
  using G = GramTile<KP>;
  if (st != nullptr && st->done) return;
  __shared__ __align__(16) double Xs[C::ROWS * KP];
  __shared__ __align__(16) double Ys[C::ROWS * KP];
  __shared__ __align__(16) double red[G::RED];
  const OzPart qp = oz_part(const_cast<double*>(Qpart), n, KP, ksplit);
  const size_t total = (size_t)n * KP;
  const long long U = (long long)((n + kOzMT - 1) / kOzMT) * nW;
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  G g;
  g.init(tid);
  for (int base = r0; base < r1; base += C::ROWS) {
    // the tile's ROWS x KP outputs, thread e -> (row e % ROWS, column e / ROWS): the partials of a
    // column are consecutive in memory
#pragma unroll
    for (int e = tid; e < C::ROWS * KP; e += kThreads) {
      const int rr = e % C::ROWS, j = e / C::ROWS, i = base + rr;
      double y = 0.0;
      if (i < r1) {
        const int ns = oz_slices(i / kOzMT, nW, nctas, U);
        y = oz_scale(oz_slice_value<ONCE>(qp, (size_t)j * n + i, total, ns, ksplit),
                     emaxA[i] - 1022 + emaxP[kMaxKP + j] - 1022);
      }
      Ys[rr * KP + j] = y;
    }
    const int i = base + rl;
    double xv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) xv[c] = 0.0;
    if (i < r1) ldv<C::CPT>(P + (size_t)i * KP + j0, xv);
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) Xs[rl * KP + j0 + c] = xv[c];
    __syncthreads();
    if (i < r1) {
      double yv[C::CPT];
#pragma unroll
      for (int c = 0; c < C::CPT; ++c) yv[c] = Ys[rl * KP + j0 + c];
      stv<C::CPT>(Q + (size_t)i * KP + j0, yv);
    }
    g.accumulate(Xs, Ys, min(C::ROWS, r1 - base));
    __syncthreads();
  }
  g.finish(red, part + (size_t)blockIdx.x * pstride);
  if (blockIdx.x == 0 && tid < KP) emaxP[tid] = 0;
}

// ------------------------------------------------------------------------------------ launchers

size_t oz_a_tiles_bytes(int n) {
  const size_t nM = (n + kOzMT - 1) / kOzMT, nK = (n + kOzKC - 1) / kOzKC;
  return nM * nK * kOzSetsPerChunk * kASetBytes;
}
size_t oz_p_chunks_bytes(int n, int kp) {
  const int kpt = kp < 16 ? 16 : kp;
  const size_t nK = (n + kOzKC - 1) / kOzKC;
  return nK * (size_t)kOzDigits * kpt * kOzKC * 2;
}
namespace {
// The work split of k_dense_tc for n rows on `sms` SMs: one CTA per SM (at most one per window);
// windows of two chunks unless that leaves SMs idle. Every SM takes part: each CTA's time is set
// by its own MMA and drain pipeline rather than by HBM, so more CTAs finish sooner.
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
  cudaMemsetAsync(Atiles, 0x80, oz_a_tiles_bytes(n), s);  // digit 0 everywhere (byte = digit + 128)
  k_oz_rowexp<<<(n * 32 + 255) / 256, 256, 0, s>>>(n, A, emaxA);
  const int nS = (n + kOzKC - 1) / kOzKC * kOzSetsPerChunk;
  k_oz_slice_a8<<<4096, 256, 0, s>>>(n, nS, A, emaxA, Atiles);
}

template <int KP, int KPT, bool ONCE>
static void oz_product_kp(cudaStream_t s, int n, int sms, const uint8_t* Atiles, const int* emaxA, const double* P,
                          uint8_t* Pchunks, int* emaxP, double* Qpart, double* Q, int* err, const SolveState* st,
                          double* part, int pstride, int nb, int exp_ready) {
  using C = OzCfg<KPT>;
  ensure_dynamic_smem(k_dense_tc<KPT, ONCE>, C::kSmem);
  const OzSplit sp(n, sms > 0 ? sms : 1);
  const int g = (int)(((size_t)n * KP + 255) / 256);
  if (!exp_ready) {
    cudaMemsetAsync(emaxP, 0, sizeof(int) * KP, s);
    k_oz_colexp<KP><<<g < 1024 ? g : 1024, 256, 0, s>>>(n, P, emaxP, st);
  }
  k_oz_slice_p<KP, KPT><<<g < 4096 ? g : 4096, 256, 0, s>>>(n, P, emaxP, reinterpret_cast<uint16_t*>(Pchunks), st);
  const int ks = oz_ksplit(n, sms);
  k_dense_tc<KPT, ONCE><<<sp.G, kOzTcThreads, C::kSmem, s>>>(n, KP, sp.nK, sp.wl, sp.nW, Atiles, emaxA, Pchunks,
                                                             emaxP, Qpart, ks, err, st, 0);
  if (part != nullptr)
    k_oz_sum_gram<KP, ONCE><<<nb, kThreads, 0, s>>>(n, sp.nW, Qpart, P, Q, emaxA, emaxP, part, pstride, st, sp.G, ks);
  else k_oz_sum<KP, ONCE><<<g < 4096 ? g : 4096, 256, 0, s>>>(n, sp.nW, Qpart, Q, emaxA, emaxP, st, sp.G, ks);
}

template <int KPT>
static void oz_mma_kp(cudaStream_t s, int n, int KP, int sms, const uint8_t* Atiles, const int* emaxA,
                      const uint8_t* Pchunks, const int* emaxP, double* Qpart) {
  using C = OzCfg<KPT>;
  ensure_dynamic_smem(k_dense_tc<KPT, false>, C::kSmem);
  const OzSplit sp(n, sms > 0 ? sms : 1);
  k_dense_tc<KPT, false><<<sp.G, kOzTcThreads, C::kSmem, s>>>(n, KP, sp.nK, sp.wl, sp.nW, Atiles, emaxA, Pchunks,
                                                              const_cast<int*>(emaxP), Qpart, oz_ksplit(n, sms),
                                                              nullptr, nullptr, 0);
}

void oz_mma(cudaStream_t s, int n, int kp, int sms, const uint8_t* Atiles, const int* emaxA, const uint8_t* Pchunks,
            const int* emaxP, double* Qpart) {
  if (kp >= 32) oz_mma_kp<32>(s, n, kp, sms, Atiles, emaxA, Pchunks, emaxP, Qpart);
  else oz_mma_kp<16>(s, n, kp, sms, Atiles, emaxA, Pchunks, emaxP, Qpart);
}

void oz_product(cudaStream_t s, int n, int kp, int sms, const uint8_t* Atiles, const int* emaxA, const double* P,
                uint8_t* Pchunks, int* emaxP, double* Qpart, double* Q, int* err, const SolveState* st, double* part,
                int pstride, int nb, int exp_ready, int once) {
#define OZ_ARGS s, n, sms, Atiles, emaxA, P, Pchunks, emaxP, Qpart, Q, err, st, part, pstride, nb, exp_ready
#define OZ_CASE(KP, KPT)                                                         \
  if (once) oz_product_kp<KP, KPT, true>(OZ_ARGS);                                \
  else oz_product_kp<KP, KPT, false>(OZ_ARGS);
  switch (kp) {
    case 1: OZ_CASE(1, 16) break;
    case 2: OZ_CASE(2, 16) break;
    case 4: OZ_CASE(4, 16) break;
    case 8: OZ_CASE(8, 16) break;
    case 16: OZ_CASE(16, 16) break;
    default: OZ_CASE(32, 32) break;
  }
#undef OZ_CASE
#undef OZ_ARGS
}

}  // namespace mbpcg
