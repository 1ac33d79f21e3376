// FP32 dense product of the mixed-precision inner solve (MBPCG_MIXED_FP32 on a dense matrix):
// Q = A P, A the FP32 copy of the scaled matrix in tiles (below), P and Q row-major n x KP FP32
// blocks. The product of Algorithm 1 (the Xi step's A P) is the only step that touches A; in
// the mixed inner solve it reads 4 bytes per entry of A instead of the 8 of FP64 or the 16 of the
// tensor-core digits, and runs on the FP32 pipe (the FP64 pipe of this GPU is 64 times slower).
//
// Layout of A. The FP32 copy is stored as tiles of 256 rows x 32 values of l (32 KB, row-major inside
// the tile, zero past n), the tiles of one row tile adjacent: every chunk a CTA reads is one
// contiguous block, so HBM is read sequentially. (Row-major A read 32 values of l at a time takes
// 128 B from each of 256 rows 16 KB apart and ran at 1 TB/s.)
//
// Tiling. A CTA owns 256 rows of Q and a K range; its 8 warps own 32 rows each, a thread an
// RT x CT register tile (rows ty + TY k, columns CT tx + c). A and P chunks of 32 values of l move
// into shared memory with cp.async (3 stages; rows of A padded by 4 floats to spread the banks; P
// zero-filled past n). The K ranges of one row tile are
// the CTAs of a thread-block cluster (up to 8): at the end each CTA puts its partial tile in its
// shared memory and adds, for its share of the rows, the partial tiles of all CTAs of the cluster
// in rank order through distributed shared memory. No partial sums go to HBM and the result does
// not depend on timing. Accumulation is FP32 (error <= n 2^-24 |A||P|, a bound the inner solve's
// tolerance of 1e-5 leaves far behind).
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace mbpcg {

namespace {

constexpr int kDfBM = 256;       // rows of Q per CTA (and of an A tile)
constexpr int kDfBK = 32;        // values of l per chunk (and per A tile)
constexpr int kDfStages = 3;
constexpr int kDfThreads = 256;  // 8 warps x 32 rows
constexpr int kDfLdA = kDfBK + 4;  // padded row of an A chunk in shared memory (144 B: 16-B aligned, spreads banks)
constexpr int kDfMaxCluster = 8;

template <int KP>
struct DfCfg {
  static constexpr int CT = KP >= 16 ? 4 : (KP >= 8 ? 2 : 1);  // columns per thread
  static constexpr int TX = KP / CT;                           // threads along the columns of a warp
  static constexpr int TY = 32 / TX;                           // threads along the rows of a warp
  static constexpr int RT = 32 / TY;                           // rows per thread
  static constexpr int A_FLOATS = kDfBM * kDfLdA;
  static constexpr int P_FLOATS = kDfBK * KP;
  static constexpr int STAGE_FLOATS = A_FLOATS + P_FLOATS;
  static constexpr size_t SMEM = (size_t)kDfStages * STAGE_FLOATS * sizeof(float);
  static_assert(TX * CT == KP && TY * TX == 32 && RT * TY == 32, "warp tile");
  static_assert(kDfStages * STAGE_FLOATS >= kDfBM * KP, "the partial tile reuses the stages");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// cp.async of `bytes` (4, 8 or 16) from global to shared memory; only the first src_bytes are read,
// the rest of the destination is zero-filled (src_bytes = 0: nothing is read).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, int src_bytes) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Chunk kc of row tile mt: the A tile (one contiguous 32 KB block) and rows k0..k0+31 of P.
template <int KP>
__device__ __forceinline__ void df_load_chunk(float* stage, int n, const float* __restrict__ At,
                                              const float* __restrict__ P, int mt, int kc, int nKc) {
  using C = DfCfg<KP>;
  float* As = stage;
  float* Ps = stage + C::A_FLOATS;
  const int tid = threadIdx.x, k0 = kc * kDfBK;
  const float* tile = At + ((size_t)mt * nKc + kc) * (kDfBM * kDfBK);
  // A: 256 rows x 32 values = 2048 pieces of 16 B, 8 per thread, consecutive threads on consecutive pieces
#pragma unroll
  for (int q0 = 0; q0 < kDfBM * kDfBK / 4; q0 += kDfThreads) {
    const int q = q0 + tid, r = q / (kDfBK / 4), c4 = q % (kDfBK / 4);
    cp_async<16>(As + r * kDfLdA + 4 * c4, tile + 4 * q, 16);
  }
  // P: 16 rows of KP values
  if constexpr (KP >= 4) {
    constexpr int PIECES = kDfBK * KP / 4;
    for (int q = tid; q < PIECES; q += kDfThreads) {
      const int r = q / (KP / 4), c = 4 * (q % (KP / 4)), l = k0 + r;
      cp_async<16>(Ps + r * KP + c, l < n ? P + (size_t)l * KP + c : P, l < n ? 16 : 0);
    }
  } else {
    if (tid < kDfBK) {
      const int l = k0 + tid;
      cp_async<4 * KP>(Ps + tid * KP, l < n ? P + (size_t)l * KP : P, l < n ? 4 * KP : 0);
    }
  }
}

// Q = A P over the K range of this CTA, reduced over the cluster (blockIdx.y = rank = K range).
template <int KP>
__global__ void __launch_bounds__(kDfThreads)
k_dense_f(int n, const float* __restrict__ At, const float* __restrict__ P, float* __restrict__ Q,
          const SolveState* __restrict__ st) {
  using C = DfCfg<KP>;
  if (st != nullptr && st->done) return;  // uniform over the grid, so over every cluster
  extern __shared__ __align__(16) float dsm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int KS = (int)gridDim.y, ks = (int)blockIdx.y;
  const int mt = (int)blockIdx.x, m0 = mt * kDfBM;
  const int nKc = (n + kDfBK - 1) / kDfBK;
  const int c0 = (int)((long long)nKc * ks / KS), c1 = (int)((long long)nKc * (ks + 1) / KS);
  const int nch = c1 - c0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tx = lane % C::TX, ty = lane / C::TX;
  const int rbase = 32 * warp + ty;  // rows rbase + TY k of the tile

  float acc[C::RT][C::CT];
#pragma unroll
  for (int k = 0; k < C::RT; ++k)
#pragma unroll
    for (int c = 0; c < C::CT; ++c) acc[k][c] = 0.f;

#pragma unroll
  for (int s = 0; s < kDfStages - 1; ++s) {
    if (s < nch) df_load_chunk<KP>(dsm + s * C::STAGE_FLOATS, n, At, P, mt, c0 + s, nKc);
    cp_async_commit();
  }
  for (int i = 0; i < nch; ++i) {
    cp_async_wait<kDfStages - 2>();
    __syncthreads();  // chunk i is in place for every thread; every thread is done with chunk i - 1
    const int nx = i + kDfStages - 1;
    if (nx < nch) df_load_chunk<KP>(dsm + (nx % kDfStages) * C::STAGE_FLOATS, n, At, P, mt, c0 + nx, nKc);
    cp_async_commit();
    const float* As = dsm + (i % kDfStages) * C::STAGE_FLOATS;
    const float* Ps = As + C::A_FLOATS;
#pragma unroll
    for (int l4 = 0; l4 < kDfBK; l4 += 4) {
      float4 a[C::RT];
#pragma unroll
      for (int k = 0; k < C::RT; ++k) a[k] = *reinterpret_cast<const float4*>(As + (rbase + C::TY * k) * kDfLdA + l4);
#pragma unroll
      for (int ll = 0; ll < 4; ++ll) {
        float p[C::CT];
        const float* pr = Ps + (l4 + ll) * KP + C::CT * tx;
        if constexpr (C::CT == 4) {
          const float4 v = *reinterpret_cast<const float4*>(pr);
          p[0] = v.x, p[1] = v.y, p[2] = v.z, p[3] = v.w;
        } else if constexpr (C::CT == 2) {
          const float2 v = *reinterpret_cast<const float2*>(pr);
          p[0] = v.x, p[1] = v.y;
        } else {
          p[0] = pr[0];
        }
#pragma unroll
        for (int k = 0; k < C::RT; ++k) {
          const float av = ll == 0 ? a[k].x : ll == 1 ? a[k].y : ll == 2 ? a[k].z : a[k].w;
#pragma unroll
          for (int c = 0; c < C::CT; ++c) acc[k][c] = fmaf(av, p[c], acc[k][c]);
        }
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();  // the stages are free: the partial tile goes there
  float* part = dsm;  // [kDfBM][KP]
#pragma unroll
  for (int k = 0; k < C::RT; ++k)
#pragma unroll
    for (int c = 0; c < C::CT; ++c) part[(rbase + C::TY * k) * KP + C::CT * tx + c] = acc[k][c];
  cluster.sync();
  // rows [r0, r1) of the tile are summed by this CTA over the ranks in order, four values at a
  // time: every remote load of a rank is issued before the first add
  const int r0 = kDfBM * ks / KS, r1 = kDfBM * (ks + 1) / KS;
  if constexpr (KP >= 4) {
    for (int e = r0 * KP + 4 * tid; e < r1 * KP; e += 4 * kDfThreads) {
      float4 pv[kDfMaxCluster];
#pragma unroll
      for (int r = 0; r < kDfMaxCluster; ++r)
        if (r < KS) pv[r] = *reinterpret_cast<const float4*>(cluster.map_shared_rank(part, r) + e);
      float4 v = pv[0];
#pragma unroll
      for (int r = 1; r < kDfMaxCluster; ++r)
        if (r < KS) v.x += pv[r].x, v.y += pv[r].y, v.z += pv[r].z, v.w += pv[r].w;
      if (m0 + e / KP < n) *reinterpret_cast<float4*>(Q + (size_t)m0 * KP + e) = v;
    }
  } else {
    for (int e = r0 * KP + tid; e < r1 * KP; e += kDfThreads) {
      float pv[kDfMaxCluster];
#pragma unroll
      for (int r = 0; r < kDfMaxCluster; ++r)
        if (r < KS) pv[r] = cluster.map_shared_rank(part, r)[e];
      float v = pv[0];
#pragma unroll
      for (int r = 1; r < kDfMaxCluster; ++r)
        if (r < KS) v += pv[r];
      if (m0 + e / KP < n) Q[(size_t)m0 * KP + e] = v;
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its partial tile
}

template <int KP>
void dense_f32_kp(cudaStream_t s, int n, int sms, const float* At, const float* P, float* Q, const SolveState* st) {
  using C = DfCfg<KP>;
  ensure_dynamic_smem(k_dense_f<KP>, C::SMEM);
  const int mt = (n + kDfBM - 1) / kDfBM, nKc = (n + kDfBK - 1) / kDfBK;
  int ks = sms / mt;
  ks = ks < 1 ? 1 : (ks > kDfMaxCluster ? kDfMaxCluster : ks);
  if (ks > nKc) ks = nKc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(mt, ks, 1);
  cfg.blockDim = dim3(kDfThreads, 1, 1);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = ks;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_dense_f<KP>, n, At, P, Q, st);
}

}  // namespace

size_t dense_f32_tiles_bytes(int n) {
  const size_t mt = (n + kDfBM - 1) / kDfBM, nKc = (n + kDfBK - 1) / kDfBK;
  return mt * nKc * kDfBM * kDfBK * sizeof(float);
}

// FP32 tiles of the column-major FP64 symmetric A (row i = column i): tile (mt, kc) holds rows
// 256 mt + r, values 32 kc + c of l at r * 32 + c; entries past n are zero.
__global__ void k_dense_to_f32_tiles(int n, const double* __restrict__ A, float* __restrict__ At) {
  const int nKc = (n + kDfBK - 1) / kDfBK;
  const size_t total = (size_t)((n + kDfBM - 1) / kDfBM) * nKc * kDfBM * kDfBK;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const size_t t = q / (kDfBM * kDfBK);
    const int e = (int)(q % (kDfBM * kDfBK));
    const int i = (int)(t / nKc) * kDfBM + e / kDfBK, l = (int)(t % nKc) * kDfBK + e % kDfBK;
    At[q] = (i < n && l < n) ? (float)A[(size_t)i * n + l] : 0.f;  // A[i*n + l] = column i = row i
  }
}

void dense_f32_product(cudaStream_t s, int kp, int n, int sms, const float* At, const float* P, float* Q,
                       const SolveState* st) {
  switch (kp) {
    case 1: dense_f32_kp<1>(s, n, sms, At, P, Q, st); break;
    case 2: dense_f32_kp<2>(s, n, sms, At, P, Q, st); break;
    case 4: dense_f32_kp<4>(s, n, sms, At, P, Q, st); break;
    case 8: dense_f32_kp<8>(s, n, sms, At, P, Q, st); break;
    case 16: dense_f32_kp<16>(s, n, sms, At, P, Q, st); break;
    default: dense_f32_kp<32>(s, n, sms, At, P, Q, st); break;
  }
}

}  // namespace mbpcg
