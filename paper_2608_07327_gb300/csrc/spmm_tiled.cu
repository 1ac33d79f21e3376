// CSR product A P of Algorithm 1 with the rows of P a tile needs staged in shared memory (sm_103a).
//
// The rows of A are cut into tiles of R consecutive rows. At create, for every tile, the distinct
// columns its nonzeros touch are collected and merged into runs of consecutive columns (for a
// stencil or banded matrix: a few runs, one per neighbouring grid line or plane segment), and
// every nonzero gets the position of its column inside the tile's window (a 16-bit local index,
// which also halves the index bytes streamed per nonzero). In the loop, a CTA copies its tile's
// runs of P -- contiguous rows, read once with 16-byte loads -- into shared memory and forms its
// rows' products from there, instead of gathering a row of P from L2 for every nonzero (27
// gathers of 64 bytes per row of the 27-point stencil at s = 16, eight times the bytes of P).
// Each row is summed in the order of its nonzeros, as the gather kernel does, so both give the
// same bits. R is the largest power of two (<= 4096) for which every tile's window fits the
// shared-memory budget; matrices whose windows never fit keep the gather kernel.
#include <algorithm>
#include <vector>

#include "kernels.h"
#include "row_kernels.cuh"
#include "row_kernels_f32.cuh"

namespace mbpcg {

namespace {

constexpr size_t kWindowBytes = 96 * 1024;  // shared memory of one tile's window (two CTAs per SM)
constexpr int kMaxTileRows = 4096;
constexpr int kMinTileRows = 32;

// Staged rows of the tile's window: rows [run_start, run_start + run_len) of P, run after run.
template <typename T, int KP>
__device__ __forceinline__ void stage_window(const SpmmPlan& pl, int t, const T* __restrict__ P, T* __restrict__ Ps) {
  constexpr int VE = 16 / sizeof(T);  // values per 16-byte load
  int off = 0;
  for (int q = pl.run_ptr[t]; q < pl.run_ptr[t + 1]; ++q) {
    const int r0 = pl.run_start[q], len = pl.run_len[q];
    const T* src = P + (size_t)r0 * KP;
    T* dst = Ps + (size_t)off * KP;
    const int cnt = len * KP;
    if constexpr (KP % VE == 0) {
      for (int e = threadIdx.x; e < cnt / VE; e += kThreads)
        reinterpret_cast<uint4*>(dst)[e] = __ldg(reinterpret_cast<const uint4*>(src) + e);
    } else {
      for (int e = threadIdx.x; e < cnt; e += kThreads) dst[e] = __ldg(src + e);
    }
    off += len;
  }
}

}  // namespace

// Q = A P for the rows of each tile of this CTA (tiles t = blockIdx.x, + gridDim.x, ...) and, when
// GRAM, the CTA partials of the upper triangle of P^T Q (as k_spmm writes them).
template <int KP, bool GRAM>
__global__ void __launch_bounds__(kThreads)
k_spmm_tiled(int n, const int* __restrict__ rp, const double* __restrict__ av, SpmmPlan pl,
             const double* __restrict__ P, double* __restrict__ Q, double* __restrict__ part, int pstride,
             const SolveState* __restrict__ st) {
  using C = Cfg<KP>;
  using G = GramTile<KP>;
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(16) double tsm[];
  double* Ps = tsm;
  __shared__ __align__(16) double Xs[GRAM ? C::ROWS * KP : 2];
  __shared__ __align__(16) double Ys[GRAM ? C::ROWS * KP : 2];
  __shared__ __align__(16) double red[GRAM ? G::RED : 2];
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  G g;
  if constexpr (GRAM) g.init(tid);
  for (int t = blockIdx.x; t < pl.ntiles; t += gridDim.x) {
    const int r0 = t * pl.R, r1 = min(n, r0 + pl.R);
    __syncthreads();  // the previous tile has finished with the window
    stage_window<double, KP>(pl, t, P, Ps);
    __syncthreads();
    for (int base = r0; base < r1; base += C::ROWS) {
      const int i = base + rl;
      double acc[C::CPT], pv[C::CPT];
#pragma unroll
      for (int c = 0; c < C::CPT; ++c) acc[c] = pv[c] = 0.0;
      if (i < r1) {
        const int pe = __ldg(rp + i + 1);
#pragma unroll 4
        for (int p = __ldg(rp + i); p < pe; ++p) {
          const double a = __ldg(av + p);
          const int l = __ldg(pl.cl + p);
          double x[C::CPT];
          ldv_plain<C::CPT>(Ps + l * KP + j0, x);
#pragma unroll
          for (int c = 0; c < C::CPT; ++c) acc[c] = fma(a, x[c], acc[c]);
        }
        stv<C::CPT>(Q + (size_t)i * KP + j0, acc);
        if constexpr (GRAM) ldv<C::CPT>(P + (size_t)i * KP + j0, pv);
      }
      if constexpr (GRAM) {
#pragma unroll
        for (int c = 0; c < C::CPT; ++c) {
          Xs[rl * KP + j0 + c] = pv[c];
          Ys[rl * KP + j0 + c] = acc[c];
        }
        __syncthreads();
        g.accumulate(Xs, Ys, min(C::ROWS, r1 - base));
        __syncthreads();
      }
    }
  }
  if constexpr (GRAM) g.finish(red, part + (size_t)blockIdx.x * pstride);
}

// The FP32 form (mixed-precision inner solve): FP32 values, P and Q, FP32 accumulation, no Gram.
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_spmm_tiled_f(int n, const int* __restrict__ rp, const float* __restrict__ av, SpmmPlan pl,
               const float* __restrict__ P, float* __restrict__ Q, const SolveState* __restrict__ st) {
  using C = CfgF<KP>;
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(16) double tsm[];
  float* Ps = reinterpret_cast<float*>(tsm);
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  for (int t = blockIdx.x; t < pl.ntiles; t += gridDim.x) {
    const int r0 = t * pl.R, r1 = min(n, r0 + pl.R);
    __syncthreads();
    stage_window<float, KP>(pl, t, P, Ps);
    __syncthreads();
    for (int base = r0; base < r1; base += C::ROWS) {
      const int i = base + rl;
      if (i < r1) {
        float acc[C::CPT];
#pragma unroll
        for (int c = 0; c < C::CPT; ++c) acc[c] = 0.f;
        const int pe = __ldg(rp + i + 1);
#pragma unroll 4
        for (int p = __ldg(rp + i); p < pe; ++p) {
          const float a = __ldg(av + p);
          const int l = __ldg(pl.cl + p);
          float x[C::CPT];
          ldvf_plain<C::CPT>(Ps + l * KP + j0, x);
#pragma unroll
          for (int c = 0; c < C::CPT; ++c) acc[c] = fmaf(a, x[c], acc[c]);
        }
        stvf<C::CPT>(Q + (size_t)i * KP + j0, acc);
      }
    }
  }
}

// ------------------------------------------------------------------------------------ host side

size_t spmm_plan_window_rows(int kp, size_t elem) { return kWindowBytes / ((size_t)kp * elem); }

int spmm_plan_build(int n, const int* rp, const int* ci, int kp, size_t elem, SpmmPlanHost* out) {
  const size_t wmax = spmm_plan_window_rows(kp, elem);
  const long long nnz = rp[n];
  if (n < 1 || nnz < 1) return 0;
  std::vector<int> pos(n, -1);
  for (int R = kMaxTileRows; R >= kMinTileRows; R /= 2) {
    const int ntiles = (n + R - 1) / R;
    std::vector<int> run_ptr(ntiles + 1, 0), run_start, run_len;
    std::vector<uint16_t> cl((size_t)nnz);
    std::vector<int> cols;
    bool fits = true;
    int wmax_used = 0;
    for (int t = 0; t < ntiles && fits; ++t) {
      const int r0 = t * R, r1 = std::min(n, r0 + R);
      cols.assign(ci + rp[r0], ci + rp[r1]);
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      if (cols.size() > wmax || cols.size() > 65535) {
        fits = false;
        break;
      }
      wmax_used = std::max(wmax_used, (int)cols.size());
      for (size_t q = 0; q < cols.size(); ++q) {
        pos[cols[q]] = (int)q;
        if (q == 0 || cols[q] != cols[q - 1] + 1) {
          run_start.push_back(cols[q]);
          run_len.push_back(1);
        } else {
          ++run_len.back();
        }
      }
      run_ptr[t + 1] = (int)run_start.size();
      for (long long p = rp[r0]; p < rp[r1]; ++p) cl[(size_t)p] = (uint16_t)pos[ci[p]];
      for (int c : cols) pos[c] = -1;
    }
    if (!fits) continue;
    out->R = R;
    out->ntiles = ntiles;
    out->wmax = wmax_used;
    out->run_ptr.swap(run_ptr);
    out->run_start.swap(run_start);
    out->run_len.swap(run_len);
    out->cl.swap(cl);
    return 1;
  }
  return 0;
}

size_t spmm_plan_smem(int kp, size_t elem, int wmax) { return (size_t)wmax * kp * elem; }

namespace {

template <int KP>
void tiled_kp(cudaStream_t s, int nb, int n, const int* rp, const double* av, const SpmmPlan& pl, const double* P,
              double* Q, double* part, int pstride, const SolveState* st, int gram) {
  const size_t smem = spmm_plan_smem(KP, sizeof(double), pl.wmax);
  ensure_dynamic_smem(k_spmm_tiled<KP, true>, kWindowBytes);
  ensure_dynamic_smem(k_spmm_tiled<KP, false>, kWindowBytes);
  if (gram) k_spmm_tiled<KP, true><<<nb, kThreads, smem, s>>>(n, rp, av, pl, P, Q, part, pstride, st);
  else k_spmm_tiled<KP, false><<<nb, kThreads, smem, s>>>(n, rp, av, pl, P, Q, part, pstride, st);
}

template <int KP>
void tiled_f_kp(cudaStream_t s, int nb, int n, const int* rp, const float* av, const SpmmPlan& pl, const float* P,
                float* Q, const SolveState* st) {
  const size_t smem = spmm_plan_smem(KP, sizeof(float), pl.wmax);
  ensure_dynamic_smem(k_spmm_tiled_f<KP>, kWindowBytes);
  k_spmm_tiled_f<KP><<<nb, kThreads, smem, s>>>(n, rp, av, pl, P, Q, st);
}

}  // namespace

void spmm_tiled(cudaStream_t s, int kp, int nb, int n, const int* rp, const double* av, const SpmmPlan& pl,
                const double* P, double* Q, double* part, int pstride, const SolveState* st, int gram) {
  switch (kp) {
    case 1: tiled_kp<1>(s, nb, n, rp, av, pl, P, Q, part, pstride, st, gram); break;
    case 2: tiled_kp<2>(s, nb, n, rp, av, pl, P, Q, part, pstride, st, gram); break;
    case 4: tiled_kp<4>(s, nb, n, rp, av, pl, P, Q, part, pstride, st, gram); break;
    case 8: tiled_kp<8>(s, nb, n, rp, av, pl, P, Q, part, pstride, st, gram); break;
    case 16: tiled_kp<16>(s, nb, n, rp, av, pl, P, Q, part, pstride, st, gram); break;
    default: tiled_kp<32>(s, nb, n, rp, av, pl, P, Q, part, pstride, st, gram); break;
  }
}

void spmm_tiled_f(cudaStream_t s, int kp, int nb, int n, const int* rp, const float* av, const SpmmPlan& pl,
                  const float* P, float* Q, const SolveState* st) {
  switch (kp) {
    case 1: tiled_f_kp<1>(s, nb, n, rp, av, pl, P, Q, st); break;
    case 2: tiled_f_kp<2>(s, nb, n, rp, av, pl, P, Q, st); break;
    case 4: tiled_f_kp<4>(s, nb, n, rp, av, pl, P, Q, st); break;
    case 8: tiled_f_kp<8>(s, nb, n, rp, av, pl, P, Q, st); break;
    case 16: tiled_f_kp<16>(s, nb, n, rp, av, pl, P, Q, st); break;
    default: tiled_f_kp<32>(s, nb, n, rp, av, pl, P, Q, st); break;
  }
}

}  // namespace mbpcg
