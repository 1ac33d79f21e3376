// FP32 CSR product A P of the mixed-precision inner solve with wide CTAs (sm_103a).
//
// On a stencil at s = 16 the gather kernel is bound by its gathers of P rows (27 rows of 64 bytes
// per row of the 27-point stencil, about eight times the bytes of P), and these reach L2 because
// the L1 of an SM does not hold what its CTAs read: with 8 CTAs of 256 threads, an SM works on 8
// unrelated row ranges at once. With CTAs of 512 or 1024 threads and 1 to 4 of them per SM, the
// rows an SM has in flight are few contiguous ranges, whose P rows (the rows of the neighbouring
// grid lines and planes) are read by many of its rows while still in L1. Each thread sums one row
// (or KP / TPR columns of it) in the order of its nonzeros, as the gather kernel does: the same
// bits for any launch shape.
#include "kernels.h"
#include "row_kernels_f32.cuh"

namespace mbpcg {

template <int KP, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_spmm_wide_f(int n, const int* __restrict__ rp, const int* __restrict__ ci, const float* __restrict__ av,
              const float* __restrict__ P, float* __restrict__ Q, const SolveState* __restrict__ st) {
  using C = CfgF<KP>;
  constexpr int ROWS = THREADS / C::TPR;
  if (st != nullptr && st->done) return;
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  for (int i = r0 + rl; i < r1; i += ROWS) {
    float acc[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) acc[c] = 0.f;
    const int pe = __ldg(rp + i + 1);
#pragma unroll 8
    for (int p = __ldg(rp + i); p < pe; ++p) {
      const int col = __ldg(ci + p);
      const float a = __ldg(av + p);
      float x[C::CPT];
      ldvf<C::CPT>(P + (size_t)col * KP + j0, x);
#pragma unroll
      for (int c = 0; c < C::CPT; ++c) acc[c] = fmaf(a, x[c], acc[c]);
    }
    stvf<C::CPT>(Q + (size_t)i * KP + j0, acc);
  }
}

namespace {

template <int KP>
void wide_kp(cudaStream_t s, int threads, int nb, int n, const int* rp, const int* ci, const float* av,
             const float* P, float* Q, const SolveState* st) {
  if (threads == 1024) k_spmm_wide_f<KP, 1024><<<nb, 1024, 0, s>>>(n, rp, ci, av, P, Q, st);
  else k_spmm_wide_f<KP, 512><<<nb, 512, 0, s>>>(n, rp, ci, av, P, Q, st);
}

}  // namespace

void spmm_wide_f(cudaStream_t s, int kp, int threads, int nb, int n, const int* rp, const int* ci, const float* av,
                 const float* P, float* Q, const SolveState* st) {
  switch (kp) {
    case 1: wide_kp<1>(s, threads, nb, n, rp, ci, av, P, Q, st); break;
    case 2: wide_kp<2>(s, threads, nb, n, rp, ci, av, P, Q, st); break;
    case 4: wide_kp<4>(s, threads, nb, n, rp, ci, av, P, Q, st); break;
    case 8: wide_kp<8>(s, threads, nb, n, rp, ci, av, P, Q, st); break;
    case 16: wide_kp<16>(s, threads, nb, n, rp, ci, av, P, Q, st); break;
    default: wide_kp<32>(s, threads, nb, n, rp, ci, av, P, Q, st); break;
  }
}

}  // namespace mbpcg
