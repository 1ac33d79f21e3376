// Row kernels of the mixed-precision inner solve (MBPCG_MIXED_FP32): the n x s blocks of
// Algorithm 1 (U, X0, X~, R, W, P, A P, V) and the sparse matrix values are FP32, products and block
// updates run in FP32 with FP32 accumulation; the k x k matrices stay FP64 (converted to FP32
// where a block is multiplied by them), and every reduction that feeds a k x k step (the Grams
// P^T A P, V^T V, R^T R and the norms nu_j) is accumulated with FP64-class accuracy: each FP32
// product is split exactly into a sum of two FP32 numbers and added with an error-free
// transformation, the compensated dot product "Dot2" of Ogita, Rump & Oishi (SIAM J. Sci. Comput.
// 26, 2005), whose result is as accurate as if computed in twice the working precision. This
// keeps the FP64 pipe (about 2 FMAs per cycle per SM on GB300) out of the n-proportional work.
//
// Layout and conventions are those of row_kernels.cuh: row-major n x KP blocks, balanced row
// ranges per CTA, per-CTA FP64 partials summed in a fixed order by k_reduce, early return once the
// solve is done.
#pragma once
#include "mbpcg_device.cuh"

namespace mbpcg {

// Columns per thread (one 16-byte vector at most), threads per row, rows per tile.
template <int KP>
struct CfgF {
  static constexpr int CPT = KP <= 4 ? KP : 4;
  static constexpr int TPR = KP / CPT;
  static constexpr int ROWS = kThreads / TPR;
  static constexpr int NPACK = KP * (KP + 1) / 2;
};

template <int C>
__device__ __forceinline__ void ldvf(const float* __restrict__ p, float (&v)[C]) {
  if constexpr (C == 1) {
    v[0] = __ldg(p);
  } else if constexpr (C == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  } else {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
}
template <int C>
__device__ __forceinline__ void ldvf_plain(const float* p, float (&v)[C]) {
  if constexpr (C == 1) {
    v[0] = *p;
  } else if constexpr (C == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x;
    v[1] = t.y;
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
}
template <int C>
__device__ __forceinline__ void stvf(float* p, const float (&v)[C]) {
  if constexpr (C == 1) {
    *p = v[0];
  } else if constexpr (C == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// (s, c) += x y with s + c carrying the sum: the product is split exactly (x y = p + pe, pe from
// one FMA), p is added to s by Knuth's TwoSum (s + p = t + se exactly), and the two error terms
// go to c. The _rn intrinsics keep the compiler from contracting the steps into FMAs.
__device__ __forceinline__ void dot2_add(float& s, float& c, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float pe = fmaf(x, y, -p);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(se, pe));
}

// Upper triangle of X^T Y over a tile of FP32 rows in shared memory (row stride KP), with Dot2
// accumulators; same thread layout as GramTile (2 x 2 blocks, row classes), FP64 partials.
template <int KP>
struct GramTileF {
  static constexpr int NB2 = (KP + 1) / 2;
  static constexpr int NBLK = NB2 * (NB2 + 1) / 2;
  static constexpr int RS = kThreads / NBLK;
  static constexpr int RED = RS * NBLK * 4;  // doubles of shared scratch for finish()
  int bl, bj, blk, split;
  bool active;
  float s00, s01, s10, s11, c00, c01, c10, c11;

  __device__ __forceinline__ void init(int tid) {
    active = tid < NBLK * RS;
    blk = tid % NBLK;
    split = tid / NBLK;
    bj = 0;
    while ((bj + 1) * (bj + 2) / 2 <= blk) ++bj;
    bl = blk - bj * (bj + 1) / 2;
    s00 = s01 = s10 = s11 = c00 = c01 = c10 = c11 = 0.f;
  }
  __device__ __forceinline__ void accumulate(const float* Xs, const float* Ys, int nrows) {
    if (!active) return;
    if constexpr (KP == 1) {
      for (int r = split; r < nrows; r += RS) dot2_add(s00, c00, Xs[r], Ys[r]);
    } else {
      for (int r = split; r < nrows; r += RS) {
        const float2 x = *reinterpret_cast<const float2*>(Xs + r * KP + 2 * bl);
        const float2 y = *reinterpret_cast<const float2*>(Ys + r * KP + 2 * bj);
        dot2_add(s00, c00, x.x, y.x);
        dot2_add(s01, c01, x.x, y.y);
        dot2_add(s10, c10, x.y, y.x);
        dot2_add(s11, c11, x.y, y.y);
      }
    }
  }
  __device__ void finish(double* red, double* out) {
    __syncthreads();
    if (active) {
      const int o = (split * NBLK + blk) * 4;
      red[o] = (double)s00 + (double)c00;
      red[o + 1] = (double)s01 + (double)c01;
      red[o + 2] = (double)s10 + (double)c10;
      red[o + 3] = (double)s11 + (double)c11;
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

// Q = A P (FP32 CSR values, FP32 accumulation) and, when GRAM, the Dot2 partials of the upper
// triangle of P^T Q (Algorithm 1, the A P product and the Gram that defines Xi). Four threads own a
// row (16-byte vectors of P), UNR nonzeros of a row are in flight per thread. On the 27-point
// stencil at KP = 16 this form is bound by the gathers of P rows through L2 (27 x 64 bytes per row),
// not by the CSR stream: staging the CSR slice of a warp in shared memory or prefetching it did
// not make it faster.
template <int KP, bool GRAM, int UNR = 8>
__global__ void __launch_bounds__(kThreads)
k_spmm_f(int n, const int* __restrict__ rp, const int* __restrict__ ci, const float* __restrict__ av,
         const float* __restrict__ P, float* __restrict__ Q, double* __restrict__ part, int pstride,
         const SolveState* __restrict__ st) {
  using C = CfgF<KP>;
  using G = GramTileF<KP>;
  if (st != nullptr && st->done) return;
  __shared__ __align__(16) float Xs[GRAM ? C::ROWS * KP : 4];
  __shared__ __align__(16) float Ys[GRAM ? C::ROWS * KP : 4];
  __shared__ __align__(16) double red[GRAM ? G::RED : 2];
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  G g;
  if constexpr (GRAM) g.init(tid);
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    float acc[C::CPT], pv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) acc[c] = pv[c] = 0.f;
    if (i < r1) {
      const int pe = __ldg(rp + i + 1);
#pragma unroll UNR
      for (int p = __ldg(rp + i); p < pe; ++p) {
        const int col = __ldg(ci + p);
        const float a = __ldg(av + p);
        float x[C::CPT];
        ldvf<C::CPT>(P + (size_t)col * KP + j0, x);
#pragma unroll
        for (int c = 0; c < C::CPT; ++c) acc[c] = fmaf(a, x[c], acc[c]);
      }
      stvf<C::CPT>(Q + (size_t)i * KP + j0, acc);
      if constexpr (GRAM) ldvf<C::CPT>(P + (size_t)i * KP + j0, pv);
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
  if constexpr (GRAM) g.finish(red, part + (size_t)blockIdx.x * pstride);
}

// Dot2 partials of the upper triangle of X^T Y for FP32 blocks (the Gram P^T (A P) of the mixed
// inner solve, as a pass of its own after the product: fusing it into the gather-bound product
// serialised the two inside each CTA and cost more than re-reading P and A P).
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_gram_f(int n, const float* __restrict__ X, const float* __restrict__ Y, double* __restrict__ part, int pstride,
         const SolveState* __restrict__ st) {
  using C = CfgF<KP>;
  using G = GramTileF<KP>;
  if (st != nullptr && st->done) return;
  __shared__ __align__(16) float Xs[C::ROWS * KP];
  __shared__ __align__(16) float Ys[C::ROWS * KP];
  __shared__ __align__(16) double red[G::RED];
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  G g;
  g.init(tid);
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    float xv[C::CPT], yv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) xv[c] = yv[c] = 0.f;
    if (i < r1) {
      ldvf<C::CPT>(X + (size_t)i * KP + j0, xv);
      ldvf<C::CPT>(Y + (size_t)i * KP + j0, yv);
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
}

// Block update of Algorithm 1 in FP32: X~ += P T, R -= (A P) T, V = W - (A P) Xi (T, Xi converted
// from FP64), with Dot2 partials of nu_j = ||(D R)_j||^2 at part[NPACK + j] and of V^T V at
// part[0..). wdiag32 = diag(A) in FP32 (D^2) or NULL.
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_axpy_f(int n, const float* __restrict__ P, const float* __restrict__ Q, const float* __restrict__ W,
         float* __restrict__ R, float* __restrict__ Xt, float* __restrict__ V, const double* __restrict__ Tg,
         const double* __restrict__ Xig, const float* __restrict__ wdiag, double* __restrict__ part, int pstride,
         const SolveState* __restrict__ st) {
  using C = CfgF<KP>;
  using G = GramTileF<KP>;
  constexpr int RED = (G::RED > C::ROWS * KP) ? G::RED : C::ROWS * KP;
  if (st->done) return;
  __shared__ __align__(16) float Ts[KP * KP];
  __shared__ __align__(16) float Xis[KP * KP];
  __shared__ __align__(16) float Ps[C::ROWS * KP];
  __shared__ __align__(16) float Qs[C::ROWS * KP];
  __shared__ __align__(16) float Vs[C::ROWS * KP];
  __shared__ __align__(16) double red[RED];
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  for (int q = tid; q < KP * KP; q += kThreads) {  // column-major in global -> row-major here
    const int l = q % KP, jj = q / KP;
    Ts[l * KP + jj] = (float)Tg[q];
    Xis[l * KP + jj] = (float)Xig[q];
  }
  int r0, r1;
  row_range(n, r0, r1);
  G g;
  g.init(tid);
  float nus[C::CPT], nuc[C::CPT];
#pragma unroll
  for (int c = 0; c < C::CPT; ++c) nus[c] = nuc[c] = 0.f;
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    const bool valid = i < r1;
    float pv[C::CPT], qv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) pv[c] = qv[c] = 0.f;
    if (valid) {
      ldvf<C::CPT>(P + (size_t)i * KP + j0, pv);
      ldvf<C::CPT>(Q + (size_t)i * KP + j0, qv);
    }
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) {
      Ps[rl * KP + j0 + c] = pv[c];
      Qs[rl * KP + j0 + c] = qv[c];
    }
    __syncthreads();
    float vv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) vv[c] = 0.f;
    if (valid) {
      float xv[C::CPT], rv[C::CPT];
      ldvf_plain<C::CPT>(Xt + (size_t)i * KP + j0, xv);
      ldvf_plain<C::CPT>(R + (size_t)i * KP + j0, rv);
      ldvf<C::CPT>(W + (size_t)i * KP + j0, vv);
#pragma unroll 8
      for (int l = 0; l < KP; ++l) {
        const float pl = Ps[rl * KP + l], ql = Qs[rl * KP + l];
#pragma unroll
        for (int c = 0; c < C::CPT; ++c) {
          const float t = Ts[l * KP + j0 + c];
          xv[c] = fmaf(pl, t, xv[c]);
          rv[c] = fmaf(-ql, t, rv[c]);
          vv[c] = fmaf(-ql, Xis[l * KP + j0 + c], vv[c]);
        }
      }
      stvf<C::CPT>(Xt + (size_t)i * KP + j0, xv);
      stvf<C::CPT>(R + (size_t)i * KP + j0, rv);
      stvf<C::CPT>(V + (size_t)i * KP + j0, vv);
      const float wi = (wdiag != nullptr) ? __ldg(wdiag + i) : 1.f;
#pragma unroll
      for (int c = 0; c < C::CPT; ++c) dot2_add(nus[c], nuc[c], rv[c] * wi, rv[c]);
    }
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) Vs[rl * KP + j0 + c] = vv[c];
    __syncthreads();
    g.accumulate(Vs, Vs, min(C::ROWS, r1 - base));
    __syncthreads();
  }
  double* out = part + (size_t)blockIdx.x * pstride;
  g.finish(red, out);
#pragma unroll
  for (int c = 0; c < C::CPT; ++c) red[rl * KP + j0 + c] = (double)nus[c] + (double)nuc[c];
  cta_tree_sum(red, C::ROWS, KP);
  for (int jj = tid; jj < KP; jj += kThreads) out[C::NPACK + jj] = red[jj];
}

// W = V zeta^{-1}, then P = W + P zeta^T (or P = W when SETP): one thread per row, FP32, with the
// two triangular factors (FP64 in global) in FP32 shared memory.
template <int KP, bool SETP>
__global__ void __launch_bounds__(kThreads)
k_pw_f(int n, const float* __restrict__ V, float* __restrict__ W, float* __restrict__ P,
       const double* __restrict__ Zinvg, const double* __restrict__ Zg, const SolveState* __restrict__ st) {
  if (st != nullptr && st->pw_skip) return;
  __shared__ float Zis[KP * KP];
  __shared__ float Zs[KP * KP];
  const int tid = threadIdx.x;
  for (int q = tid; q < KP * KP; q += kThreads) {
    const int l = q % KP, jj = q / KP;
    Zis[l * KP + jj] = (float)Zinvg[q];
    Zs[l * KP + jj] = SETP ? 0.f : (float)Zg[q];
  }
  __syncthreads();
  constexpr int VC = KP <= 4 ? KP : 4;
  int r0, r1;
  row_range(n, r0, r1);
  for (int i = r0 + tid; i < r1; i += kThreads) {
    float v[KP], w[KP];
#pragma unroll
    for (int c = 0; c < KP; c += VC) {
      float t[VC];
      ldvf<VC>(V + (size_t)i * KP + c, t);
#pragma unroll
      for (int e = 0; e < VC; ++e) v[c + e] = t[e];
    }
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l <= j; ++l) a = fmaf(v[l], Zis[l * KP + j], a);
      w[j] = a;
    }
#pragma unroll
    for (int c = 0; c < KP; c += VC) {
      float t[VC];
#pragma unroll
      for (int e = 0; e < VC; ++e) t[e] = w[c + e];
      stvf<VC>(W + (size_t)i * KP + c, t);
    }
    if constexpr (SETP) {
#pragma unroll
      for (int c = 0; c < KP; c += VC) {
        float t[VC];
#pragma unroll
        for (int e = 0; e < VC; ++e) t[e] = w[c + e];
        stvf<VC>(P + (size_t)i * KP + c, t);
      }
    } else {
      float p[KP];
#pragma unroll
      for (int c = 0; c < KP; c += VC) {
        float t[VC];
        ldvf_plain<VC>(P + (size_t)i * KP + c, t);
#pragma unroll
        for (int e = 0; e < VC; ++e) p[c + e] = t[e];
      }
#pragma unroll
      for (int c = 0; c < KP; c += VC) {
        float t[VC];
#pragma unroll
        for (int e = 0; e < VC; ++e) {
          const int j = c + e;
          float a = w[j];
#pragma unroll
          for (int l = j; l < KP; ++l) a = fmaf(p[l], Zs[j * KP + l], a);
          t[e] = a;
        }
        stvf<VC>(P + (size_t)i * KP + c, t);
      }
    }
  }
}

// Set-up norms: bs = D^{-1} rhs (FP64), partials of ||rhs||^2, ||bs||^2 (FP64) and ||A U||_F^2
// (Dot2 over the FP32 block).
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_setup_norms_f(int n, const double* __restrict__ rhs, const double* __restrict__ d, double* __restrict__ bs,
                const float* __restrict__ AU, double* __restrict__ part, int pstride) {
  __shared__ double red[3 * kThreads];
  constexpr int VC = KP <= 4 ? KP : 4;
  int r0, r1;
  row_range(n, r0, r1);
  double s0 = 0.0, s1 = 0.0;
  float s2 = 0.f, c2 = 0.f;
  for (int i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const double b = rhs[i];
    const double v = (d != nullptr) ? d[i] * b : b;
    bs[i] = v;
    s0 = fma(b, b, s0);
    s1 = fma(v, v, s1);
#pragma unroll
    for (int c = 0; c < KP; c += VC) {
      float t[VC];
      ldvf<VC>(AU + (size_t)i * KP + c, t);
#pragma unroll
      for (int e = 0; e < VC; ++e) dot2_add(s2, c2, t[e], t[e]);
    }
  }
  red[threadIdx.x * 3] = s0;
  red[threadIdx.x * 3 + 1] = s1;
  red[threadIdx.x * 3 + 2] = (double)s2 + (double)c2;
  cta_tree_sum(red, kThreads, 3);
  if (threadIdx.x < 3) part[(size_t)blockIdx.x * pstride + threadIdx.x] = red[threadIdx.x];
}

// X0 = scale U; X~ = 0; R = bs 1^T - scale (A U) (columns < s) in FP32, with Dot2 partials of R^T R.
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_init_f(int n, int s, const float* __restrict__ U, const float* __restrict__ AU, const double* __restrict__ bs,
         float* __restrict__ X0, float* __restrict__ Xt, float* __restrict__ R, double* __restrict__ part,
         int pstride, const SolveState* __restrict__ st) {
  using C = CfgF<KP>;
  using G = GramTileF<KP>;
  __shared__ __align__(16) float Rs[C::ROWS * KP];
  __shared__ __align__(16) double red[G::RED];
  const float scale = (float)st->scale;
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  G g;
  g.init(tid);
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    float rv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) rv[c] = 0.f;
    if (i < r1) {
      float u[C::CPT], au[C::CPT], x0[C::CPT], z[C::CPT];
      ldvf<C::CPT>(U + (size_t)i * KP + j0, u);
      ldvf<C::CPT>(AU + (size_t)i * KP + j0, au);
      const float b = (float)bs[i];
#pragma unroll
      for (int c = 0; c < C::CPT; ++c) {
        x0[c] = scale * u[c];
        z[c] = 0.f;
        rv[c] = (j0 + c < s) ? fmaf(-scale, au[c], b) : 0.f;
      }
      stvf<C::CPT>(X0 + (size_t)i * KP + j0, x0);
      stvf<C::CPT>(Xt + (size_t)i * KP + j0, z);
      stvf<C::CPT>(R + (size_t)i * KP + j0, rv);
    }
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) Rs[rl * KP + j0 + c] = rv[c];
    __syncthreads();
    g.accumulate(Rs, Rs, min(C::ROWS, r1 - base));
    __syncthreads();
  }
  g.finish(red, part + (size_t)blockIdx.x * pstride);
}

// Exit Gram of M = [rhs | D R] in FP64 (R read in FP32): the least-squares combination of
// Section 2 is formed once per inner solve, so it uses the FP64 Gram tiles of row_kernels.cuh.
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_ls_gram_f(int n, const float* __restrict__ R, const double* __restrict__ rhs, const double* __restrict__ sqd,
            double* __restrict__ part, int pstride) {
  using C = CfgF<KP>;
  using G = GramTile<KP>;
  constexpr int RED = (G::RED > C::ROWS * (KP + 1)) ? G::RED : C::ROWS * (KP + 1);
  __shared__ __align__(16) double Ms[C::ROWS * KP];
  __shared__ __align__(16) double red[RED];
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  G g;
  g.init(tid);
  double br[C::CPT], bb = 0.0;
#pragma unroll
  for (int c = 0; c < C::CPT; ++c) br[c] = 0.0;
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    double mv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) mv[c] = 0.0;
    if (i < r1) {
      float rf[C::CPT];
      ldvf<C::CPT>(R + (size_t)i * KP + j0, rf);
      const double di = (sqd != nullptr) ? sqd[i] : 1.0;
      const double b = rhs[i];
#pragma unroll
      for (int c = 0; c < C::CPT; ++c) {
        mv[c] = (double)rf[c] * di;
        br[c] = fma(b, mv[c], br[c]);
      }
      if (j0 == 0) bb = fma(b, b, bb);
    }
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) Ms[rl * KP + j0 + c] = mv[c];
    __syncthreads();
    g.accumulate(Ms, Ms, min(C::ROWS, r1 - base));
    __syncthreads();
  }
  double* out = part + (size_t)blockIdx.x * pstride;
  g.finish(red, out);
#pragma unroll
  for (int c = 0; c < C::CPT; ++c) red[rl * (KP + 1) + j0 + c] = br[c];
  if (j0 == 0) red[rl * (KP + 1) + KP] = bb;
  cta_tree_sum(red, C::ROWS, KP + 1);
  for (int jj = tid; jj <= KP; jj += kThreads) out[C::NPACK + jj] = red[jj];
}

// x += D^{-1} (X~ + X0) c in FP64 from the FP32 blocks.
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_combine_f(int n, int s, const float* __restrict__ Xt, const float* __restrict__ X0, const double* __restrict__ c,
            const double* __restrict__ d, double* __restrict__ x) {
  __shared__ double cs[KP];
  constexpr int VC = KP <= 4 ? KP : 4;
  if (threadIdx.x < KP) cs[threadIdx.x] = (int)threadIdx.x < s ? c[threadIdx.x] : 0.0;
  __syncthreads();
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
    double a = 0.0;
#pragma unroll
    for (int cc = 0; cc < KP; cc += VC) {
      float xt[VC], x0[VC];
      ldvf<VC>(Xt + (size_t)i * KP + cc, xt);
      ldvf<VC>(X0 + (size_t)i * KP + cc, x0);
#pragma unroll
      for (int e = 0; e < VC; ++e) a = fma((double)xt[e] + (double)x0[e], cs[cc + e], a);
    }
    x[i] += (d != nullptr) ? d[i] * a : a;
  }
}

// U[i][j] = 2 u01(seed, stream 1 + j, index i) - 1 (rounded to FP32) for j < s, 0 in the padding.
template <int KP>
__global__ void k_gen_u_f(int n, int s, unsigned long long seed, float* __restrict__ U) {
  const size_t total = (size_t)n * KP;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q % KP);
    const size_t i = q / KP;
    U[q] = (j < s) ? (float)(2.0 * splitmix_uniform01(seed, 1 + j, i) - 1.0) : 0.f;
  }
}

// Column-major n x s FP64 (leading dimension n) -> row-major n x KP FP32 with zero padding.
template <int KP>
__global__ void k_from_colmajor_f(int n, int s, const double* __restrict__ src, float* __restrict__ dst) {
  const size_t total = (size_t)n * KP;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q % KP);
    const size_t i = q / KP;
    dst[q] = (j < s) ? (float)src[(size_t)j * n + i] : 0.f;
  }
}

}  // namespace mbpcg
