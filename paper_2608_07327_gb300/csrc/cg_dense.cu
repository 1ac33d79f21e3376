// Chronopoulos-Gear CG (the paper's baseline, Sections 1 and 4) on a dense A: one launch per
// iteration (sm_103a).
//
// Iteration j of the method, on the scaled system, with u = r (no further preconditioner):
//   w_j = A r_j;  gamma_j = (r_j, r_j), delta_j = (w_j, r_j);  test ||D r_j|| < tol ||rhs||;
//   beta_j = gamma_j / gamma_{j-1} (beta_0 = 0);  alpha_j = gamma_j / (delta_j - beta_j gamma_j / alpha_{j-1});
//   p_j = r_j + beta_j p_{j-1};  s_j = w_j + beta_j s_{j-1};  x_{j+1} = x_j + alpha_j p_j;  r_{j+1} = r_j - alpha_j s_j.
//
// Launch j does, in this order:
//   1. the vector updates of iteration j-1 (alpha_{j-1}, beta_{j-1} from the solve state): every CTA
//      forms the whole new r_j into shared memory (it is the vector of its product) and writes the
//      updated p, s, x, r for its own rows;
//   2. w_j = A r_j for its own rows (A streamed once from HBM, FP64 FMAs);
//   3. its partial sums of gamma_j, delta_j and ||D r_j||^2;
//   4. the last CTA to finish (arrival counter) sums the partials in a fixed order, runs the test,
//      computes alpha_j and beta_j, writes the solve state and sets the loop condition.
// Vectors read whole by every CTA while their owners update them (r, w, s) are kept in two copies,
// selected by the parity of j; p and x are touched only by their owners and live in one copy.
//
// Roofline: 2 n^2 FP64 flop and 8 n^2 bytes of A per iteration. On GB300 the FP64 pipe (2 DFMA per
// clock per SM) binds: n = 4096 takes 26.7 us at 2.07 GHz; A at the HBM read rate takes about 24 us.
// Work split: each CTA owns a balanced range of rows (one CTA per SM). Its rows are cut into chunks
// of 512 columns (8 double2 loads per lane), and the flat list of its chunks into 16 equal
// contiguous ranges, one per warp, so every warp streams the same number of bytes; the next chunk's
// loads are in flight while the current one is multiplied (two independent FMA chains per lane).
// A warp's range covers a few rows: each row fragment leaves one lane partial, and the partials of
// 8 fragments are reduced together by a transposed butterfly (9 additions per lane for 8 sums);
// the fragment sums of a row are added in warp order. Every sum has a fixed order, so repeated
// solves give identical bits.
#include "kernels.h"
#include "mbpcg_device.cuh"
#include "tma.cuh"

namespace mbpcg {

namespace {

constexpr int kCgThreads = 512;
constexpr int kCgWarps = kCgThreads / 32;
constexpr int kSegD2 = 8;              // double2 loads per lane per item
constexpr int kSegCols = 64 * kSegD2;  // 512 columns per item
constexpr int kBatch = 8;              // row fragments per transposed warp reduction

__device__ __forceinline__ double2 ld_stream(const double* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(p), "l"(pol));
  return v;
}

// Loads of chunk c of the CTA's flat chunk list (row_local = c / cpr, columns 512 (c % cpr) + ...);
// zero past the matrix.
__device__ __forceinline__ void load_chunk(const double* __restrict__ A, int n, int r0, int cpr, int c, int lane,
                                           uint64_t pol, double2 (&buf)[kSegD2]) {
  const double* base = A + (size_t)(r0 + c / cpr) * n;
  const int col0 = (c % cpr) * kSegCols + 2 * lane;
#pragma unroll
  for (int j = 0; j < kSegD2; ++j) {
    const int col = col0 + 64 * j;
    buf[j] = col < n ? ld_stream(base + col, pol) : make_double2(0.0, 0.0);
  }
}

// Sums over the 32 lanes of the 8 values s[0..7] at once (transposed butterfly): afterwards lane L
// holds the sum of value q = bits 2..4 of L (returned in q), the same in the 4 lanes of a group.
__device__ __forceinline__ double butterfly8(double (&s)[kBatch], int lane, int& q) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double keep = b4 ? s[j + 4] : s[j], send = b4 ? s[j] : s[j + 4];
    s[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double keep = b3 ? s[j + 2] : s[j], send = b3 ? s[j] : s[j + 2];
    s[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  double t;
  {
    const double keep = b2 ? s[1] : s[0], send = b2 ? s[0] : s[1];
    t = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  q = (b2 ? 1 : 0) + (b3 ? 2 : 0) + (b4 ? 4 : 0);
  return t;
}

}  // namespace

// Most row fragments one warp's chunk range can meet: ceil(rows * cpr / 8) chunks span at most
// that many / cpr + 2 rows (rows = the most rows a CTA owns).
__host__ __device__ int cg_dense_fragments(int n, int nb) {
  const int rows = (n + nb - 1) / nb, cpr = (n + kSegCols - 1) / kSegCols;
  const int per_warp = (rows * cpr + kCgWarps - 1) / kCgWarps;
  return per_warp / cpr + 2;
}

__global__ void __launch_bounds__(kCgThreads, 1)
k_cg_dense_iter(int n, const double* __restrict__ A, CgVectors v, const double* __restrict__ wdiag,
                double* __restrict__ part, int pstride, unsigned int* __restrict__ counter, SolveState* st,
                cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(16) double cg_smem[];
  double* u = cg_smem;                      // r_j, the whole vector
  double* fsum = cg_smem + ((n + 1) & ~1);  // row-fragment sums, [warp][fragment]
  __shared__ double red[3 * kCgWarps];
  __shared__ int wrow[2 * kCgWarps];  // first and last local row of each warp's chunk range (empty: 1, 0)
  __shared__ int last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int it = st->it, par = it & 1;  // read with the done flag: one round trip for both
  const double alpha = st->cg_alpha, beta = st->cg_beta;
  if (st->done) {
    if (use_cond && blockIdx.x == 0 && tid == 0) cudaGraphSetConditional(cond, 0);
    return;
  }
  int r0, r1;
  row_range(n, r0, r1);
  const uint64_t pol = l2_policy_evict_first();
  const int cpr = (n + kSegCols - 1) / kSegCols;  // chunks per row
  const int nchunks = (r1 - r0) * cpr;
  const int fmax = cg_dense_fragments(n, gridDim.x);
  const int c0 = (int)((long long)nchunks * warp / kCgWarps), c1 = (int)((long long)nchunks * (warp + 1) / kCgWarps);
  if (lane == 0) {
    wrow[2 * warp] = c0 < c1 ? c0 / cpr : 1;
    wrow[2 * warp + 1] = c0 < c1 ? (c1 - 1) / cpr : 0;
  }
  // the first chunk's loads do not depend on r_j: issue them before the vector updates
  double2 bufA[kSegD2], bufB[kSegD2];
  if (c0 < c1) load_chunk(A, n, r0, cpr, c0, lane, pol, bufA);

  // 1. updates of iteration j-1; u = r_j (every CTA forms the whole vector: sharing the work
  // across a cluster costs more than it saves, since clusters of one CTA per SM do not all fit on
  // the GPU at once)
  const int n2 = n / 2;
  if (it == 0) {
    const double2* rv = reinterpret_cast<const double2*>(v.r[0]);
    for (int e = tid; e < n2; e += kCgThreads) reinterpret_cast<double2*>(u)[e] = __ldcg(rv + e);
  } else {
    const double* ro = v.r[par ^ 1];
    const double* wo = v.w[par ^ 1];
    const double* so = v.s[par];
    // batches of kUpd elements per thread, every load of a batch in flight before its arithmetic
    constexpr int kUpd = 4;
    for (int e0 = tid; e0 < n2; e0 += kUpd * kCgThreads) {
      double2 rr[kUpd], ww[kUpd], ss[kUpd];
#pragma unroll
      for (int b = 0; b < kUpd; ++b) {
        const int e = e0 + b * kCgThreads;
        if (e < n2) {
          rr[b] = __ldcg(reinterpret_cast<const double2*>(ro) + e);
          ww[b] = __ldcg(reinterpret_cast<const double2*>(wo) + e);
          ss[b] = __ldcg(reinterpret_cast<const double2*>(so) + e);
        }
      }
#pragma unroll
      for (int b = 0; b < kUpd; ++b) {
        const int e = e0 + b * kCgThreads;
        if (e < n2) {
          double2 r2;
          r2.x = fma(-alpha, fma(beta, ss[b].x, ww[b].x), rr[b].x);
          r2.y = fma(-alpha, fma(beta, ss[b].y, ww[b].y), rr[b].y);
          reinterpret_cast<double2*>(u)[e] = r2;
        }
      }
    }
    // own rows: p, s, x and r of iteration j (the same expressions as u above, so the same bits)
    double* rn = v.r[par];
    double* sn = v.s[par ^ 1];
    for (int l = r0 + tid; l < r1; l += kCgThreads) {
      const double rl0 = __ldcg(ro + l);
      const double sl = fma(beta, __ldcg(so + l), __ldcg(wo + l));
      const double pl = fma(beta, v.p[l], rl0);
      v.p[l] = pl;
      v.x[l] = fma(alpha, pl, v.x[l]);
      sn[l] = sl;
      rn[l] = fma(-alpha, sl, rl0);
    }
  }
  __syncthreads();

  // 2. w_j = A r_j on the own rows: chunks [c0, c1) of this warp, fragment sums into fsum
  {
    double acc0 = 0.0, acc1 = 0.0, v[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; ++q) v[q] = 0.0;
    int nf = 0, fbase = 0;  // fragments in the current batch, index of its first fragment
    auto consume = [&](int c, const double2(&buf)[kSegD2]) {
      const int col0 = (c % cpr) * kSegCols + 2 * lane;
#pragma unroll
      for (int j = 0; j < kSegD2; ++j) {
        const int col = col0 + 64 * j;
        const double2 uu = col < n ? *reinterpret_cast<const double2*>(u + col) : make_double2(0.0, 0.0);
        acc0 = fma(buf[j].x, uu.x, acc0);
        acc1 = fma(buf[j].y, uu.y, acc1);
      }
      if (c + 1 == c1 || (c + 1) % cpr == 0) {  // end of a row fragment
        const double f = acc0 + acc1;
#pragma unroll
        for (int q = 0; q < kBatch; ++q)
          if (q == nf) v[q] = f;
        acc0 = acc1 = 0.0;
        if (++nf == kBatch || c + 1 == c1) {
          int q;
          const double t = butterfly8(v, lane, q);
          if ((lane & 3) == 0 && q < nf) fsum[warp * fmax + fbase + q] = t;
#pragma unroll
          for (int k = 0; k < kBatch; ++k) v[k] = 0.0;
          fbase += nf;
          nf = 0;
        }
      }
    };
    for (int c = c0; c < c1; c += 2) {
      if (c + 1 < c1) load_chunk(A, n, r0, cpr, c + 1, lane, pol, bufB);
      consume(c, bufA);
      if (c + 1 >= c1) break;
      if (c + 2 < c1) load_chunk(A, n, r0, cpr, c + 2, lane, pol, bufA);
      consume(c + 1, bufB);
    }
  }
  __syncthreads();

  // 3. w_j on the own rows (fragment sums in warp order) and the CTA partials of the three sums
  double g = 0.0, dl = 0.0, nu = 0.0;
  for (int t = tid; t < r1 - r0; t += kCgThreads) {
    double w = 0.0;
#pragma unroll
    for (int wp = 0; wp < kCgWarps; ++wp) {  // warps whose chunk range meets row t, in warp order
      const int f0 = wrow[2 * wp];
      if (f0 <= t && t <= wrow[2 * wp + 1]) w += fsum[wp * fmax + t - f0];
    }
    const int row = r0 + t;
    v.w[par][row] = w;
    const double ri = u[row];
    g = fma(ri, ri, g);
    dl = fma(w, ri, dl);
    nu = (wdiag != nullptr) ? fma(ri * wdiag[row], ri, nu) : fma(ri, ri, nu);
  }
  // (FP64 instructions hold the unit for a whole warp slot: only warps that own rows reduce)
  const int rwarps = min(kCgWarps, (r1 - r0 + 31) / 32);
  if (warp < rwarps) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      g += __shfl_xor_sync(0xffffffffu, g, off);
      dl += __shfl_xor_sync(0xffffffffu, dl, off);
      nu += __shfl_xor_sync(0xffffffffu, nu, off);
    }
    if (lane == 0) {
      red[3 * warp] = g;
      red[3 * warp + 1] = dl;
      red[3 * warp + 2] = nu;
    }
  }
  __syncthreads();
  if (tid < 3) {
    double a = 0.0;
    for (int w = 0; w < rwarps; ++w) a += red[3 * w + tid];
    part[(size_t)blockIdx.x * pstride + tid] = a;
  }
  __syncthreads();

  // 4. the last CTA: fixed-order sum of the partials, the test and the scalars of iteration j
  if (tid == 0) {  // the arrival releases this CTA's partials (ordered before it by the barrier)
    unsigned int old;  // and acquires the other CTAs' ones
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(counter) : "memory");
    last = old == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  // warps 0, 1, 2 of the last CTA sum the partials of gamma, delta and ||D r||^2, one sum each (a
  // warp has one FP64 instruction in flight: three chains in one warp would run one after another),
  // each over the CTAs in lane-strided order and then a butterfly
  __shared__ double tot[3];
  if (warp < 3) {
    double a = 0.0;
    constexpr int kTail = 8;  // partials per lane loaded together (grids up to 256 CTAs in one batch)
    for (int q0 = lane; q0 < (int)gridDim.x; q0 += 32 * kTail) {
      double pv[kTail];
#pragma unroll
      for (int b = 0; b < kTail; ++b) {
        const int q = q0 + 32 * b;
        if (q < (int)gridDim.x) pv[b] = __ldcg(part + (size_t)q * pstride + warp);
      }
#pragma unroll
      for (int b = 0; b < kTail; ++b)
        if (q0 + 32 * b < (int)gridDim.x) a += pv[b];
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if (lane == 0) tot[warp] = warp == 2 ? sqrt(a) : a;  // the norm's root beside the other sums
  }
  __syncthreads();
  if (tid != 0) return;
  *counter = 0u;
  const double gamma = tot[0], delta = tot[1], nrm = tot[2];
  st->nu_h = nrm;
  st->ls_res = nrm;
  int cont = 0;
  if (nrm < st->tol_abs) {
    st->converged = 1;
    st->done = 1;
    st->status = 0;
  } else if (it >= st->maxit) {
    st->done = 1;
    st->status = 5;
  } else {
    double alpha, beta;
    if (it == 0) {
      beta = 0.0;
      alpha = gamma / delta;
    } else {
      beta = gamma / st->cg_gamma_old;
      alpha = gamma / (delta - beta * gamma / st->cg_alpha_old);
    }
    if (!isfinite(alpha) || !(alpha > 0.0)) {
      st->done = 1;
      st->status = 6;
    } else {
      st->cg_alpha = alpha;
      st->cg_beta = beta;
      st->cg_gamma_old = gamma;
      st->cg_alpha_old = alpha;
      st->it = it + 1;
      cont = 1;
    }
  }
  if (use_cond) cudaGraphSetConditional(cond, cont);
}

bool cg_dense_fused_ok(int n) { return n >= 2 && (n % 2) == 0 && n <= kCgDenseMaxN; }

int cg_dense_grid(int n, int sms) { return max(1, min(sms > 0 ? sms : 1, (n + 7) / 8)); }

size_t cg_dense_smem_bytes(int n, int nb) {
  return ((size_t)((n + 1) & ~1) + (size_t)kCgWarps * cg_dense_fragments(n, nb)) * sizeof(double);
}

cudaError_t cg_dense_configure(int n, int nb) {
  return cudaFuncSetAttribute(k_cg_dense_iter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)cg_dense_smem_bytes(n, nb));
}

void launch_cg_dense_iter(cudaStream_t s, int nb, int n, const double* A, const CgVectors& v, const double* wdiag,
                          double* part, int pstride, unsigned int* counter, SolveState* st,
                          cudaGraphConditionalHandle cond, int use_cond) {
  k_cg_dense_iter<<<nb, kCgThreads, cg_dense_smem_bytes(n, nb), s>>>(n, A, v, wdiag, part, pstride, counter, st,
                                                                    cond, use_cond);
}

}  // namespace mbpcg
