// Row-parallel kernels of Algorithm 1 (one template per padded block width KP).
//
// Each CTA owns a balanced contiguous range of rows and walks it in tiles; per-CTA partial sums
// of the k x k reductions go to part[blockIdx.x * pstride + ...] and are summed in a fixed order
// by k_reduce (small_kernels.cu). Every kernel that runs inside the iteration loop returns at
// once when the solve has finished (SolveState::done), so a CUDA-graph loop body costs nothing
// after convergence.
#pragma once
#include "mbpcg_device.cuh"
#include "tma.cuh"

namespace mbpcg {

// ------------------------------------------------------------------------------------------------
// Q = A P for CSR A (Algorithm 1, the A P^{i-1} product; the paper's dominant step, Table 2) and,
// when GRAM, the CTA partials of the upper triangle of P^T Q (the Gram that defines Xi), so that
// A P is never read back. Threads own CPT consecutive columns of a row; the row of P that a
// nonzero selects is KP*8 contiguous bytes, read with 16-byte vector loads.
template <int KP, bool GRAM>
__global__ void __launch_bounds__(kThreads)
k_spmm(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ av,
       const double* __restrict__ P, double* __restrict__ Q, double* __restrict__ part, int pstride,
       const SolveState* __restrict__ st) {
  using C = Cfg<KP>;
  using G = GramTile<KP>;
  if (st != nullptr && st->done) return;
  __shared__ __align__(16) double Xs[GRAM ? C::ROWS * KP : 2];
  __shared__ __align__(16) double Ys[GRAM ? C::ROWS * KP : 2];
  __shared__ __align__(16) double red[GRAM ? G::RED : 2];
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x;
  const int rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  G g;
  if constexpr (GRAM) g.init(tid);
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    double acc[C::CPT], pv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) acc[c] = pv[c] = 0.0;
    if (i < r1) {
      const int pe = __ldg(rp + i + 1);
#pragma unroll 4
      for (int p = __ldg(rp + i); p < pe; ++p) {
        const int col = __ldg(ci + p);
        const double a = __ldg(av + p);
        double x[C::CPT];
        ldv<C::CPT>(P + (size_t)col * KP + j0, x);
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
  if constexpr (GRAM) g.finish(red, part + (size_t)blockIdx.x * pstride);
}

// ------------------------------------------------------------------------------------------------
// Q = A P for dense symmetric A stored column-major (row i of A is column i, contiguous).
// One CTA per SM owns a balanced range of rows and walks it in passes of G rows. The reduction index
// l is split into chunks of LC: for each chunk the A rows (G x LC) and the P rows (LC x KP) are
// copied into shared memory by 1-D TMA bulk copies (cp.async.bulk) that complete on an mbarrier,
// STAGES chunks in flight, so HBM latency is hidden behind the FP64 FMAs. Each thread owns a
// TR x TC register tile of the output and a residue class of l (LS classes, summed at the end in a
// fixed order). Rows of odd length (n odd) break the 16-byte rule of bulk copies; then the same
// pipeline is filled with ordinary loads. Every mbarrier wait is bounded: on a timeout the CTA sets
// *err (if given), waits (bounded) for the copies it still has in flight, and returns.
template <int KP>
struct DenseCfg {
  static constexpr int G = 32;
  static constexpr int LC = 128;
  static constexpr int LDA = LC + 2;  // shared-memory row stride of the A tile (keeps 16-byte rows)
  static constexpr int STAGES = 3;
  static constexpr int TR = (KP <= 2) ? 1 : 2;
  static constexpr int TC = (KP == 1) ? 1 : 2;
  static constexpr int RT = G / TR;
  static constexpr int CT = KP / TC;
  static constexpr int LS = kThreads / (RT * CT);
  static constexpr int A_ELEMS = G * LDA;
  static constexpr int STAGE_ELEMS = A_ELEMS + LC * KP;
  static constexpr int RED_ELEMS = (LS > 1) ? LS * G * KP : 1;
  static constexpr size_t SMEM = (size_t)(STAGES * STAGE_ELEMS + RED_ELEMS) * sizeof(double) + STAGES * 8;
};

template <int KP>
__global__ void __launch_bounds__(kThreads, 1)
k_dense(int n, const double* __restrict__ A, const double* __restrict__ P, double* __restrict__ Q,
        const SolveState* __restrict__ st, int* __restrict__ err) {
  using D = DenseCfg<KP>;
  if (st != nullptr && st->done) return;
  extern __shared__ __align__(128) double dsm[];
  double* red = dsm + D::STAGES * D::STAGE_ELEMS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + D::RED_ELEMS);
  __shared__ int abort_flag;
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x;
  const int q = tid % D::LS, tile = tid / D::LS, ct = tile % D::CT, rt = tile / D::CT;
  const bool tma = (n % 2) == 0;
  if (tid == 0) {
    for (int s = 0; s < D::STAGES; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
    abort_flag = 0;
  }
  __syncthreads();
  const int nchunks = (n + D::LC - 1) / D::LC;
  int g_next = 0;  // global index of the next chunk to consume (stage = g % STAGES)
  for (int base = r0; base < r1; base += D::G) {
    const int rows = min(D::G, r1 - base);
    const int g0 = g_next;
    auto issue = [&](int c) {
      const int g = g0 + c, stage = g % D::STAGES, l0 = c * D::LC, lc = min(D::LC, n - l0);
      double* As = dsm + stage * D::STAGE_ELEMS;
      double* Ps = As + D::A_ELEMS;
      if (tma) {
        if (tid < 32) {
          if (tid == 0) mbar_arrive_expect_tx(&bars[stage], (uint32_t)((rows + KP) * lc * sizeof(double)));
          __syncwarp();
          for (int r = tid; r < rows; r += 32)
            tma_load_1d(As + r * D::LDA, A + (size_t)(base + r) * n + l0, (uint32_t)(lc * sizeof(double)),
                        &bars[stage]);
          if (tid == 0)
            tma_load_1d(Ps, P + (size_t)l0 * KP, (uint32_t)(lc * KP * sizeof(double)), &bars[stage]);
        }
      } else {
        for (int e = tid; e < rows * lc; e += kThreads) {
          const int r = e / lc, l = e - r * lc;
          As[r * D::LDA + l] = A[(size_t)(base + r) * n + l0 + l];
        }
        for (int e = tid; e < lc * KP; e += kThreads) Ps[e] = P[(size_t)l0 * KP + e];
      }
    };
    double acc[D::TR][D::TC];
#pragma unroll
    for (int r = 0; r < D::TR; ++r)
#pragma unroll
      for (int c = 0; c < D::TC; ++c) acc[r][c] = 0.0;
    const int pre = min(D::STAGES - 1, nchunks);
    for (int c = 0; c < pre; ++c) issue(c);
    int issued = pre;
    __syncthreads();
    for (int c = 0; c < nchunks; ++c) {
      if (c + D::STAGES - 1 < nchunks) {
        issue(c + D::STAGES - 1);
        issued = c + D::STAGES;
      }
      const int g = g0 + c, stage = g % D::STAGES;
      bool ok = true;
      if (tma) ok = mbar_wait_bounded(&bars[stage], (uint32_t)((g / D::STAGES) & 1));
      if (!ok) abort_flag = 1;
      if (ok && rt * D::TR < rows) {
        const double* As = dsm + stage * D::STAGE_ELEMS;
        const double* Ps = As + D::A_ELEMS;
        const int lc = min(D::LC, n - c * D::LC);
        for (int l = q; l < lc; l += D::LS) {
          double a[D::TR], p[D::TC];
#pragma unroll
          for (int r = 0; r < D::TR; ++r) a[r] = As[(rt * D::TR + r) * D::LDA + l];
          if constexpr (D::TC == 2) {
            const double2 t = *reinterpret_cast<const double2*>(Ps + l * KP + ct * 2);
            p[0] = t.x;
            p[1] = t.y;
          } else {
            p[0] = Ps[l * KP + ct];
          }
#pragma unroll
          for (int r = 0; r < D::TR; ++r)
#pragma unroll
            for (int cc = 0; cc < D::TC; ++cc) acc[r][cc] = fma(a[r], p[cc], acc[r][cc]);
        }
      }
      __syncthreads();
      if (abort_flag) {
        if (tid == 0) {
          if (err != nullptr) atomicExch(err, 1);
          for (int c2 = c; c2 < issued; ++c2) {  // drain the copies still in flight (bounded)
            const int g2 = g0 + c2;
            mbar_wait_bounded(&bars[g2 % D::STAGES], (uint32_t)((g2 / D::STAGES) & 1));
          }
        }
        __syncthreads();
        return;
      }
    }
    g_next = g0 + nchunks;
    // sum the LS residue classes in a fixed order, then store the valid rows
    if constexpr (D::LS > 1) {
#pragma unroll
      for (int r = 0; r < D::TR; ++r)
#pragma unroll
        for (int cc = 0; cc < D::TC; ++cc) red[(q * D::G + rt * D::TR + r) * KP + ct * D::TC + cc] = acc[r][cc];
      cta_tree_sum(red, D::LS, D::G * KP);
      for (int e = tid; e < rows * KP; e += kThreads) Q[(size_t)base * KP + e] = red[e];
      __syncthreads();
    } else {
#pragma unroll
      for (int r = 0; r < D::TR; ++r) {
        const int row = rt * D::TR + r;
        if (row < rows) {
#pragma unroll
          for (int cc = 0; cc < D::TC; ++cc) Q[(size_t)(base + row) * KP + ct * D::TC + cc] = acc[r][cc];
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// CTA partials of the upper triangle of X^T Y (used for the dense-A Gram P^T (A P), for
// R^T R of the set-up Cholesky QR, and for the exit Gram).
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_gram(int n, const double* __restrict__ X, const double* __restrict__ Y, double* __restrict__ part,
       int pstride, const SolveState* __restrict__ st) {
  using C = Cfg<KP>;
  using G = GramTile<KP>;
  if (st != nullptr && st->done) return;
  __shared__ __align__(16) double Xs[C::ROWS * KP];
  __shared__ __align__(16) double Ys[C::ROWS * KP];
  __shared__ __align__(16) double red[G::RED];
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
      ldv<C::CPT>(X + (size_t)i * KP + j0, xv);
      ldv<C::CPT>(Y + (size_t)i * KP + j0, yv);
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

// ------------------------------------------------------------------------------------------------
// Block update of Algorithm 1 with its three products given (computed on the tensor cores):
//   X~ += PT,  R -= QT,  V = W - QXi,
// with the same CTA partials as k_axpy (explicit residual): nu_j at part[NPACK + j] and the upper
// triangle of V^T V at part[0..).
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_axpy_pre(int n, const double* __restrict__ PT, const double* __restrict__ QT, const double* __restrict__ QXi,
           const double* __restrict__ W, double* __restrict__ R, double* __restrict__ Xt, double* __restrict__ V,
           const double* __restrict__ wdiag, double* __restrict__ part, int pstride, const SolveState* __restrict__ st) {
  using C = Cfg<KP>;
  using G = GramTile<KP>;
  constexpr int RED = (G::RED > C::ROWS * KP) ? G::RED : C::ROWS * KP;
  if (st->done) return;
  __shared__ __align__(16) double Vs[C::ROWS * KP];
  __shared__ __align__(16) double red[RED];
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  int r0, r1;
  row_range(n, r0, r1);
  G g;
  g.init(tid);
  double nu[C::CPT];
#pragma unroll
  for (int c = 0; c < C::CPT; ++c) nu[c] = 0.0;
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    double vv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) vv[c] = 0.0;
    if (i < r1) {
      const size_t o = (size_t)i * KP + j0;
      double xv[C::CPT], pt[C::CPT], rv[C::CPT], qt[C::CPT], qx[C::CPT];
      ldv_plain<C::CPT>(Xt + o, xv);
      ldv<C::CPT>(PT + o, pt);
      ldv_plain<C::CPT>(R + o, rv);
      ldv<C::CPT>(QT + o, qt);
      ldv<C::CPT>(W + o, vv);
      ldv<C::CPT>(QXi + o, qx);
#pragma unroll
      for (int c = 0; c < C::CPT; ++c) {
        xv[c] += pt[c];
        rv[c] -= qt[c];
        vv[c] -= qx[c];
      }
      stv<C::CPT>(Xt + o, xv);
      stv<C::CPT>(R + o, rv);
      stv<C::CPT>(V + o, vv);
      if (wdiag != nullptr) {
        const double w2 = __ldg(wdiag + i);
#pragma unroll
        for (int c = 0; c < C::CPT; ++c) nu[c] = fma(rv[c] * w2, rv[c], nu[c]);
      } else {  // the same bits as with w2 = 1, one FP64 product fewer per entry
#pragma unroll
        for (int c = 0; c < C::CPT; ++c) nu[c] = fma(rv[c], rv[c], nu[c]);
      }
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
  for (int c = 0; c < C::CPT; ++c) red[rl * KP + j0 + c] = nu[c];
  cta_tree_sum(red, C::ROWS, KP);
  for (int jj = tid; jj < KP; jj += kThreads) out[C::NPACK + jj] = red[jj];
}

// W/P update of Algorithm 1 with its products given: W = VZi, P = W + PZt, and the column
// exponents of the new P (atomicMax into emax, when given) for the tensor-core A P product.
// Element-parallel: the thread stride is a multiple of KP, so each thread stays on one column.
template <int KP>
__global__ void k_pw_pre(int n, const double* __restrict__ VZi, const double* __restrict__ PZt, double* __restrict__ W,
                         double* __restrict__ P, const SolveState* __restrict__ st, int* __restrict__ emax) {
  const size_t total = (size_t)n * KP, stride = (size_t)gridDim.x * blockDim.x;
  const size_t q0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  // the first element's loads go out with the solve state's (a skipped launch discards them)
  double w0 = q0 < total ? VZi[q0] : 0.0, z0 = q0 < total ? PZt[q0] : 0.0;
  if (st != nullptr && st->pw_skip) return;
  __shared__ int em[KP];
  if (threadIdx.x < KP) em[threadIdx.x] = 0;
  __syncthreads();
  int loc = 0;
  for (size_t q = q0; q < total; q += stride) {
    if (q != q0) {
      w0 = VZi[q];
      z0 = PZt[q];
    }
    const double w = w0, p = w + z0;
    W[q] = w;
    P[q] = p;
    loc = max(loc, (int)((__double_as_longlong(p) >> 52) & 0x7FF));
  }
  if (emax != nullptr) {
    atomicMax(&em[q0 % KP], loc);
    __syncthreads();
    if (threadIdx.x < KP) atomicMax(&emax[threadIdx.x], em[threadIdx.x]);
  }
}

// ------------------------------------------------------------------------------------------------
// Block update of Algorithm 1, one pass over the rows:
//   X~ += P T,  R -= (A P) T  with T = Xi Sigma;   V = W - (A P) Xi   (input of the Cholesky QR)
// plus CTA partials of nu_j = ||(D R)_j||^2 (the original-system residual norms used for the
// best-basis test, Section 1) at part[NPACK + j] and of the upper triangle of V^T V at part[0..).
// wdiag = diag(A) of the original matrix (D^2), or NULL without scaling.
// RFREE (implicit residual, R = W Sigma): R is neither read nor written and nu is not formed here;
// with scaling the CTA partials of V^T D^2 V go to part[NPACK + KP ...) instead (nu_j is then
// sigma_j^T (V^T D^2 V) sigma_j, since the new residual block is V Sigma).
template <int KP, bool RFREE>
__global__ void __launch_bounds__(kThreads)
k_axpy(int n, const double* __restrict__ P, const double* __restrict__ Q, const double* __restrict__ W,
       double* __restrict__ R, double* __restrict__ Xt, double* __restrict__ V,
       const double* __restrict__ Tg, const double* __restrict__ Xig, const double* __restrict__ wdiag,
       double* __restrict__ part, int pstride, const SolveState* __restrict__ st) {
  using C = Cfg<KP>;
  using G = GramTile<KP>;
  constexpr int RED = (G::RED > C::ROWS * KP) ? G::RED : C::ROWS * KP;
  if (st->done) return;
  __shared__ __align__(16) double Ts[KP * KP];
  __shared__ __align__(16) double Xis[KP * KP];
  __shared__ __align__(16) double Ps[C::ROWS * KP];
  __shared__ __align__(16) double Qs[C::ROWS * KP];
  __shared__ __align__(16) double Vs[C::ROWS * KP];
  __shared__ __align__(16) double Vws[RFREE ? C::ROWS * KP : 2];
  __shared__ __align__(16) double red[RED];
  const bool wgram = RFREE && wdiag != nullptr;
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  for (int q = tid; q < KP * KP; q += kThreads) {  // column-major in global -> row-major here
    const int l = q % KP, jj = q / KP;
    Ts[l * KP + jj] = Tg[q];
    Xis[l * KP + jj] = Xig[q];
  }
  int r0, r1;
  row_range(n, r0, r1);
  G g, g2;
  g.init(tid);
  if (wgram) g2.init(tid);
  double nu[C::CPT];
#pragma unroll
  for (int c = 0; c < C::CPT; ++c) nu[c] = 0.0;
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    const bool valid = i < r1;
    double pv[C::CPT], qv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) pv[c] = qv[c] = 0.0;
    if (valid) {
      ldv<C::CPT>(P + (size_t)i * KP + j0, pv);
      ldv<C::CPT>(Q + (size_t)i * KP + j0, qv);
    }
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) {
      Ps[rl * KP + j0 + c] = pv[c];
      Qs[rl * KP + j0 + c] = qv[c];
    }
    __syncthreads();
    double vv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) vv[c] = 0.0;
    double wi = 1.0;
    if (valid) {
      double xv[C::CPT], rv[C::CPT];
      ldv_plain<C::CPT>(Xt + (size_t)i * KP + j0, xv);
      if constexpr (!RFREE) ldv_plain<C::CPT>(R + (size_t)i * KP + j0, rv);
      ldv<C::CPT>(W + (size_t)i * KP + j0, vv);
#pragma unroll 8
      for (int l = 0; l < KP; ++l) {
        const double pl = Ps[rl * KP + l], ql = Qs[rl * KP + l];
#pragma unroll
        for (int c = 0; c < C::CPT; ++c) {
          const double t = Ts[l * KP + j0 + c];
          xv[c] = fma(pl, t, xv[c]);
          if constexpr (!RFREE) rv[c] = fma(-ql, t, rv[c]);
          vv[c] = fma(-ql, Xis[l * KP + j0 + c], vv[c]);
        }
      }
      stv<C::CPT>(Xt + (size_t)i * KP + j0, xv);
      stv<C::CPT>(V + (size_t)i * KP + j0, vv);
      if constexpr (!RFREE) {
        stv<C::CPT>(R + (size_t)i * KP + j0, rv);
        if (wdiag != nullptr) {
          const double w2 = __ldg(wdiag + i);
#pragma unroll
          for (int c = 0; c < C::CPT; ++c) nu[c] = fma(rv[c] * w2, rv[c], nu[c]);
        } else {
#pragma unroll
          for (int c = 0; c < C::CPT; ++c) nu[c] = fma(rv[c], rv[c], nu[c]);
        }
      } else if (wgram) {
        wi = __ldg(wdiag + i);
      }
    }
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) {
      Vs[rl * KP + j0 + c] = vv[c];
      if constexpr (RFREE) Vws[rl * KP + j0 + c] = wi * vv[c];
    }
    __syncthreads();
    g.accumulate(Vs, Vs, min(C::ROWS, r1 - base));
    if (wgram) g2.accumulate(Vws, Vs, min(C::ROWS, r1 - base));
    __syncthreads();
  }
  double* out = part + (size_t)blockIdx.x * pstride;
  g.finish(red, out);
  if constexpr (!RFREE) {
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) red[rl * KP + j0 + c] = nu[c];
    cta_tree_sum(red, C::ROWS, KP);
    for (int jj = tid; jj < KP; jj += kThreads) out[C::NPACK + jj] = red[jj];
  } else if (wgram) {
    g2.finish(red, out + C::NPACK + KP);
  }
}

// Exit of the implicit-residual mode: R = X Sigma (Sigma upper triangular, column-major KP x KP),
// X = V when the loop ended at a test or a breakdown of the zeta step (the residual block of the
// last iteration is V Sigma), X = W otherwise. Nothing is done when no iteration ran (R holds R^0).
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_rsig(int n, const double* __restrict__ V, const double* __restrict__ W, const double* __restrict__ Sg,
       double* __restrict__ R, const SolveState* __restrict__ st) {
  __shared__ double Ss[KP * KP];
  if (st->it == 0) return;
  const double* X = st->r_from_v ? V : W;
  for (int q = threadIdx.x; q < KP * KP; q += kThreads) Ss[q] = Sg[q];
  __syncthreads();
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
    double x[KP], r[KP];
    ldv<KP>(X + (size_t)i * KP, x);
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      double a = 0.0;
#pragma unroll
      for (int l = 0; l <= j; ++l) a = fma(x[l], Ss[l + j * KP], a);
      r[j] = a;
    }
    stv<KP>(R + (size_t)i * KP, r);
  }
}

// ------------------------------------------------------------------------------------------------
// Second half of the Cholesky QR and the search-block update of Algorithm 1:
//   W = V zeta^{-1}   (zeta upper triangular, its inverse precomputed by the k x k kernel)
//   P = W + P zeta^T  (SETP == false)   or   P = W  (SETP == true: the set-up P^0 = W^0)
// For KP >= 8 a thread owns columns j and KP-1-j of a row: the two triangular dot products then
// total KP+1 terms for every thread, so a warp never idles on a short triangle.
// emax != NULL (tensor-core product): also the largest biased exponent of every column of the new
// P, combined with atomicMax into emax (which the product has cleared), for the digit splitting.
template <int KP, bool SETP>
__global__ void __launch_bounds__(kThreads)
k_pw(int n, const double* __restrict__ V, double* __restrict__ W, double* __restrict__ P,
     const double* __restrict__ Zinvg, const double* __restrict__ Zg, const SolveState* __restrict__ st,
     int* __restrict__ emax) {
  using C = Cfg<KP>;
  if (st != nullptr && st->pw_skip) return;
  __shared__ __align__(16) double Zis[KP * KP];
  __shared__ __align__(16) double Zs[KP * KP];
  __shared__ int em[KP];
  const int tid = threadIdx.x;
  if (tid < KP) em[tid] = 0;
  auto bexp = [](double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); };
  for (int q = tid; q < KP * KP; q += kThreads) {
    const int l = q % KP, jj = q / KP;
    Zis[l * KP + jj] = Zinvg[q];
    Zs[l * KP + jj] = SETP ? 0.0 : Zg[q];
  }
  __syncthreads();
  int r0, r1;
  row_range(n, r0, r1);
  if constexpr (C::TPR == 1) {
    for (int i = r0 + tid; i < r1; i += kThreads) {
      double v[KP], w[KP];
      ldv<KP>(V + (size_t)i * KP, v);
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        double a = 0.0;
#pragma unroll
        for (int l = 0; l <= j; ++l) a = fma(v[l], Zis[l * KP + j], a);
        w[j] = a;
      }
      stv<KP>(W + (size_t)i * KP, w);
      if constexpr (SETP) {
        stv<KP>(P + (size_t)i * KP, w);
        if (emax != nullptr)
#pragma unroll
          for (int j = 0; j < KP; ++j) atomicMax(&em[j], bexp(w[j]));
      } else {
        double p[KP], pn[KP];
        ldv_plain<KP>(P + (size_t)i * KP, p);
#pragma unroll
        for (int j = 0; j < KP; ++j) {
          double a = w[j];
#pragma unroll
          for (int l = j; l < KP; ++l) a = fma(p[l], Zs[j * KP + l], a);
          pn[j] = a;
        }
        stv<KP>(P + (size_t)i * KP, pn);
        if (emax != nullptr)
#pragma unroll
          for (int j = 0; j < KP; ++j) atomicMax(&em[j], bexp(pn[j]));
      }
    }
  } else {
    __shared__ __align__(16) double Vs[C::ROWS * KP];
    __shared__ __align__(16) double Psm[C::ROWS * KP];
    const int rl = tid / C::TPR, g = tid % C::TPR;
    const int ja = g, jb = KP - 1 - g;
    for (int base = r0; base < r1; base += C::ROWS) {
      const int i = base + rl;
      const bool valid = i < r1;
      double v2[2] = {0.0, 0.0}, p2[2] = {0.0, 0.0};
      if (valid) {
        ldv<2>(V + (size_t)i * KP + 2 * g, v2);
        if constexpr (!SETP) ldv_plain<2>(P + (size_t)i * KP + 2 * g, p2);
      }
      Vs[rl * KP + 2 * g] = v2[0];
      Vs[rl * KP + 2 * g + 1] = v2[1];
      Psm[rl * KP + 2 * g] = p2[0];
      Psm[rl * KP + 2 * g + 1] = p2[1];
      __syncthreads();
      if (valid) {
        const double* vr = Vs + rl * KP;
        // W_ia = sum_{l<=ja} V_il Zi_l,ja ; W_ib = sum_{l<=jb} V_il Zi_l,jb   (KP+1 terms in total)
        double acc = 0.0, wa = 0.0;
#pragma unroll 4
        for (int t = 0; t <= KP; ++t) {
          const bool first = t <= ja;
          const int l = first ? t : t - ja - 1;
          const int col = first ? ja : jb;
          acc = fma(vr[l], Zis[l * KP + col], acc);
          if (t == ja) {
            wa = acc;
            acc = 0.0;
          }
        }
        const double wb = acc;
        W[(size_t)i * KP + ja] = wa;
        W[(size_t)i * KP + jb] = wb;
        if constexpr (SETP) {
          P[(size_t)i * KP + ja] = wa;
          P[(size_t)i * KP + jb] = wb;
          if (emax != nullptr) {
            atomicMax(&em[ja], bexp(wa));
            atomicMax(&em[jb], bexp(wb));
          }
        } else {
          // P_ia = W_ia + sum_{l>=ja} P_il Z_ja,l ; P_ib = W_ib + sum_{l>=jb} P_il Z_jb,l
          const double* pr = Psm + rl * KP;
          const int na = KP - ja;  // terms of column ja
          double acc2 = wa, pa = 0.0;
#pragma unroll 4
          for (int t = 0; t <= KP; ++t) {
            const bool first = t < na;
            const int l = first ? ja + t : jb + (t - na);
            const int row = first ? ja : jb;
            acc2 = fma(pr[l], Zs[row * KP + l], acc2);
            if (t == na - 1) {
              pa = acc2;
              acc2 = wb;
            }
          }
          P[(size_t)i * KP + ja] = pa;
          P[(size_t)i * KP + jb] = acc2;
          if (emax != nullptr) {
            atomicMax(&em[ja], bexp(pa));
            atomicMax(&em[jb], bexp(acc2));
          }
        }
      }
      __syncthreads();
    }
  }
  if (emax != nullptr) {
    __syncthreads();
    if (tid < KP && em[tid] > 0) atomicMax(&emax[tid], em[tid]);
  }
}

// ------------------------------------------------------------------------------------------------
// Set-up norms: bs = D^{-1} rhs (the scaled right-hand side of Section 1), and CTA partials of
// ||rhs||^2, ||bs||^2 and ||A U||_F^2 (for X0 = (||B||_F / ||A U||_F) U of Algorithm 1).
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_setup_norms(int n, const double* __restrict__ rhs, const double* __restrict__ d, double* __restrict__ bs,
              const double* __restrict__ AU, double* __restrict__ part, int pstride) {
  __shared__ double red[3 * kThreads];
  int r0, r1;
  row_range(n, r0, r1);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += kThreads) {
    const double b = rhs[i];
    const double v = (d != nullptr) ? d[i] * b : b;
    bs[i] = v;
    s0 = fma(b, b, s0);
    s1 = fma(v, v, s1);
    double au[KP];
    ldv<KP>(AU + (size_t)i * KP, au);
#pragma unroll
    for (int j = 0; j < KP; ++j) s2 = fma(au[j], au[j], s2);
  }
  red[threadIdx.x * 3] = s0;
  red[threadIdx.x * 3 + 1] = s1;
  red[threadIdx.x * 3 + 2] = s2;
  cta_tree_sum(red, kThreads, 3);
  if (threadIdx.x < 3) part[(size_t)blockIdx.x * pstride + threadIdx.x] = red[threadIdx.x];
}

// X0 = scale U;  X~ = 0;  R = B~ = bs 1^T - scale (A U)  (columns < s; padded columns stay 0);
// and the CTA partials of R^T R for the set-up Cholesky QR (W^0, Sigma^0 = qr(R^0)).
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_init(int n, int s, const double* __restrict__ U, const double* __restrict__ AU, const double* __restrict__ bs,
       double* __restrict__ X0, double* __restrict__ Xt, double* __restrict__ R, double* __restrict__ part,
       int pstride, const SolveState* __restrict__ st) {
  using C = Cfg<KP>;
  using G = GramTile<KP>;
  __shared__ __align__(16) double Rs[C::ROWS * KP];
  __shared__ __align__(16) double red[G::RED];
  const double scale = st->scale;
  int r0, r1;
  row_range(n, r0, r1);
  const int tid = threadIdx.x, rl = tid / C::TPR, j0 = (tid % C::TPR) * C::CPT;
  G g;
  g.init(tid);
  for (int base = r0; base < r1; base += C::ROWS) {
    const int i = base + rl;
    double rv[C::CPT];
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) rv[c] = 0.0;
    if (i < r1) {
      double u[C::CPT], au[C::CPT], x0[C::CPT], z[C::CPT];
      ldv<C::CPT>(U + (size_t)i * KP + j0, u);
      ldv<C::CPT>(AU + (size_t)i * KP + j0, au);
      const double b = bs[i];
#pragma unroll
      for (int c = 0; c < C::CPT; ++c) {
        x0[c] = scale * u[c];
        z[c] = 0.0;
        rv[c] = (j0 + c < s) ? fma(-scale, au[c], b) : 0.0;
      }
      stv<C::CPT>(X0 + (size_t)i * KP + j0, x0);
      stv<C::CPT>(Xt + (size_t)i * KP + j0, z);
      stv<C::CPT>(R + (size_t)i * KP + j0, rv);
    }
#pragma unroll
    for (int c = 0; c < C::CPT; ++c) Rs[rl * KP + j0 + c] = rv[c];
    __syncthreads();
    g.accumulate(Rs, Rs, min(C::ROWS, r1 - base));
    __syncthreads();
  }
  g.finish(red, part + (size_t)blockIdx.x * pstride);
}

// ------------------------------------------------------------------------------------------------
// Exit (least-squares combination of Section 2): CTA partials of the Gram of M = [rhs | D R] in
// the original metric: upper triangle of (DR)^T (DR) at [0, NPACK), rhs^T (DR)_j at NPACK + j,
// rhs^T rhs at NPACK + KP. sqd = sqrt(diag A) (= D), or NULL without scaling.
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_ls_gram(int n, const double* __restrict__ R, const double* __restrict__ rhs, const double* __restrict__ sqd,
          double* __restrict__ part, int pstride) {
  using C = Cfg<KP>;
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
      ldv<C::CPT>(R + (size_t)i * KP + j0, mv);
      const double di = (sqd != nullptr) ? sqd[i] : 1.0;
      const double b = rhs[i];
#pragma unroll
      for (int c = 0; c < C::CPT; ++c) {
        mv[c] *= di;
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

// x += D^{-1} (X~ + X0) c  (Algorithm 1: X = X~ + X0, x = X c, back to the original unknowns).
template <int KP>
__global__ void __launch_bounds__(kThreads)
k_combine(int n, int s, const double* __restrict__ Xt, const double* __restrict__ X0, const double* __restrict__ c,
          const double* __restrict__ d, double* __restrict__ x) {
  __shared__ double cs[KP];
  if (threadIdx.x < KP) cs[threadIdx.x] = (int)threadIdx.x < s ? c[threadIdx.x] : 0.0;
  __syncthreads();
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
    double xt[KP], x0[KP];
    ldv<KP>(Xt + (size_t)i * KP, xt);
    ldv<KP>(X0 + (size_t)i * KP, x0);
    double a = 0.0;
#pragma unroll
    for (int j = 0; j < KP; ++j) a = fma(xt[j] + x0[j], cs[j], a);
    x[i] += (d != nullptr) ? d[i] * a : a;
  }
}

// U[i][j] = 2 u01(seed, stream 1 + j, index i) - 1 for j < s, 0 in the padded columns.
template <int KP>
__global__ void k_gen_u(int n, int s, unsigned long long seed, double* __restrict__ U) {
  const size_t total = (size_t)n * KP;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q % KP);
    const size_t i = q / KP;
    U[q] = (j < s) ? 2.0 * splitmix_uniform01(seed, 1 + j, i) - 1.0 : 0.0;
  }
}

// Column-major n x s (leading dimension n) <-> row-major n x KP with zero padding.
template <int KP>
__global__ void k_from_colmajor(int n, int s, const double* __restrict__ src, double* __restrict__ dst) {
  const size_t total = (size_t)n * KP;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q % KP);
    const size_t i = q / KP;
    dst[q] = (j < s) ? src[(size_t)j * n + i] : 0.0;
  }
}
template <int KP>
__global__ void k_to_colmajor(int n, int s, const double* __restrict__ src, double* __restrict__ dst) {
  const size_t total = (size_t)n * s;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const size_t j = q / n, i = q % n;
    dst[q] = src[i * KP + j];
  }
}

}  // namespace mbpcg
