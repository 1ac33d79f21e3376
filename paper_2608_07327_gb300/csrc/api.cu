// Host runtime of the MBPCG library: handles, workspace layout, the CUDA-graph solve loop and the
// C ABI declared in include/mbpcg.h and include/mbpcg_kernels.h.
//
// A solve is one graph launch per inner solve: set-up kernels, a device-side WHILE conditional
// node whose body is one iteration of Algorithm 1 (the k x k kernel at the end of the body sets
// the loop condition), and the exit kernels (least-squares combination, x update, true residual).
// The host only reads the 200-byte solve state after each launch to decide on a true-residual
// restart.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>
#include <new>
#include <string>

#include "../../include/mbpcg.h"
#include "../../include/mbpcg_kernels.h"
#include "kernels.h"
#include "small_kernels.cuh"

using namespace mbpcg;

namespace {

thread_local std::string g_err;

int set_err(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return set_err(MBPCG_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

constexpr size_t kAlign = 256;
constexpr int kMixedRestarts = 12;       // refinement steps of the mixed-precision solve
constexpr int kTuneVariants = 11;        // FP32 A P launch shapes tried by the autotuner
constexpr int kTiledMinRows = 65536;     // smaller systems sit in L2 and keep the gather kernel
constexpr double kMixedInnerTol = 1e-5;  // smallest relative tolerance asked of an FP32 inner solve
constexpr int kBodyUnroll = 8;           // loop iterations per pass of the graph's WHILE node
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
// Runs of staged rows the workspace holds for a CSR plan (a stencil needs a few per tile; a
// matrix that needs more keeps the gather kernel).
inline size_t plan_runs_cap(long long nnz) { return (size_t)(nnz / 8 > 1024 ? nnz / 8 : 1024); }

struct Dims {
  int n, kp, nb, nb_dense, nbmax, pstride;
  long long nnz;
  int dense, algo, tc, sms;
  int mixed;  // MBPCG_MIXED_FP32: FP32 blocks and values in the inner solve
  int cg_fused;  // dense CG in one launch per iteration (k_cg_dense_iter)
  int nb_cg;     // its CTAs (a multiple of the cluster size)
};

int num_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

Dims make_dims(int n, long long nnz, int s, int algo, int dense, int sms) {
  Dims d;
  d.n = n;
  d.nnz = nnz;
  d.dense = dense;
  d.algo = algo;
  d.kp = (algo == MBPCG_ALGO_CG) ? 1 : padded_width(s);
  const int sm = sms > 0 ? sms : 1;
  // row kernels: at most 2 CTAs per SM, and at least 8 rows per CTA at KP = 32 (the FP64 block
  // updates are bound by the FP64 pipe and gain from more CTAs: dense n = 4096, s = 32, 157 against
  // 162 us per iteration) or 32 rows below (latency-bound: Poisson n = 4096, s = 4, 38 against 41)
  // Sparse systems: up to 8 CTAs per SM -- the CSR product and the row passes of a large sparse
  // system are bound by memory latency and bandwidth (diffusion 128^3, s = 1: the product takes 76 us
  // with 2 CTAs per SM, a latency chain per row with 16 warps per SM).
  const int rows_per_cta = d.kp >= 32 ? 8 : 32;
  const long long cap = dense ? 2LL * sm : 8LL * sm;
  long long want = ((long long)n + rows_per_cta - 1) / rows_per_cta;
  d.nb = (int)(want < cap ? (want > 0 ? want : 1) : cap);
  long long wd = ((long long)n + 7) / 8;
  d.nb_dense = (int)(wd < sm ? (wd > 0 ? wd : 1) : sm);
  d.nbmax = d.nb > d.nb_dense ? d.nb : d.nb_dense;
  d.pstride = (npack(d.kp) + d.kp + 1 + 3) / 4 * 4;
  d.tc = 0;
  d.mixed = 0;
  d.sms = sm;
  d.cg_fused = (dense && algo == MBPCG_ALGO_CG && cg_dense_fused_ok(n)) ? 1 : 0;
  d.nb_cg = d.cg_fused ? cg_dense_grid(n, sm) : 0;
  if (d.nb_cg > d.nbmax) d.nbmax = d.nb_cg;
  return d;
}

// Partial-sum slots of a solver handle also hold the weighted Gram V^T D^2 V of the
// implicit-residual mode (after the KP norms); the component entry points keep the narrower slots.
void widen_for_handle(Dims& d) { d.pstride = (2 * npack(d.kp) + d.kp + 1 + 3) / 4 * 4; }

// The FP32 row kernels of the mixed-precision inner solve are bound by memory latency and
// bandwidth, not by the FP64 pipe: they get up to 8 CTAs per SM instead of 2.
void apply_mixed(Dims& d) {
  d.mixed = 1;
  long long want = ((long long)d.n + 31) / 32;
  d.nb = (int)(want < 8LL * d.sms ? (want > 0 ? want : 1) : 8LL * d.sms);
  d.nbmax = d.nb > d.nb_dense ? d.nb : d.nb_dense;
}

// Byte offsets of every buffer inside one workspace.
struct Layout {
  size_t rp, ci, av, A, diag, d, sqd, b, rhs, bs, x;
  size_t U, X0, Xt, R, W, P, Q, V;    // MBPCG blocks, n x KP each
  size_t r, w, xb, p, sv;             // CG vectors
  size_t r2, w2, sv2, cnt;            // dense CG in one launch: second copies of r, w, s; arrival counter
  size_t part, red, small, st, flag;  // reductions, k x k matrices, control block
  size_t oz_a, oz_ea, oz_p, oz_ep, oz_q; // tensor-core product: digits of A and P, exponents, split sums
  size_t av32, wd32;                     // mixed precision: FP32 copies of the scaled values and of diag A
  size_t A32;                            // mixed precision, dense A: FP32 tiles (dense_f32_tiles_bytes)
  size_t xbest;                          // mixed precision: best iterate of the refinement loop
  size_t rp3;                            // tensor-core k x k-row products: 3 blocks n x KP (KP >= 16)
  size_t pl_cl, pl_rptr, pl_runs;        // CSR: the tiled product's plan (local columns, tiles, runs)
  size_t total;
};

// Tensor-core handles with KP = 16 or 32 run the k x k-row products of the loop on the tensor cores.
bool dm_uses_rowprod(const Dims& dm) { return dm.tc && dm.kp >= 16 && dm.algo == MBPCG_ALGO_MBPCG; }

Layout make_layout(const Dims& dm) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + (bytes > 0 ? bytes : 1));
    return at;
  };
  const size_t n = (size_t)dm.n;
  if (dm.dense) {
    L.A = take(n * n * sizeof(double));
    if (dm.mixed) {
      L.A32 = take(dense_f32_tiles_bytes(dm.n));
      L.wd32 = take(n * sizeof(float));
    }
  } else {
    L.rp = take((n + 1) * sizeof(int));
    L.ci = take((size_t)dm.nnz * sizeof(int));
    L.av = take((size_t)dm.nnz * sizeof(double));
    L.pl_cl = take((size_t)dm.nnz * sizeof(uint16_t));
    L.pl_rptr = take((n / 32 + 2) * sizeof(int));
    L.pl_runs = take(2 * plan_runs_cap(dm.nnz) * sizeof(int));
    if (dm.mixed) {
      L.av32 = take((size_t)dm.nnz * sizeof(float));
      L.wd32 = take(n * sizeof(float));
    }
  }
  L.diag = take(n * sizeof(double));
  L.d = take(n * sizeof(double));
  L.sqd = take(n * sizeof(double));
  L.b = take(n * sizeof(double));
  L.rhs = take(n * sizeof(double));
  L.bs = take(n * sizeof(double));
  L.x = take(n * sizeof(double));
  if (dm.mixed) L.xbest = take(n * sizeof(double));
  if (dm.algo == MBPCG_ALGO_MBPCG) {
    // Q and V are taken back to back: together they also stage a column-major n x s FP64 U
    const size_t blk = n * dm.kp * (dm.mixed ? sizeof(float) : sizeof(double));
    L.U = take(blk);
    L.X0 = take(blk);
    L.Xt = take(blk);
    L.R = take(blk);
    L.W = take(blk);
    L.P = take(blk);
    L.Q = take(blk);
    L.V = take(blk);
  } else {
    L.r = take(n * sizeof(double));
    L.w = take(n * sizeof(double));
    L.xb = take(n * sizeof(double));
    L.p = take(n * sizeof(double));
    L.sv = take(n * sizeof(double));
    if (dm.cg_fused) {
      L.r2 = take(n * sizeof(double));
      L.w2 = take(n * sizeof(double));
      L.sv2 = take(n * sizeof(double));
      L.cnt = take(sizeof(unsigned int));
    }
  }
  if (dm.tc) {
    L.oz_a = take(oz_a_tiles_bytes(dm.n));
    L.oz_ea = take(n * sizeof(int));
    L.oz_p = take(oz_p_chunks_bytes(dm.n, dm.kp));
    L.oz_ep = take(2 * kMaxKP * sizeof(int));  // the column exponents of P and the product's copy of them
    // raw partial sums of the product's slices: int64 and FP32 per entry
    L.oz_q = take((size_t)oz_ksplit(dm.n, dm.sms) * n * dm.kp * 2 * sizeof(long long));
    if (dm_uses_rowprod(dm)) L.rp3 = take(3 * n * dm.kp * sizeof(double));
  }
  L.part = take((size_t)dm.nbmax * dm.pstride * sizeof(double));
  L.red = take((size_t)dm.pstride * sizeof(double));
  L.small = take(8 * (size_t)kMaxKP * kMaxKP * sizeof(double));
  L.st = take(sizeof(SolveState));
  L.flag = take(sizeof(int));
  L.total = o;
  return L;
}

}  // namespace

struct mbpcg_ctx {
  Dims dm;
  int s, precond, algo, precision;
  unsigned long long seed;
  cudaStream_t stream;
  int own_stream;
  char* ws;
  int own_ws;
  Layout L;
  // device pointers
  int *rp, *ci, *flag;
  double *av, *A, *diag, *d, *sqd, *wdiag, *b, *rhs, *bs, *x, *xbest;
  double *U, *X0, *Xt, *R, *W, *P, *Q, *V;
  double *r, *w, *xb, *p, *sv;
  double *r2, *w2, *sv2;
  unsigned int* cg_cnt;
  double *part, *red;
  double *Sigma, *SigmaInv, *Xi, *T, *Zeta, *ZetaInv, *c, *Gtmp;
  SolveState* st;
  SolveState* st_host;  // host copy of the solve state (pageable: no device-wide synchronisation on free)
  uint8_t *oz_a, *oz_p;
  int *oz_ea, *oz_ep;
  double* oz_q;
  double* rp3;  // tensor-core k x k-row products (3 blocks), or NULL
  // mixed precision (FP32 views of the block buffers)
  float *fU, *fX0, *fXt, *fR, *fW, *fP, *fQ, *fV;
  float *av32, *wd32;
  float* A32;  // dense A in FP32 tiles
  cudaGraphExec_t exec;
  cudaGraphConditionalHandle cond;
  int graph_ready;
  int launch_mode;  // MBPCG_LAUNCH_GRAPH or MBPCG_LAUNCH_EAGER
  int rfree;        // MBPCG_RESIDUAL_IMPLICIT: R = W Sigma is not formed inside the loop
  // launch shape of the FP32 A P of the mixed inner solve, picked by autotune_spmm_f at create
  int spmm_unroll, spmm_ctas_per_sm, spmm_nb;
  float spmm_us[kTuneVariants];  // the measured shapes (0: not timed)
  int use_cond;     // 1 while the loop body is captured into the WHILE node
  SpmmPlan plan;    // CSR: rows of P staged per tile (see spmm_tiled.cu)
  int use_tiled;    // 1: the matrix has a tiling plan
  int plan_tried;   // 1: build_plan has run (a plan is built at most once)
  int prod64;       // the FP64 CSR product kernel: MBPCG_PRODUCT_CSR_GATHER or _TILED
  int round_once;   // tensor-core product: MBPCG_ROUND_ONCE (levels 5..8 exact) instead of the FP32 carry
  float spmm64_us[2];  // the FP64 product at create: gather and tiled kernels (0: not timed)
  cudaEvent_t e0, e1;
};

// A set of handles whose inner solves run as independent chains of one CUDA graph (one launch).
struct mbpcg_batch_ctx {
  std::vector<mbpcg_ctx*> h;
  cudaStream_t stream = nullptr;
  int own_stream = 0;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ready;  // one per member: its inputs are in place
  cudaEvent_t done = nullptr;      // the batch graph has finished
};

namespace {

template <typename T>
T* at(mbpcg_ctx* h, size_t off) {
  return reinterpret_cast<T*>(h->ws + off);
}

void bind(mbpcg_ctx* h) {
  const Layout& L = h->L;
  if (h->dm.dense) {
    h->A = at<double>(h, L.A);
    h->rp = nullptr;
    h->ci = nullptr;
    h->av = nullptr;
  } else {
    h->rp = at<int>(h, L.rp);
    h->ci = at<int>(h, L.ci);
    h->av = at<double>(h, L.av);
    h->A = nullptr;
  }
  h->diag = at<double>(h, L.diag);
  h->d = at<double>(h, L.d);
  h->sqd = at<double>(h, L.sqd);
  h->b = at<double>(h, L.b);
  h->rhs = at<double>(h, L.rhs);
  h->bs = at<double>(h, L.bs);
  h->x = at<double>(h, L.x);
  h->xbest = h->dm.mixed ? at<double>(h, L.xbest) : nullptr;
  if (h->algo == MBPCG_ALGO_MBPCG) {
    h->U = at<double>(h, L.U);
    h->X0 = at<double>(h, L.X0);
    h->Xt = at<double>(h, L.Xt);
    h->R = at<double>(h, L.R);
    h->W = at<double>(h, L.W);
    h->P = at<double>(h, L.P);
    h->Q = at<double>(h, L.Q);
    h->V = at<double>(h, L.V);
  } else {
    h->r = at<double>(h, L.r);
    h->w = at<double>(h, L.w);
    h->xb = at<double>(h, L.xb);
    h->p = at<double>(h, L.p);
    h->sv = at<double>(h, L.sv);
    if (h->dm.cg_fused) {
      h->r2 = at<double>(h, L.r2);
      h->w2 = at<double>(h, L.w2);
      h->sv2 = at<double>(h, L.sv2);
      h->cg_cnt = at<unsigned int>(h, L.cnt);
    }
  }
  h->part = at<double>(h, L.part);
  h->red = at<double>(h, L.red);
  double* sm = at<double>(h, L.small);
  const size_t q = (size_t)kMaxKP * kMaxKP;
  h->Sigma = sm;
  h->SigmaInv = sm + q;
  h->Xi = sm + 2 * q;
  h->T = sm + 3 * q;
  h->Zeta = sm + 4 * q;
  h->ZetaInv = sm + 5 * q;
  h->c = sm + 6 * q;
  h->Gtmp = sm + 7 * q;
  h->st = at<SolveState>(h, L.st);
  h->flag = at<int>(h, L.flag);
  if (h->dm.mixed) {
    h->fU = at<float>(h, L.U);
    h->fX0 = at<float>(h, L.X0);
    h->fXt = at<float>(h, L.Xt);
    h->fR = at<float>(h, L.R);
    h->fW = at<float>(h, L.W);
    h->fP = at<float>(h, L.P);
    h->fQ = at<float>(h, L.Q);
    h->fV = at<float>(h, L.V);
    h->av32 = h->dm.dense ? nullptr : at<float>(h, L.av32);
    h->wd32 = at<float>(h, L.wd32);
    h->A32 = h->dm.dense ? at<float>(h, L.A32) : nullptr;
  }
  if (h->dm.tc) {
    h->oz_a = at<uint8_t>(h, L.oz_a);
    h->oz_ea = at<int>(h, L.oz_ea);
    h->oz_p = at<uint8_t>(h, L.oz_p);
    h->oz_ep = at<int>(h, L.oz_ep);
    h->oz_q = at<double>(h, L.oz_q);
    h->rp3 = (dm_uses_rowprod(h->dm)) ? at<double>(h, L.rp3) : nullptr;
  }
}

int check_common(int n, int s, int precond, int algo, int precision, int mem) {
  if (n < 1) return set_err(MBPCG_ERR_INVALID, "n must be >= 1 (got %d)", n);
  if (algo != MBPCG_ALGO_MBPCG && algo != MBPCG_ALGO_CG) return set_err(MBPCG_ERR_INVALID, "unknown algo %d", algo);
  if (algo == MBPCG_ALGO_MBPCG && (s < 1 || s > 32)) return set_err(MBPCG_ERR_INVALID, "s must be in [1, 32] (got %d)", s);
  if (precond != MBPCG_PRECOND_NONE && precond != MBPCG_PRECOND_JACOBI)
    return set_err(MBPCG_ERR_INVALID, "unknown precond %d", precond);
  if (precision == MBPCG_MIXED_BF16)
    return set_err(MBPCG_ERR_INVALID, "MBPCG_MIXED_BF16 is reserved and not built (use MBPCG_FP64_TC for dense A)");
  if (precision != MBPCG_FP64 && precision != MBPCG_FP64_TC && precision != MBPCG_MIXED_FP32)
    return set_err(MBPCG_ERR_INVALID, "unsupported precision %d", precision);
  if (precision == MBPCG_MIXED_FP32 && algo != MBPCG_ALGO_MBPCG)
    return set_err(MBPCG_ERR_INVALID, "the mixed-precision inner solve is for MBPCG");
  if (mem != 0 && mem != 1) return set_err(MBPCG_ERR_INVALID, "mem must be 0 (host) or 1 (device)");
  return MBPCG_OK;
}

int alloc_handle(mbpcg_ctx** out, const Dims& dm, int s, int precond, int algo, int precision,
                 unsigned long long seed, void* workspace, size_t workspace_bytes, void* stream) {
  mbpcg_ctx* h = new (std::nothrow) mbpcg_ctx;
  if (!h) return set_err(MBPCG_ERR_OOM, "host allocation failed");
  std::memset(h, 0, sizeof(*h));
  h->dm = dm;
  h->s = (algo == MBPCG_ALGO_CG) ? 1 : s;
  h->precond = precond;
  h->algo = algo;
  h->precision = precision;
  h->seed = seed;
  h->L = make_layout(dm);
  *out = h;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    CUDA_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = 1;
  }
  if (workspace) {
    if (workspace_bytes < h->L.total)
      return set_err(MBPCG_ERR_OOM, "workspace of %zu bytes is smaller than the %zu bytes needed", workspace_bytes,
                     h->L.total);
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0)
      return set_err(MBPCG_ERR_INVALID, "workspace must be %zu-byte aligned", kAlign);
    h->ws = static_cast<char*>(workspace);
  } else {
    if (cudaMalloc(&h->ws, h->L.total) != cudaSuccess) {
      cudaGetLastError();
      h->ws = nullptr;
      return set_err(MBPCG_ERR_OOM, "cudaMalloc of %zu bytes failed", h->L.total);
    }
    h->own_ws = 1;
  }
  h->st_host = new (std::nothrow) SolveState;
  if (!h->st_host) return set_err(MBPCG_ERR_OOM, "host allocation failed");
  CUDA_TRY(cudaEventCreate(&h->e0));
  CUDA_TRY(cudaEventCreate(&h->e1));
  bind(h);
  CUDA_TRY(cudaMemsetAsync(h->ws, 0, h->L.total, h->stream));
  return MBPCG_OK;
}

void release(mbpcg_ctx* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph_ready) cudaGraphExecDestroy(h->exec);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  delete h->st_host;
  if (h->e0) cudaEventDestroy(h->e0);
  if (h->e1) cudaEventDestroy(h->e1);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int read_flag(mbpcg_ctx* h, int* flag) {
  CUDA_TRY(cudaMemcpyAsync(h->st_host, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  std::memcpy(flag, h->st_host, sizeof(int));
  return MBPCG_OK;
}

// Grid of the FP32 A P for `ctas_per_sm` CTAs per SM, at most one tile of rows per CTA.
int spmm_grid(const Dims& dm, int ctas_per_sm) {
  const int rows = rows_per_tile_f(dm.kp);
  const long long tiles = ((long long)dm.n + rows - 1) / rows, cap = (long long)ctas_per_sm * dm.sms;
  return (int)(tiles < cap ? tiles : cap);
}

// FP32 A P launch shapes tried by the autotuner, as (variant, CTAs per SM): variant 4 or 8 is the
// gather kernel (CTAs of 256 threads) with that many nonzeros of a row in flight per thread; 1 and
// 2 the wide-CTA kernel (spmm_wide.cu) with 1024 and 512 threads per CTA; 0 the tiled kernel
// (spmm_tiled.cu; rows of P staged per tile, two CTAs per SM, only with a tiling plan).
constexpr int kShapeUnroll[kTuneVariants] = {4, 4, 4, 8, 8, 8, 0, 1, 1, 2, 2};
constexpr int kShapeCtas[kTuneVariants] = {4, 8, 16, 4, 8, 16, 2, 1, 2, 2, 4};

int shape_grid(const mbpcg_ctx* h, int unroll, int ctas_per_sm) {
  if (unroll == 0) return std::min(h->plan.ntiles, 2 * h->dm.sms);
  if (unroll <= 2) {  // wide CTAs: 4 or 2 times the rows of a 256-thread CTA's pass
    const long long rows = (long long)rows_per_tile_f(h->dm.kp) * (unroll == 1 ? 4 : 2);
    const long long want = (h->dm.n + rows - 1) / rows, cap = (long long)ctas_per_sm * h->dm.sms;
    return (int)std::max(1LL, std::min(want, cap));
  }
  return spmm_grid(h->dm, ctas_per_sm);
}

void launch_spmm_f(mbpcg_ctx* h, int unroll, int nb, const float* X, float* Y, const SolveState* st) {
  const Dims& dm = h->dm;
  if (unroll == 0) spmm_tiled_f(h->stream, dm.kp, nb, dm.n, h->rp, h->av32, h->plan, X, Y, st);
  else if (unroll <= 2) spmm_wide_f(h->stream, dm.kp, unroll == 1 ? 1024 : 512, nb, dm.n, h->rp, h->ci, h->av32, X, Y, st);
  else row_ops_f(dm.kp)->spmm(h->stream, nb, dm.n, h->rp, h->ci, h->av32, X, Y, nullptr, 0, st, 0, unroll);
}

// Autotuner of the FP32 A P (the dominant kernel of the mixed inner solve): times every shape above
// on this handle's own matrix, three launches each after one untimed, and keeps the fastest. Every
// shape sums each row in the order of its nonzeros, so the choice changes the time, never the result.
int autotune_spmm_f(mbpcg_ctx* h) {
  float best = 1e30f;
  for (int v = 0; v < kTuneVariants; ++v) {
    h->spmm_us[v] = 0.f;
    if (kShapeUnroll[v] == 0 && !h->use_tiled) continue;
    const int nb = shape_grid(h, kShapeUnroll[v], kShapeCtas[v]);
    launch_spmm_f(h, kShapeUnroll[v], nb, h->fU, h->fQ, nullptr);
    CUDA_TRY(cudaEventRecord(h->e0, h->stream));
    for (int r = 0; r < 3; ++r) launch_spmm_f(h, kShapeUnroll[v], nb, h->fU, h->fQ, nullptr);
    CUDA_TRY(cudaEventRecord(h->e1, h->stream));
    CUDA_TRY(cudaEventSynchronize(h->e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, h->e0, h->e1));
    h->spmm_us[v] = ms * 1e3f / 3.f;
    if (h->spmm_us[v] < best) {
      best = h->spmm_us[v];
      h->spmm_unroll = kShapeUnroll[v];
      h->spmm_ctas_per_sm = kShapeCtas[v];
      h->spmm_nb = nb;
    }
  }
  return MBPCG_OK;
}

// The tiled product's plan (spmm_tiled.cu) for a validated CSR matrix of at least kTiledMinRows
// rows, when every tile's window fits and the runs fit the workspace; otherwise the handle keeps
// the gather kernel. The structure is read on the host (copied back when it was given on the device,
// or when row_ptr is NULL: the handle's own copy). Built at most once per handle.
int build_plan(mbpcg_ctx* h, const int* row_ptr, const int* col_idx, int mem) {
  const Dims& dm = h->dm;
  if (h->plan_tried) return MBPCG_OK;
  h->plan_tried = 1;
  h->use_tiled = 0;
  if (!row_ptr) mem = 1;
  if (dm.n < kTiledMinRows || dm.nnz < 1) return MBPCG_OK;
  std::vector<int> rp_h, ci_h;
  const int* rp = row_ptr;
  const int* ci = col_idx;
  if (mem) {
    rp_h.resize((size_t)dm.n + 1);
    ci_h.resize((size_t)dm.nnz);
    CUDA_TRY(cudaMemcpyAsync(rp_h.data(), h->rp, rp_h.size() * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(ci_h.data(), h->ci, ci_h.size() * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    rp = rp_h.data();
    ci = ci_h.data();
  }
  SpmmPlanHost ph;
  if (!spmm_plan_build(dm.n, rp, ci, dm.kp, dm.mixed ? sizeof(float) : sizeof(double), &ph)) return MBPCG_OK;
  if (ph.run_start.size() > plan_runs_cap(dm.nnz) || ph.ntiles + 1 > dm.n / 32 + 2) return MBPCG_OK;
  int* rptr = at<int>(h, h->L.pl_rptr);
  int* runs = at<int>(h, h->L.pl_runs);
  uint16_t* cl = at<uint16_t>(h, h->L.pl_cl);
  const size_t nr = ph.run_start.size();
  CUDA_TRY(cudaMemcpyAsync(rptr, ph.run_ptr.data(), ph.run_ptr.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(runs, ph.run_start.data(), nr * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(runs + nr, ph.run_len.data(), nr * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaMemcpyAsync(cl, ph.cl.data(), ph.cl.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
  h->plan.R = ph.R;
  h->plan.ntiles = ph.ntiles;
  h->plan.wmax = ph.wmax;
  h->plan.run_ptr = rptr;
  h->plan.run_start = runs;
  h->plan.run_len = runs + nr;
  h->plan.cl = cl;
  h->use_tiled = 1;
  return MBPCG_OK;
}

// The FP64 CSR product of the loop (with the Gram partials for MBPCG, as the loop launches it) timed
// with kernel v on the handle's own matrix, for the record (mbpcg_get_product_kernel): the gather
// kernel at create, the tiled kernel when its plan is built. Both sum each row of A P in the same
// order (the same bits); the tiled kernel groups the Gram partials by tile (other rounding). The
// gather kernel stays the loop's product -- it was the faster on every stencil measured, and a
// solve's result must not depend on a timing -- and the tiled kernel runs only when imposed.
void enqueue_product(mbpcg_ctx* h, const RowOps* ops, const double* X, double* Y, int gram, const SolveState* st);

int time_spmm64(mbpcg_ctx* h, int v) {
  const Dims& dm = h->dm;
  const RowOps* ops = row_ops(dm.kp);
  const int gram = h->algo == MBPCG_ALGO_MBPCG ? 1 : 0;
  const double* X = gram ? h->P : h->r;
  double* Y = gram ? h->Q : h->w;
  const int keep = h->prod64;
  CUDA_TRY(cudaMemsetAsync((void*)X, 0, (size_t)dm.n * dm.kp * sizeof(double), h->stream));
  h->prod64 = v;
  enqueue_product(h, ops, X, Y, gram, nullptr);
  CUDA_TRY(cudaEventRecord(h->e0, h->stream));
  for (int r = 0; r < 3; ++r) enqueue_product(h, ops, X, Y, gram, nullptr);
  CUDA_TRY(cudaEventRecord(h->e1, h->stream));
  CUDA_TRY(cudaEventSynchronize(h->e1));
  h->prod64 = keep;
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, h->e0, h->e1));
  h->spmm64_us[v] = ms * 1e3f / 3.f;
  return MBPCG_OK;
}

// Diagonal, scaling vectors and the in-place scaled matrix (Section 1).
int finish_create(mbpcg_ctx* h) {
  const int n = h->dm.n;
  const int g = (n + 255) / 256;
  CUDA_TRY(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
  const long long nvals = h->dm.dense ? (long long)n * n : h->dm.nnz;
  if (nvals > 0) k_check_finite<<<4 * h->dm.sms, 256, 0, h->stream>>>(nvals, h->dm.dense ? h->A : h->av, h->flag);
  if (h->dm.dense) k_diag_dense<<<g, 256, 0, h->stream>>>(n, h->A, h->diag, h->flag);
  else k_diag_csr<<<g, 256, 0, h->stream>>>(n, h->rp, h->ci, h->av, h->diag, h->flag);
  CUDA_TRY(cudaGetLastError());
  int flag = 0;
  int rc = read_flag(h, &flag);
  if (rc) return rc;
  if (flag & 4) return set_err(MBPCG_ERR_INVALID, "an entry of A is NaN or infinite");
  if (flag & 2) return set_err(MBPCG_ERR_NOT_SPD, "a diagonal entry of A is missing, not positive or not finite");
  if (h->precond == MBPCG_PRECOND_JACOBI) {
    k_make_scaling<<<g, 256, 0, h->stream>>>(n, h->diag, h->d, h->sqd);
    if (h->dm.dense) k_scale_dense<<<4 * h->dm.sms, 256, 0, h->stream>>>(n, h->A, h->d);
    else k_scale_csr<<<g, 256, 0, h->stream>>>(n, h->rp, h->ci, h->av, h->d);
    CUDA_TRY(cudaGetLastError());
    h->wdiag = h->diag;
  } else {
    h->d = nullptr;
    h->sqd = nullptr;
    h->wdiag = nullptr;
  }
  if (h->dm.mixed) {
    if (h->dm.dense) k_dense_to_f32_tiles<<<4 * h->dm.sms, 256, 0, h->stream>>>(n, h->A, h->A32);
    else k_to_f32<<<1024, 256, 0, h->stream>>>((long long)h->dm.nnz, h->av, h->av32);
    if (h->wdiag != nullptr) k_to_f32<<<(n + 255) / 256, 256, 0, h->stream>>>(n, h->wdiag, h->wd32);
    else h->wd32 = nullptr;
    CUDA_TRY(cudaGetLastError());
    if (!h->dm.dense) {
      h->spmm_unroll = 8;
      h->spmm_ctas_per_sm = 8;
      h->spmm_nb = spmm_grid(h->dm, 8);
      int rc = autotune_spmm_f(h);
      if (rc) return rc;
    }
  }
  // (a mixed handle's loop has no FP64 product: mbpcg_apply_dev alone reaches it, by the gather kernel)
  if (!h->dm.dense && !h->dm.mixed) {
    h->prod64 = MBPCG_PRODUCT_CSR_GATHER;
    int rc = time_spmm64(h, MBPCG_PRODUCT_CSR_GATHER);
    if (rc) return rc;
  }
  if (h->dm.cg_fused) CUDA_TRY(cg_dense_configure(n, h->dm.nb_cg));
  if (h->dm.tc) {
    oz_prepare_a(h->stream, n, h->A, h->oz_ea, h->oz_a);
    CUDA_TRY(cudaMemsetAsync(h->oz_p, 0, oz_p_chunks_bytes(n, h->dm.kp), h->stream));
    // the split sum reads every slice of the partials buffer (those past a tile's count unused)
    CUDA_TRY(cudaMemsetAsync(h->oz_q, 0, (size_t)oz_ksplit(n, h->dm.sms) * n * h->dm.kp * 2 * sizeof(long long),
                             h->stream));
    CUDA_TRY(cudaGetLastError());
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return MBPCG_OK;
}

// ------------------------------------------------------------------------------- graph building

void enqueue_product(mbpcg_ctx* h, const RowOps* ops, const double* X, double* Y, int gram, const SolveState* st) {
  const Dims& dm = h->dm;
  if (dm.dense && dm.tc) {
    // the loop's product reads P, whose column exponents the W/P update has already formed
    oz_product(h->stream, dm.n, dm.kp, dm.sms, h->oz_a, h->oz_ea, X, h->oz_p, h->oz_ep, h->oz_q, Y, &h->st->kerr, st,
               gram ? h->part : nullptr, dm.pstride, dm.nb, X == h->P ? 1 : 0, h->round_once);
  } else if (dm.dense) {
    ops->dense(h->stream, dm.nb_dense, dm.n, h->A, X, Y, st, &h->st->kerr);
    if (gram) ops->gram(h->stream, dm.nb, dm.n, X, Y, h->part, dm.pstride, st);
  } else if (h->prod64 == MBPCG_PRODUCT_CSR_TILED) {
    spmm_tiled(h->stream, dm.kp, dm.nb, dm.n, h->rp, h->av, h->plan, X, Y, h->part, dm.pstride, st, gram);
  } else {
    ops->spmm(h->stream, dm.nb, dm.n, h->rp, h->ci, h->av, X, Y, h->part, dm.pstride, st, gram);
  }
}

void enqueue_reduce(mbpcg_ctx* h, int nent, const SolveState* st) {
  launch_reduce(h->stream, h->part, h->dm.nb, h->dm.pstride, h->red, nent, st);
}

void enqueue_true_residual(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  if (dm.dense)
    k_resid_dense<<<dm.nb_dense, kThreads, 0, h->stream>>>(dm.n, h->A, h->sqd, h->b, h->x, h->rhs, h->part, dm.pstride);
  else
    k_resid_csr<<<dm.nb, kThreads, 0, h->stream>>>(dm.n, h->rp, h->ci, h->av, h->sqd, h->b, h->x, h->rhs, h->part,
                                                   dm.pstride);
  // the dense residual uses nb_dense partial slots
  launch_reduce(h->stream, h->part, dm.dense ? dm.nb_dense : dm.nb, dm.pstride, h->red, 1, nullptr);
  k_small_true<<<1, 1, 0, h->stream>>>(h->st, h->red);
}

void enqueue_mbpcg_setup(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  const RowOps* ops = row_ops(dm.kp);
  const int kp = dm.kp, n = dm.n;
  enqueue_product(h, ops, h->U, h->Q, 0, nullptr);  // A U
  ops->setup_norms(h->stream, dm.nb, n, h->rhs, h->d, h->bs, h->Q, h->part, dm.pstride);
  enqueue_reduce(h, 3, nullptr);
  k_small_setup<<<1, 1, 0, h->stream>>>(h->st, h->red);
  ops->init(h->stream, dm.nb, n, h->s, h->U, h->Q, h->bs, h->X0, h->Xt, h->R, h->part, dm.pstride, h->st);
  enqueue_reduce(h, npack(kp), nullptr);
  launch_small_sigma(h->stream, kp, h->st, h->red, h->Sigma, h->SigmaInv);
  ops->pw(h->stream, dm.nb, n, h->R, h->W, h->P, h->SigmaInv, nullptr, nullptr, 1, dm.tc ? h->oz_ep : nullptr);
}

void enqueue_mbpcg_body(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  const RowOps* ops = row_ops(dm.kp);
  const int kp = dm.kp, n = dm.n;
  // tensor-core handles at KP >= 16: the k x k-row products of the two row passes on the tensor cores
  const bool tcrows = h->rp3 != nullptr && !h->rfree;
  double *Y0 = h->rp3, *Y1 = Y0 + (size_t)n * kp, *Y2 = Y1 + (size_t)n * kp;
  enqueue_product(h, ops, h->P, h->Q, 1, h->st);
  enqueue_reduce(h, npack(kp), h->st);
  launch_small_xi(h->stream, kp, h->st, h->red, h->Sigma, h->Xi, h->T);
  if (tcrows) {
    const RowProdJobs jb = {{{h->P, h->T, 0, Y0}, {h->Q, h->T, 0, Y1}, {h->Q, h->Xi, 0, Y2}}};
    rowprod_tc(h->stream, n, kp, jb, 3, h->st, 0, &h->st->kerr);
    ops->axpy_pre(h->stream, dm.nb, n, Y0, Y1, Y2, h->W, h->R, h->Xt, h->V, h->wdiag, h->part, dm.pstride, h->st);
  } else {
    ops->axpy(h->stream, dm.nb, n, h->P, h->Q, h->W, h->R, h->Xt, h->V, h->T, h->Xi, h->wdiag, h->part, dm.pstride,
              h->st, h->rfree);
  }
  if (h->rfree) {  // nu_j from the Gram of V (weighted with scaling) and Sigma
    const bool w = h->wdiag != nullptr;
    enqueue_reduce(h, w ? 2 * npack(kp) + kp : npack(kp), h->st);
    k_small_nu<<<kp, 32, 0, h->stream>>>(h->st, h->red, h->Sigma, kp, w ? npack(kp) + kp : 0);
  } else {
    enqueue_reduce(h, npack(kp) + kp, h->st);
  }
  launch_small_zeta(h->stream, kp, h->st, h->red, h->Sigma, h->Zeta, h->ZetaInv, h->cond, h->use_cond);
  if (tcrows) {
    const RowProdJobs jb = {{{h->V, h->ZetaInv, 0, Y0}, {h->P, h->Zeta, 1, Y1}, {nullptr, nullptr, 0, nullptr}}};
    rowprod_tc(h->stream, n, kp, jb, 2, h->st, 1, &h->st->kerr);
    ops->pw_pre(h->stream, n, Y0, Y1, h->W, h->P, h->st, h->oz_ep);
  } else {
    ops->pw(h->stream, dm.nb, n, h->V, h->W, h->P, h->ZetaInv, h->Zeta, h->st, 0, dm.tc ? h->oz_ep : nullptr);
  }
}

void enqueue_mbpcg_exit(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  const RowOps* ops = row_ops(dm.kp);
  const int kp = dm.kp, n = dm.n;
  if (h->rfree) ops->rsig(h->stream, dm.nb, n, h->V, h->W, h->Sigma, h->R, h->st);
  ops->ls_gram(h->stream, dm.nb, n, h->R, h->rhs, h->sqd, h->part, dm.pstride);
  enqueue_reduce(h, npack(kp) + kp + 1, nullptr);
  k_small_ls<<<1, kSmallThreads, 0, h->stream>>>(h->st, h->red, kp, h->c);
  ops->combine(h->stream, dm.nb, n, h->s, h->Xt, h->X0, h->c, h->d, h->x);
  enqueue_true_residual(h);
}

// Mixed precision (MBPCG_MIXED_FP32): the same steps with the FP32 row kernels; the reductions,
// the k x k steps, the exit combination and the true residual stay as above.
void enqueue_product_f(mbpcg_ctx* h, const RowOpsF* ops, const float* X, float* Y, const SolveState* st) {
  const Dims& dm = h->dm;
  if (dm.dense) dense_f32_product(h->stream, dm.kp, dm.n, dm.sms, h->A32, X, Y, st);
  else launch_spmm_f(h, h->spmm_unroll, h->spmm_nb, X, Y, st);
}

void enqueue_mbpcg_setup_f(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  const RowOpsF* ops = row_ops_f(dm.kp);
  const int kp = dm.kp, n = dm.n;
  enqueue_product_f(h, ops, h->fU, h->fQ, nullptr);  // A U
  ops->setup_norms(h->stream, dm.nb, n, h->rhs, h->d, h->bs, h->fQ, h->part, dm.pstride);
  enqueue_reduce(h, 3, nullptr);
  k_small_setup<<<1, 1, 0, h->stream>>>(h->st, h->red);
  ops->init(h->stream, dm.nb, n, h->s, h->fU, h->fQ, h->bs, h->fX0, h->fXt, h->fR, h->part, dm.pstride, h->st);
  enqueue_reduce(h, npack(kp), nullptr);
  launch_small_sigma(h->stream, kp, h->st, h->red, h->Sigma, h->SigmaInv);
  ops->pw(h->stream, dm.nb, n, h->fR, h->fW, h->fP, h->SigmaInv, nullptr, nullptr, 1);
}

void enqueue_mbpcg_body_f(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  const RowOpsF* ops = row_ops_f(dm.kp);
  const int kp = dm.kp, n = dm.n;
  enqueue_product_f(h, ops, h->fP, h->fQ, h->st);
  ops->gram(h->stream, dm.nb, n, h->fP, h->fQ, h->part, dm.pstride, h->st);
  enqueue_reduce(h, npack(kp), h->st);
  launch_small_xi(h->stream, kp, h->st, h->red, h->Sigma, h->Xi, h->T);
  ops->axpy(h->stream, dm.nb, n, h->fP, h->fQ, h->fW, h->fR, h->fXt, h->fV, h->T, h->Xi, h->wd32, h->part,
            dm.pstride, h->st);
  enqueue_reduce(h, npack(kp) + kp, h->st);
  launch_small_zeta(h->stream, kp, h->st, h->red, h->Sigma, h->Zeta, h->ZetaInv, h->cond, h->use_cond);
  ops->pw(h->stream, dm.nb, n, h->fV, h->fW, h->fP, h->ZetaInv, h->Zeta, h->st, 0);
}

void enqueue_mbpcg_exit_f(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  const RowOpsF* ops = row_ops_f(dm.kp);
  const int kp = dm.kp, n = dm.n;
  ops->ls_gram(h->stream, dm.nb, n, h->fR, h->rhs, h->sqd, h->part, dm.pstride);
  enqueue_reduce(h, npack(kp) + kp + 1, nullptr);
  k_small_ls<<<1, kSmallThreads, 0, h->stream>>>(h->st, h->red, kp, h->c);
  ops->combine(h->stream, dm.nb, n, h->s, h->fXt, h->fX0, h->c, h->d, h->x);
  enqueue_true_residual(h);
}

void enqueue_cg_setup(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  k_cg_init<<<dm.nb, kThreads, 0, h->stream>>>(dm.n, h->rhs, h->d, h->r, h->xb, h->p, h->sv, h->part, dm.pstride);
  if (dm.cg_fused) {  // s_{-1} = 0 in the second copy; the arrival counter starts at zero
    cudaMemsetAsync(h->sv2, 0, (size_t)dm.n * sizeof(double), h->stream);
    cudaMemsetAsync(h->cg_cnt, 0, sizeof(unsigned int), h->stream);
  }
  enqueue_reduce(h, 1, nullptr);
  k_small_cg_setup<<<1, 1, 0, h->stream>>>(h->st, h->red);
}

void enqueue_cg_body(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  if (dm.cg_fused) {
    const CgVectors v = {{h->r, h->r2}, {h->w, h->w2}, {h->sv, h->sv2}, h->p, h->xb};
    launch_cg_dense_iter(h->stream, dm.nb_cg, dm.n, h->A, v, h->wdiag, h->part, dm.pstride, h->cg_cnt, h->st,
                         h->cond, h->use_cond);
    return;
  }
  const RowOps* ops = row_ops(1);
  enqueue_product(h, ops, h->r, h->w, 0, h->st);  // w = A u, u = r
  k_cg_dots<<<dm.nb, kThreads, 0, h->stream>>>(dm.n, h->r, h->w, h->wdiag, h->part, dm.pstride, h->st);
  enqueue_reduce(h, 3, h->st);
  k_small_cg<<<1, 1, 0, h->stream>>>(h->st, h->red, h->cond, h->use_cond);
  k_cg_update<<<dm.nb, kThreads, 0, h->stream>>>(dm.n, h->r, h->w, h->xb, h->p, h->sv, h->st);
}

void enqueue_cg_exit(mbpcg_ctx* h) {
  const Dims& dm = h->dm;
  k_cg_finish<<<dm.nb, kThreads, 0, h->stream>>>(dm.n, h->xb, h->d, h->x);
  enqueue_true_residual(h);
}

// Captures one inner solve of the handle -- set-up, a WHILE node over the loop body, exit -- into
// g, as a chain of its own (no dependency on what g already holds). The loop condition is created
// on g and stored in *cond; the captured kernels carry it.
cudaError_t capture_solve(mbpcg_ctx* h, cudaGraph_t g, cudaGraphConditionalHandle* cond) {
  cudaError_t e = cudaGraphConditionalHandleCreate(cond, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  const cudaGraphConditionalHandle own = h->cond;
  h->cond = *cond;
  const bool cg = h->algo == MBPCG_ALGO_CG;
  e = cudaStreamBeginCaptureToGraph(h->stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    if (cg) enqueue_cg_setup(h);
    else if (h->dm.mixed) enqueue_mbpcg_setup_f(h);
    else enqueue_mbpcg_setup(h);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
    cudaGraphNode_t cnode = nullptr;
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) {
      cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
      np.conditional.handle = *cond;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      e = cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &np);
      if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(h->stream, &cnode, nullptr, 1,
                                                                  cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
      if (cg) enqueue_cg_exit(h);
      else if (h->dm.mixed) enqueue_mbpcg_exit_f(h);
      else enqueue_mbpcg_exit(h);
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &captured);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) {
      e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        // kBodyUnroll iterations per pass of the WHILE node: a pass costs ~3 us of its own on
        // this GPU, on top of ~1 us per kernel; every loop kernel returns at once after the
        // iteration in which the solve stopped, and the last one of a pass sets the condition
        h->use_cond = 1;
        for (int u = 0; u < kBodyUnroll; ++u) {
          if (cg) enqueue_cg_body(h);
          else if (h->dm.mixed) enqueue_mbpcg_body_f(h);
          else enqueue_mbpcg_body(h);
        }
        h->use_cond = 0;
        cudaGraph_t b2 = nullptr;
        e = cudaStreamEndCapture(h->stream, &b2);
      }
    }
  }
  h->cond = own;
  return e;
}

int build_graph(mbpcg_ctx* h) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond{};
  cudaError_t e = capture_solve(h, g, &cond);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(MBPCG_ERR_CUDA, "building the solve graph failed: %s", cudaGetErrorString(e));
  }
  h->cond = cond;
  h->graph_ready = 1;
  return MBPCG_OK;
}

// One inner solve with ordinary launches (no graph): set-up, the loop body until the state says
// done (checked every 16 iterations), exit. Same kernels as the graph; used for profiling, since
// profilers do not see kernel nodes inside graphs that have conditional nodes.
int run_eager(mbpcg_ctx* h, int maxit_inner) {
  const bool cg = h->algo == MBPCG_ALGO_CG;
  h->use_cond = 0;
  if (cg) enqueue_cg_setup(h);
  else if (h->dm.mixed) enqueue_mbpcg_setup_f(h);
    else enqueue_mbpcg_setup(h);
  CUDA_TRY(cudaGetLastError());
  for (int i = 0; i < maxit_inner + 1; ++i) {
    if (cg) enqueue_cg_body(h);
    else if (h->dm.mixed) enqueue_mbpcg_body_f(h);
        else enqueue_mbpcg_body(h);
    CUDA_TRY(cudaGetLastError());
    if ((i & 15) == 15 || i == maxit_inner) {
      CUDA_TRY(cudaMemcpyAsync(h->st_host, h->st, sizeof(SolveState), cudaMemcpyDeviceToHost, h->stream));
      CUDA_TRY(cudaStreamSynchronize(h->stream));
      if (h->st_host->done) break;
    }
  }
  if (cg) enqueue_cg_exit(h);
  else if (h->dm.mixed) enqueue_mbpcg_exit_f(h);
      else enqueue_mbpcg_exit(h);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

// The host side of one solve: the true-residual restart loop (FP64) or the refinement loop (mixed
// precision) around the inner solves.
struct SolveLoop {
  double tol = 0.0, tol_rel = 0.0, best_relres = INFINITY;  // best_relres: mixed precision, of xbest
  int maxit = 0, no_test = 0, total = 0, restarts = 0, max_restarts = 0, status = MBPCG_OK;
  SolveState s{};
};

// Checks the arguments, builds the graph if needed, copies b and U in (mem: 0 host, 1 device) and
// sets up the loop's variables.
int solve_begin(mbpcg_ctx* h, const double* b, const double* U, double tol, int maxit, const double* x_out,
                int mem, int no_test, SolveLoop* L) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (!b || (!x_out && !no_test)) return set_err(MBPCG_ERR_INVALID, "b and x_out must not be NULL");
  if (!(tol > 0.0) || tol != tol) return set_err(MBPCG_ERR_INVALID, "tol must be a positive number");
  if (maxit < 1 && !no_test) return set_err(MBPCG_ERR_INVALID, "maxit must be >= 1");
  const int n = h->dm.n;
  const size_t nb = (size_t)n * sizeof(double);
  const cudaMemcpyKind in_kind = mem ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!h->graph_ready && h->launch_mode == MBPCG_LAUNCH_GRAPH) {
    int rc = build_graph(h);
    if (rc) return rc;
  }
  CUDA_TRY(cudaEventRecord(h->e0, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->b, b, nb, in_kind, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->rhs, h->b, nb, cudaMemcpyDeviceToDevice, h->stream));
  CUDA_TRY(cudaMemsetAsync(h->x, 0, nb, h->stream));
  if (h->algo == MBPCG_ALGO_MBPCG && h->dm.mixed) {
    const RowOpsF* ops = row_ops_f(h->dm.kp);
    if (U) {
      // stage the column-major FP64 block across the A P and V buffers (2 n KP floats >= n s doubles)
      double* stage = reinterpret_cast<double*>(h->fQ);
      CUDA_TRY(cudaMemcpyAsync(stage, U, nb * h->s, in_kind, h->stream));
      ops->from_colmajor(h->stream, n, h->s, stage, h->fU);
    } else {
      ops->gen_u(h->stream, n, h->s, h->seed, h->fU);
    }
    CUDA_TRY(cudaGetLastError());
  } else if (h->algo == MBPCG_ALGO_MBPCG) {
    const RowOps* ops = row_ops(h->dm.kp);
    if (U) {
      // stage the column-major block in the A P buffer, then widen to row-major KP
      CUDA_TRY(cudaMemcpyAsync(h->Q, U, nb * h->s, in_kind, h->stream));
      ops->from_colmajor(h->stream, n, h->s, h->Q, h->U);
    } else {
      ops->gen_u(h->stream, n, h->s, h->seed, h->U);
    }
    CUDA_TRY(cudaGetLastError());
  }
  // FP64 inner solves: at most 3 true-residual restarts. Mixed precision: the restarts are the FP64
  // refinement loop (correction solves in FP32), at most kMixedRestarts, and an inner solve is not
  // asked for more than kMixedInnerTol relative reduction, which FP32 blocks can deliver.
  *L = SolveLoop{};
  L->tol = tol;
  L->maxit = maxit;
  L->no_test = no_test;
  L->max_restarts = h->dm.mixed ? kMixedRestarts : 3;
  L->tol_rel = h->dm.mixed ? (tol > kMixedInnerTol ? tol : kMixedInnerTol) : tol;
  return MBPCG_OK;
}

// The parameters of the next inner solve (tolerance, iteration budget, restart count).
int enqueue_inner_params(mbpcg_ctx* h, const SolveLoop& L) {
  const int maxit_inner = L.no_test ? L.maxit : (L.maxit - L.total);
  k_params<<<1, 1, 0, h->stream>>>(h->st, L.tol_rel, maxit_inner, L.no_test, L.restarts, h->s,
                                   h->dm.mixed && !L.no_test ? 1 : 0);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

// One inner solve on the handle's own stream: its parameters, then the graph (or eager launches).
int launch_inner(mbpcg_ctx* h, const SolveLoop& L) {
  int rc = enqueue_inner_params(h, L);
  if (rc) return rc;
  if (h->launch_mode == MBPCG_LAUNCH_EAGER) return run_eager(h, L.no_test ? L.maxit : (L.maxit - L.total));
  CUDA_TRY(cudaGraphLaunch(h->exec, h->stream));
  return MBPCG_OK;
}

// Starts the copy of the solve state to the host after an inner solve.
int fetch_state(mbpcg_ctx* h) {
  CUDA_TRY(cudaMemcpyAsync(h->st_host, h->st, sizeof(SolveState), cudaMemcpyDeviceToHost, h->stream));
  return MBPCG_OK;
}

// Reads the state of the inner solve just finished and decides: *more = 1 when another inner solve
// (a restart, or a refinement step) is needed, with the loop's variables updated for it.
int after_inner(mbpcg_ctx* h, SolveLoop* L, int* more) {
  *more = 0;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  SolveState& s = L->s;
  std::memcpy(&s, h->st_host, sizeof(s));
  if (s.kerr) return set_err(MBPCG_ERR_TIMEOUT, "a bounded device-side wait timed out");
  L->total += s.it;
  if (L->no_test) {
    L->status = s.status;
    return MBPCG_OK;
  }
  const size_t nb = (size_t)h->dm.n * sizeof(double);
  const double relres = (s.b_norm > 0.0) ? s.true_res / s.b_norm : 0.0;
  if (h->dm.mixed) {
    // The refinement loop keeps its best iterate: a correction from an FP32 inner solve that
    // made the FP64 residual larger (possible when kappa(A) u_fp32 is not small) ends the loop
    // with the best x found.
    if (relres < L->best_relres) {
      L->best_relres = relres;
      CUDA_TRY(cudaMemcpyAsync(h->xbest, h->x, nb, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      CUDA_TRY(cudaMemcpyAsync(h->x, h->xbest, nb, cudaMemcpyDeviceToDevice, h->stream));
      s.true_res = L->best_relres * s.b_norm;
      L->status = L->best_relres <= L->tol ? MBPCG_OK : MBPCG_NOT_CONVERGED;
      return MBPCG_OK;
    }
  }
  if (relres <= L->tol) {
    L->status = MBPCG_OK;
    return MBPCG_OK;
  }
  if (L->restarts >= L->max_restarts || L->total >= L->maxit || s.status == MBPCG_NOT_CONVERGED) {
    L->status = (s.status == MBPCG_OK) ? MBPCG_NOT_CONVERGED : s.status;
    return MBPCG_OK;
  }
  ++L->restarts;
  L->tol_rel = 0.5 * L->tol * s.b_norm / s.true_res;
  if (h->dm.mixed && L->tol_rel < kMixedInnerTol) L->tol_rel = kMixedInnerTol;
  *more = 1;
  return MBPCG_OK;
}

// Copies x out (mem: 0 host, 1 device), waits for the handle's stream and fills info.
int solve_end(mbpcg_ctx* h, const SolveLoop& L, double* x_out, int mem, mbpcg_info* info) {
  const size_t nb = (size_t)h->dm.n * sizeof(double);
  if (x_out) CUDA_TRY(cudaMemcpyAsync(x_out, h->x, nb, mem ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                      h->stream));
  CUDA_TRY(cudaEventRecord(h->e1, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->e0, h->e1);
    const SolveState& s = L.s;
    const double bn = s.b_norm;
    info->iterations = L.total;
    info->restarts = L.restarts;
    info->status = L.status;
    info->best_col = s.best_col;
    info->ls_fallback = s.ls_fallback;
    info->reserved = 0;
    info->relres_recurrence = (bn > 0.0) ? s.nu_h / bn : 0.0;
    info->relres_ls = (bn > 0.0) ? s.ls_res / bn : 0.0;
    info->relres_true = (bn > 0.0) ? s.true_res / bn : 0.0;
    info->seconds = ms * 1e-3;
  }
  return MBPCG_OK;
}

// One solve: b and U in, the inner solves with their restarts, x out.
int solve_impl(mbpcg_ctx* h, const double* b, const double* U, double tol, int maxit, double* x_out,
               mbpcg_info* info, int mem, int no_test) {
  SolveLoop L;
  int rc = solve_begin(h, b, U, tol, maxit, x_out, mem, no_test, &L);
  for (int more = 1; !rc && more;) {
    rc = launch_inner(h, L);
    if (!rc) rc = fetch_state(h);
    if (!rc) rc = after_inner(h, &L, &more);
  }
  if (!rc) rc = solve_end(h, L, x_out, mem, info);
  if (rc) return rc;
  g_err.clear();
  return L.status;
}

}  // namespace

// ===================================================================================== C ABI

extern "C" {

size_t mbpcg_workspace_size_csr(int32_t n, int64_t nnz, int32_t s, int32_t algo, int32_t precision) {
  if (n < 1 || nnz < 0) return 0;
  Dims dm = make_dims(n, nnz, s, algo, 0, num_sms());
  if (precision == MBPCG_MIXED_FP32 && algo == MBPCG_ALGO_MBPCG) apply_mixed(dm);
  widen_for_handle(dm);
  return make_layout(dm).total;
}

size_t mbpcg_workspace_size_dense(int32_t n, int32_t s, int32_t algo, int32_t precision) {
  if (n < 1) return 0;
  Dims dm = make_dims(n, (long long)n * n, s, algo, 1, num_sms());
  dm.tc = (precision == MBPCG_FP64_TC && algo == MBPCG_ALGO_MBPCG) ? 1 : 0;
  if (precision == MBPCG_MIXED_FP32 && algo == MBPCG_ALGO_MBPCG) apply_mixed(dm);
  widen_for_handle(dm);
  return make_layout(dm).total;
}

int mbpcg_create_csr(mbpcg_handle* out, int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                     const double* vals, int32_t s, int32_t precond, int32_t algo, int32_t precision, uint64_t seed,
                     int32_t mem, void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return set_err(MBPCG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int rc = check_common(n, s, precond, algo, precision, mem);
  if (rc) return rc;
  if (nnz < 0 || nnz >= (1LL << 31)) return set_err(MBPCG_ERR_INVALID, "nnz must be in [0, 2^31)");
  if (!row_ptr || (nnz > 0 && (!col_idx || !vals))) return set_err(MBPCG_ERR_INVALID, "CSR arrays must not be NULL");
  if (precision == MBPCG_FP64_TC) return set_err(MBPCG_ERR_INVALID, "the tensor-core product is for dense A");
  const int sms = num_sms();
  if (sms <= 0) return set_err(MBPCG_ERR_CUDA, "no CUDA device available");
  mbpcg_ctx* h = nullptr;
  Dims dm = make_dims(n, nnz, s, algo, 0, sms);
  if (precision == MBPCG_MIXED_FP32) apply_mixed(dm);
  widen_for_handle(dm);
  rc = alloc_handle(&h, dm, s, precond, algo, precision, seed, workspace, workspace_bytes, stream);
  if (rc) {
    release(h);
    return rc;
  }
  const cudaMemcpyKind kind = mem ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(h->rp, row_ptr, (size_t)(n + 1) * sizeof(int), kind, h->stream);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(h->ci, col_idx, (size_t)nnz * sizeof(int), kind, h->stream);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(h->av, vals, (size_t)nnz * sizeof(double), kind, h->stream);
  if (e != cudaSuccess) {
    release(h);
    return set_err(MBPCG_ERR_CUDA, "copying A: %s", cudaGetErrorString(e));
  }
  k_validate_csr<<<(n + 255) / 256, 256, 0, h->stream>>>(n, nnz, h->rp, h->ci, h->flag);
  int flag = 0;
  rc = read_flag(h, &flag);
  if (!rc && (flag & 1)) rc = set_err(MBPCG_ERR_INVALID, "malformed CSR (row_ptr or col_idx out of range)");
  // the plan costs a sort of every tile's columns on the host: built at create only where the
  // autotuner may pick the tiled kernel (the FP32 product of a mixed handle); an FP64 handle builds
  // it when the tiled kernel is imposed (mbpcg_set_product_kernel)
  if (!rc && h->dm.mixed) rc = build_plan(h, row_ptr, col_idx, mem);
  if (!rc) rc = finish_create(h);
  if (rc) {
    release(h);
    return rc;
  }
  *out = h;
  return MBPCG_OK;
}

int mbpcg_create_dense(mbpcg_handle* out, int32_t n, const double* A_colmajor, int32_t s, int32_t precond,
                       int32_t algo, int32_t precision, uint64_t seed, int32_t mem, void* workspace,
                       size_t workspace_bytes, void* stream) {
  if (!out) return set_err(MBPCG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int rc = check_common(n, s, precond, algo, precision, mem);
  if (rc) return rc;
  if (!A_colmajor) return set_err(MBPCG_ERR_INVALID, "A must not be NULL");
  if ((long long)n * n >= (1LL << 40)) return set_err(MBPCG_ERR_INVALID, "n too large for a dense matrix");
  const int sms = num_sms();
  if (sms <= 0) return set_err(MBPCG_ERR_CUDA, "no CUDA device available");
  mbpcg_ctx* h = nullptr;
  Dims dm = make_dims(n, (long long)n * n, s, algo, 1, sms);
  dm.tc = (precision == MBPCG_FP64_TC && algo == MBPCG_ALGO_MBPCG) ? 1 : 0;
  if (precision == MBPCG_MIXED_FP32) apply_mixed(dm);
  widen_for_handle(dm);
  rc = alloc_handle(&h, dm, s, precond, algo, precision, seed, workspace, workspace_bytes, stream);
  if (rc) {
    release(h);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(h->A, A_colmajor, (size_t)n * n * sizeof(double),
                                  mem ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) {
    release(h);
    return set_err(MBPCG_ERR_CUDA, "copying A: %s", cudaGetErrorString(e));
  }
  rc = finish_create(h);
  if (rc) {
    release(h);
    return rc;
  }
  *out = h;
  return MBPCG_OK;
}

int mbpcg_solve(mbpcg_handle h, const double* b, const double* U, double tol, int32_t maxit, double* x_out,
                mbpcg_info* info) {
  return solve_impl(h, b, U, tol, maxit, x_out, info, 0, 0);
}

int mbpcg_solve_dev(mbpcg_handle h, const double* b, const double* U, double tol, int32_t maxit, double* x_out,
                    mbpcg_info* info) {
  return solve_impl(h, b, U, tol, maxit, x_out, info, 1, 0);
}

int mbpcg_run_iterations_dev(mbpcg_handle h, const double* b, const double* U, int32_t iters, double* X0,
                             double* Xt, double* R, double* W, double* P, double* Sigma) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (h->algo != MBPCG_ALGO_MBPCG) return set_err(MBPCG_ERR_INVALID, "diagnostic needs an MBPCG handle");
  if (h->dm.mixed) return set_err(MBPCG_ERR_INVALID, "diagnostic needs an FP64 handle");
  if (iters < 0) return set_err(MBPCG_ERR_INVALID, "iters must be >= 0");
  int rc = solve_impl(h, b, U, 1.0, iters, nullptr, nullptr, 1, 1);
  if (rc != MBPCG_OK && rc != MBPCG_BREAKDOWN) return rc;
  const RowOps* ops = row_ops(h->dm.kp);
  const int n = h->dm.n;
  double* src[5] = {h->X0, h->Xt, h->R, h->W, h->P};
  double* dst[5] = {X0, Xt, R, W, P};
  for (int q = 0; q < 5; ++q)
    if (dst[q]) ops->to_colmajor(h->stream, n, h->s, src[q], dst[q]);
  if (Sigma)
    CUDA_TRY(cudaMemcpy2DAsync(Sigma, h->s * sizeof(double), h->Sigma, h->dm.kp * sizeof(double),
                               h->s * sizeof(double), h->s, cudaMemcpyDeviceToDevice, h->stream));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return rc;
}

int mbpcg_set_launch_mode(mbpcg_handle h, int32_t mode) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (mode != MBPCG_LAUNCH_GRAPH && mode != MBPCG_LAUNCH_EAGER) return set_err(MBPCG_ERR_INVALID, "unknown mode");
  h->launch_mode = mode;
  return MBPCG_OK;
}

int mbpcg_get_spmm_tuning(mbpcg_handle h, int32_t* unroll, int32_t* ctas_per_sm, float* times_us) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (!h->dm.mixed || h->dm.dense)
    return set_err(MBPCG_ERR_INVALID, "the FP32 sparse product is tuned for MBPCG_MIXED_FP32 CSR handles");
  if (unroll) *unroll = h->spmm_unroll;
  if (ctas_per_sm) *ctas_per_sm = h->spmm_ctas_per_sm;
  if (times_us)
    for (int v = 0; v < kTuneVariants; ++v) times_us[v] = h->spmm_us[v];
  return MBPCG_OK;
}

int mbpcg_apply_dev(mbpcg_handle h, int32_t fp32, const void* X, void* Y) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (!X || !Y) return set_err(MBPCG_ERR_INVALID, "null block");
  if (fp32 && !h->dm.mixed) return set_err(MBPCG_ERR_INVALID, "the FP32 product belongs to MBPCG_MIXED_FP32 handles");
  if (fp32) {
    enqueue_product_f(h, row_ops_f(h->dm.kp), static_cast<const float*>(X), static_cast<float*>(Y), nullptr);
  } else {
    const Dims& dm = h->dm;
    if (dm.dense && !dm.tc) row_ops(dm.kp)->dense(h->stream, dm.nb_dense, dm.n, h->A, static_cast<const double*>(X),
                                                  static_cast<double*>(Y), nullptr, nullptr);
    else enqueue_product(h, row_ops(dm.kp), static_cast<const double*>(X), static_cast<double*>(Y), 0, nullptr);
  }
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_get_product_kernel(mbpcg_handle h, int32_t fp32, int32_t* kernel, float* times_us) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (fp32 && !h->dm.mixed) return set_err(MBPCG_ERR_INVALID, "the FP32 product belongs to MBPCG_MIXED_FP32 handles");
  int k;
  if (h->dm.dense) k = fp32 ? MBPCG_PRODUCT_DENSE_FP32 : (h->dm.tc ? MBPCG_PRODUCT_DENSE_TC : MBPCG_PRODUCT_DENSE);
  else if (fp32) k = h->spmm_unroll == 0 ? MBPCG_PRODUCT_CSR_TILED
                   : (h->spmm_unroll <= 2 ? MBPCG_PRODUCT_CSR_WIDE : MBPCG_PRODUCT_CSR_GATHER);
  else k = h->prod64;
  if (kernel) *kernel = k;
  if (times_us)
    for (int v = 0; v < 2; ++v) times_us[v] = h->spmm64_us[v];
  return MBPCG_OK;
}

int mbpcg_set_product_rounding(mbpcg_handle h, int32_t mode) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (!h->dm.tc) return set_err(MBPCG_ERR_INVALID, "the rounding mode belongs to MBPCG_FP64_TC handles");
  if (mode != MBPCG_ROUND_FP32_TAIL && mode != MBPCG_ROUND_ONCE)
    return set_err(MBPCG_ERR_INVALID, "mode must be MBPCG_ROUND_FP32_TAIL or MBPCG_ROUND_ONCE");
  const int once = mode == MBPCG_ROUND_ONCE ? 1 : 0;
  if (h->graph_ready && once != h->round_once) {  // the captured launches change
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    cudaGraphExecDestroy(h->exec);
    h->graph_ready = 0;
  }
  h->round_once = once;
  return MBPCG_OK;
}

int mbpcg_set_product_kernel(mbpcg_handle h, int32_t kernel) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (h->dm.dense) return set_err(MBPCG_ERR_INVALID, "a dense handle has one FP64 product");
  if (kernel != MBPCG_PRODUCT_CSR_GATHER && kernel != MBPCG_PRODUCT_CSR_TILED)
    return set_err(MBPCG_ERR_INVALID, "kernel must be MBPCG_PRODUCT_CSR_GATHER or MBPCG_PRODUCT_CSR_TILED");
  if (kernel == MBPCG_PRODUCT_CSR_TILED && !h->dm.mixed && !h->plan_tried) {
    int rc = build_plan(h, nullptr, nullptr, 1);
    if (!rc && h->use_tiled) rc = time_spmm64(h, MBPCG_PRODUCT_CSR_TILED);
    if (rc) return rc;
  }
  if (kernel == MBPCG_PRODUCT_CSR_TILED && (!h->use_tiled || h->dm.mixed))
    return set_err(MBPCG_ERR_INVALID, "this handle's FP64 product has no tiling plan");
  if (h->graph_ready && kernel != h->prod64) {  // the captured launches change
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    cudaGraphExecDestroy(h->exec);
    h->graph_ready = 0;
  }
  h->prod64 = kernel;
  return MBPCG_OK;
}

int mbpcg_set_spmm_shape(mbpcg_handle h, int32_t unroll, int32_t ctas_per_sm) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (!h->dm.mixed || h->dm.dense)
    return set_err(MBPCG_ERR_INVALID, "the FP32 sparse product is tuned for MBPCG_MIXED_FP32 CSR handles");
  bool known = false;
  for (int v = 0; v < kTuneVariants; ++v) known = known || (kShapeUnroll[v] == unroll && kShapeCtas[v] == ctas_per_sm);
  if (!known)
    return set_err(MBPCG_ERR_INVALID, "unroll 4, 8 (gather) or 1 (staged) with ctas_per_sm 4, 8 or 16; or 0 and 2 (tiled)");
  if (unroll == 0 && !h->use_tiled) return set_err(MBPCG_ERR_INVALID, "this matrix has no tiling plan");
  if (h->graph_ready) {  // the captured launches change
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    cudaGraphExecDestroy(h->exec);
    h->graph_ready = 0;
  }
  h->spmm_unroll = unroll;
  h->spmm_ctas_per_sm = ctas_per_sm;
  h->spmm_nb = shape_grid(h, unroll, ctas_per_sm);
  return MBPCG_OK;
}

int mbpcg_set_residual_mode(mbpcg_handle h, int32_t mode) {
  if (!h) return set_err(MBPCG_ERR_INVALID, "null handle");
  if (mode != MBPCG_RESIDUAL_EXPLICIT && mode != MBPCG_RESIDUAL_IMPLICIT)
    return set_err(MBPCG_ERR_INVALID, "unknown residual mode");
  if (mode == MBPCG_RESIDUAL_IMPLICIT && (h->algo != MBPCG_ALGO_MBPCG || h->dm.mixed))
    return set_err(MBPCG_ERR_INVALID, "the implicit-residual mode is for FP64 MBPCG handles");
  const int rf = (mode == MBPCG_RESIDUAL_IMPLICIT) ? 1 : 0;
  if (rf != h->rfree && h->graph_ready) {  // the captured loop body changes
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    cudaGraphExecDestroy(h->exec);
    h->graph_ready = 0;
  }
  h->rfree = rf;
  return MBPCG_OK;
}

void mbpcg_destroy(mbpcg_handle h) { release(h); }

void mbpcg_batch_destroy(mbpcg_batch b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaEvent_t e : b->ready)
    if (e) cudaEventDestroy(e);
  if (b->done) cudaEventDestroy(b->done);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int mbpcg_batch_create(mbpcg_batch* out, const mbpcg_handle* handles, int32_t count, void* stream) {
  if (!out) return set_err(MBPCG_ERR_INVALID, "null output pointer");
  *out = nullptr;
  if (!handles || count < 1) return set_err(MBPCG_ERR_INVALID, "a batch needs at least one handle");
  for (int i = 0; i < count; ++i) {
    if (!handles[i]) return set_err(MBPCG_ERR_INVALID, "handle %d is NULL", i);
    if (handles[i]->launch_mode != MBPCG_LAUNCH_GRAPH)
      return set_err(MBPCG_ERR_INVALID, "handle %d is in eager launch mode (a batch is one graph)", i);
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return set_err(MBPCG_ERR_INVALID, "handle %d appears twice", i);
  }
  mbpcg_batch_ctx* b = new (std::nothrow) mbpcg_batch_ctx;
  if (!b) return set_err(MBPCG_ERR_OOM, "host allocation failed");
  b->h.assign(handles, handles + count);
  b->ready.assign(count, nullptr);
  int rc = MBPCG_OK;
  cudaError_t e = cudaSuccess;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = e == cudaSuccess ? 1 : 0;
  }
  for (int i = 0; e == cudaSuccess && i < count; ++i) e = cudaEventCreateWithFlags(&b->ready[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) e = cudaGraphCreate(&g, 0);
  for (int i = 0; e == cudaSuccess && i < count; ++i) {
    cudaGraphConditionalHandle cond{};
    e = capture_solve(handles[i], g, &cond);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = set_err(MBPCG_ERR_CUDA, "building the batch graph failed: %s", cudaGetErrorString(e));
    mbpcg_batch_destroy(b);
    return rc;
  }
  *out = b;
  return MBPCG_OK;
}

int mbpcg_batch_solve_dev(mbpcg_batch bt, const double* const* b, const double* const* U, double tol, int32_t maxit,
                          double* const* x_out, mbpcg_info* info) {
  if (!bt) return set_err(MBPCG_ERR_INVALID, "null batch");
  if (!b || !x_out) return set_err(MBPCG_ERR_INVALID, "b and x_out must not be NULL");
  const int K = (int)bt->h.size();
  std::vector<SolveLoop> L(K);
  // every member: inputs in, parameters of its first inner solve, then the one batch launch
  for (int i = 0; i < K; ++i) {
    mbpcg_ctx* h = bt->h[i];
    int rc = solve_begin(h, b[i], U ? U[i] : nullptr, tol, maxit, x_out[i], 1, 0, &L[i]);
    if (!rc) rc = enqueue_inner_params(h, L[i]);
    if (rc) return rc;
    CUDA_TRY(cudaEventRecord(bt->ready[i], h->stream));
    CUDA_TRY(cudaStreamWaitEvent(bt->stream, bt->ready[i], 0));
  }
  CUDA_TRY(cudaGraphLaunch(bt->exec, bt->stream));
  CUDA_TRY(cudaEventRecord(bt->done, bt->stream));
  for (int i = 0; i < K; ++i) {
    CUDA_TRY(cudaStreamWaitEvent(bt->h[i]->stream, bt->done, 0));
    int rc = fetch_state(bt->h[i]);
    if (rc) return rc;
  }
  // restarts (or refinement steps) run on each member's own graph, concurrently on their streams
  std::vector<int> active(K, 1);
  for (bool any = true; any;) {
    any = false;
    for (int i = 0; i < K; ++i) {
      if (!active[i]) continue;
      int more = 0;
      int rc = after_inner(bt->h[i], &L[i], &more);
      if (!rc && more) rc = launch_inner(bt->h[i], L[i]);
      if (!rc && more) rc = fetch_state(bt->h[i]);
      if (rc) return rc;
      active[i] = more;
      any = any || more;
    }
  }
  int status = MBPCG_OK;
  for (int i = 0; i < K; ++i) {
    int rc = solve_end(bt->h[i], L[i], x_out[i], 1, info ? &info[i] : nullptr);
    if (rc) return rc;
    if (status == MBPCG_OK && L[i].status != MBPCG_OK) status = L[i].status;
  }
  g_err.clear();
  return status;
}

const char* mbpcg_status_string(int status) {
  switch (status) {
    case MBPCG_OK: return "ok";
    case MBPCG_ERR_INVALID: return "invalid argument";
    case MBPCG_ERR_OOM: return "out of memory";
    case MBPCG_ERR_CUDA: return "CUDA error";
    case MBPCG_ERR_NOT_SPD: return "matrix is not SPD (diagonal)";
    case MBPCG_NOT_CONVERGED: return "not converged";
    case MBPCG_BREAKDOWN: return "breakdown";
    case MBPCG_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* mbpcg_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ component entry points

int32_t mbpcg_k_padded_width(int32_t s) { return (s >= 1 && s <= 32) ? padded_width(s) : 0; }

size_t mbpcg_k_scratch_bytes(int32_t n, int32_t s) {
  if (n < 1 || s < 1 || s > 32) return 0;
  Dims dm = make_dims(n, 0, s, MBPCG_ALGO_MBPCG, 0, num_sms());
  apply_mixed(dm);  // enough partial slots for the FP64 and the FP32 launch configurations
  return (size_t)(dm.nbmax + 1) * dm.pstride * sizeof(double);
}

static int k_product_gram(int dense, int32_t n, const int32_t* rp, const int32_t* ci, const double* av,
                          const double* A, int32_t s, const double* P, double* AP, double* G, void* scratch,
                          size_t scratch_bytes, void* stream) {
  if (n < 1 || s < 1 || s > 32 || !P || !AP || !G) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  if (scratch_bytes < mbpcg_k_scratch_bytes(n, s) || !scratch) return set_err(MBPCG_ERR_INVALID, "scratch too small");
  const Dims dm = make_dims(n, 0, s, MBPCG_ALGO_MBPCG, dense, num_sms());
  const RowOps* ops = row_ops(dm.kp);
  cudaStream_t st = (cudaStream_t)stream;
  double* part = static_cast<double*>(scratch);
  double* red = part + (size_t)dm.nbmax * dm.pstride;
  if (dense) {
    ops->dense(st, dm.nb_dense, n, A, P, AP, nullptr, nullptr);
    ops->gram(st, dm.nb, n, P, AP, part, dm.pstride, nullptr);
  } else {
    ops->spmm(st, dm.nb, n, rp, ci, av, P, AP, part, dm.pstride, nullptr, 1);
  }
  launch_reduce(st, part, dm.nb, dm.pstride, red, npack(dm.kp), nullptr);
  k_unpack_full<<<1, 256, 0, st>>>(red, dm.kp, s, G);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_spmm_gram(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* vals, int32_t s,
                      const double* P, double* AP, double* G, void* scratch, size_t scratch_bytes, void* stream) {
  if (!row_ptr) return set_err(MBPCG_ERR_INVALID, "row_ptr is NULL");
  return k_product_gram(0, n, row_ptr, col_idx, vals, nullptr, s, P, AP, G, scratch, scratch_bytes, stream);
}

int mbpcg_k_spmm_gram_f32(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const float* vals, int32_t s,
                          const float* P, float* AP, double* G, void* scratch, size_t scratch_bytes, void* stream) {
  if (n < 1 || s < 1 || s > 32 || !row_ptr || !P || !AP || !G) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  if (scratch_bytes < mbpcg_k_scratch_bytes(n, s) || !scratch) return set_err(MBPCG_ERR_INVALID, "scratch too small");
  Dims dm = make_dims(n, 0, s, MBPCG_ALGO_MBPCG, 0, num_sms());
  apply_mixed(dm);
  cudaStream_t st = (cudaStream_t)stream;
  double* part = static_cast<double*>(scratch);
  double* red = part + (size_t)dm.nbmax * dm.pstride;
  row_ops_f(dm.kp)->spmm(st, dm.nb, n, row_ptr, col_idx, vals, P, AP, nullptr, 0, nullptr, 0, 8);
  row_ops_f(dm.kp)->gram(st, dm.nb, n, P, AP, part, dm.pstride, nullptr);
  launch_reduce(st, part, dm.nb, dm.pstride, red, npack(dm.kp), nullptr);
  k_unpack_full<<<1, 256, 0, st>>>(red, dm.kp, s, G);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_spmm_f32(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const float* vals, int32_t s,
                     const float* P, float* AP, void* stream) {
  if (n < 1 || s < 1 || s > 32 || !row_ptr || !P || !AP) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  Dims dm = make_dims(n, 0, s, MBPCG_ALGO_MBPCG, 0, num_sms());
  apply_mixed(dm);
  row_ops_f(dm.kp)->spmm((cudaStream_t)stream, dm.nb, n, row_ptr, col_idx, vals, P, AP, nullptr, 0, nullptr, 0, 8);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

size_t mbpcg_k_dense_f32_bytes(int32_t n) { return n < 1 ? 0 : dense_f32_tiles_bytes(n); }

int mbpcg_k_dense_f32_prepare(int32_t n, const double* A, void* tiles, size_t tiles_bytes, void* stream) {
  if (n < 1 || !A || !tiles) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  if (tiles_bytes < dense_f32_tiles_bytes(n)) return set_err(MBPCG_ERR_INVALID, "tiles buffer too small");
  if (reinterpret_cast<uintptr_t>(tiles) % 16 != 0) return set_err(MBPCG_ERR_INVALID, "tiles must be 16-byte aligned");
  const int sms = num_sms();
  if (sms <= 0) return set_err(MBPCG_ERR_CUDA, "no CUDA device available");
  k_dense_to_f32_tiles<<<4 * sms, 256, 0, (cudaStream_t)stream>>>(n, A, static_cast<float*>(tiles));
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_dense_f32(int32_t n, const void* tiles, int32_t s, const float* P, float* AP, void* stream) {
  if (n < 1 || s < 1 || s > 32 || !tiles || !P || !AP) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  if ((reinterpret_cast<uintptr_t>(tiles) | reinterpret_cast<uintptr_t>(P)) % 16 != 0)
    return set_err(MBPCG_ERR_INVALID, "tiles and P must be 16-byte aligned");
  const int sms = num_sms();
  if (sms <= 0) return set_err(MBPCG_ERR_CUDA, "no CUDA device available");
  dense_f32_product((cudaStream_t)stream, padded_width(s), n, sms, static_cast<const float*>(tiles), P, AP, nullptr);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_dense_gram(int32_t n, const double* A, int32_t s, const double* P, double* AP, double* G, void* scratch,
                       size_t scratch_bytes, void* stream) {
  if (!A) return set_err(MBPCG_ERR_INVALID, "A is NULL");
  return k_product_gram(1, n, nullptr, nullptr, nullptr, A, s, P, AP, G, scratch, scratch_bytes, stream);
}

int mbpcg_k_spmm(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* vals, int32_t s,
                 const double* P, double* AP, void* stream) {
  if (n < 1 || s < 1 || s > 32 || !row_ptr || !P || !AP) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  const Dims dm = make_dims(n, 0, s, MBPCG_ALGO_MBPCG, 0, num_sms());
  row_ops(dm.kp)->spmm((cudaStream_t)stream, dm.nb, n, row_ptr, col_idx, vals, P, AP, nullptr, 0, nullptr, 0);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_dense_product(int32_t n, const double* A, int32_t s, const double* P, double* AP, void* stream) {
  if (n < 1 || s < 1 || s > 32 || !A || !P || !AP) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  const Dims dm = make_dims(n, (long long)n * n, s, MBPCG_ALGO_MBPCG, 1, num_sms());
  row_ops(dm.kp)->dense((cudaStream_t)stream, dm.nb_dense, n, A, P, AP, nullptr, nullptr);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

size_t mbpcg_k_dense_tc_scratch_bytes(int32_t n, int32_t s) {
  if (n < 1 || s < 1 || s > 32) return 0;
  const int kp = padded_width(s), sms = num_sms() > 0 ? num_sms() : 1;
  return align_up(oz_a_tiles_bytes(n)) + align_up((size_t)n * sizeof(int)) + align_up(oz_p_chunks_bytes(n, kp)) +
         align_up(2 * kMaxKP * sizeof(int)) +
         align_up((size_t)oz_ksplit(n, sms) * n * kp * 2 * sizeof(long long));
}

namespace {
struct TcScratch {
  uint8_t* at;
  int* ea;
  uint8_t* pc;
  int* ep;
  double* qp;
};
TcScratch tc_scratch(void* scratch, int n, int kp) {
  TcScratch t;
  uint8_t* p = static_cast<uint8_t*>(scratch);
  t.at = p;
  p += align_up(oz_a_tiles_bytes(n));
  t.ea = reinterpret_cast<int*>(p);
  p += align_up((size_t)n * sizeof(int));
  t.pc = p;
  p += align_up(oz_p_chunks_bytes(n, kp));
  t.ep = reinterpret_cast<int*>(p);
  p += align_up(2 * kMaxKP * sizeof(int));
  t.qp = reinterpret_cast<double*>(p);
  return t;
}
}  // namespace

int mbpcg_k_dense_tc_prepare(int32_t n, const double* A, int32_t s, void* scratch, size_t scratch_bytes,
                             void* stream) {
  if (n < 1 || s < 1 || s > 32 || !A || !scratch) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  if (scratch_bytes < mbpcg_k_dense_tc_scratch_bytes(n, s)) return set_err(MBPCG_ERR_INVALID, "scratch too small");
  const int kp = padded_width(s);
  cudaStream_t st = (cudaStream_t)stream;
  const TcScratch t = tc_scratch(scratch, n, kp);
  oz_prepare_a(st, n, A, t.ea, t.at);
  CUDA_TRY(cudaMemsetAsync(t.pc, 0, oz_p_chunks_bytes(n, kp), st));
  // the split sum reads every slice of the partials buffer (those past a tile's count unused)
  CUDA_TRY(cudaMemsetAsync(t.qp, 0, (size_t)oz_ksplit(n, num_sms() > 0 ? num_sms() : 1) * n * kp * 2 * sizeof(long long),
                           st));
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_rowprod_tc(int32_t n, int32_t width, const double* X, const double* M, int32_t transM, double* Y,
                       void* stream) {
  if (n < 1 || !X || !M || !Y || (transM != 0 && transM != 1)) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  if (width != 16 && width != 32) return set_err(MBPCG_ERR_INVALID, "width must be 16 or 32");
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) % 16 != 0)
    return set_err(MBPCG_ERR_INVALID, "X and Y must be 16-byte aligned");
  const RowProdJobs jb = {{{X, M, transM, Y}, {nullptr, nullptr, 0, nullptr}, {nullptr, nullptr, 0, nullptr}}};
  rowprod_tc((cudaStream_t)stream, n, width, jb, 1, nullptr, 0, nullptr);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_dense_tc_mma(int32_t n, int32_t s, void* scratch, size_t scratch_bytes, void* stream) {
  if (n < 1 || s < 1 || s > 32 || !scratch) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  if (scratch_bytes < mbpcg_k_dense_tc_scratch_bytes(n, s)) return set_err(MBPCG_ERR_INVALID, "scratch too small");
  const int kp = padded_width(s);
  const TcScratch t = tc_scratch(scratch, n, kp);
  oz_mma((cudaStream_t)stream, n, kp, num_sms(), t.at, t.ea, t.pc, t.ep, t.qp);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_dense_tc_product(int32_t n, int32_t s, const double* P, double* AP, void* scratch, size_t scratch_bytes,
                             void* stream) {
  if (n < 1 || s < 1 || s > 32 || !P || !AP || !scratch) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  if (scratch_bytes < mbpcg_k_dense_tc_scratch_bytes(n, s)) return set_err(MBPCG_ERR_INVALID, "scratch too small");
  const int kp = padded_width(s);
  const TcScratch t = tc_scratch(scratch, n, kp);
  oz_product((cudaStream_t)stream, n, kp, num_sms(), t.at, t.ea, P, t.pc, t.ep, t.qp, AP, nullptr, nullptr, nullptr, 0,
             0, 0, 0);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_cholesky(int32_t s, const double* G, double* Z, int32_t* status_dev, void* stream) {
  if (s < 1 || s > 32 || !G || !Z || !status_dev) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  k_chol_only<<<1, kSmallThreads, 0, (cudaStream_t)stream>>>(G, s, Z, status_dev);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

int mbpcg_k_pivot_reciprocals(int32_t n, const double* d, double* inv, double* rsq, void* stream) {
  if (n < 1 || !d || !inv || !rsq) return set_err(MBPCG_ERR_INVALID, "bad arguments");
  launch_pivot_recips((cudaStream_t)stream, n, d, inv, rsq);
  CUDA_TRY(cudaGetLastError());
  return MBPCG_OK;
}

}  // extern "C"

namespace mbpcg {

// Launch shape of the CSR product + Gram entry points (padded width, CTA count, slot stride).
void product_gram_shape(int n, int s, int* kp, int* nb, int* pstride) {
  const Dims dm = make_dims(n, 0, s, MBPCG_ALGO_MBPCG, 0, num_sms());
  *kp = dm.kp;
  *nb = dm.nb;
  *pstride = dm.pstride;
}

int set_last_error(int code, const char* msg) { return set_err(code, "%s", msg); }

// G (s x s column-major, ld s) = the full symmetric matrix of a packed upper triangle.
__global__ void k_unpack_full(const double* __restrict__ packed, int kp, int s, double* __restrict__ G) {
  for (int q = threadIdx.x; q < s * s; q += blockDim.x) {
    const int l = q % s, m = q / s;
    G[q] = (l <= m) ? packed[pidx(l, m)] : packed[pidx(m, l)];
  }
}

// Z = upper Cholesky factor of G (s x s, ld s); *status = 0 or 6 (breakdown).
__global__ void k_chol_only(const double* __restrict__ G, int s, double* __restrict__ Z, int* __restrict__ status) {
  __shared__ double A[kMaxKP * kMaxKP];
  __shared__ int flag;
  for (int q = threadIdx.x; q < kMaxKP * kMaxKP; q += blockDim.x) {
    const int l = q % kMaxKP, m = q / kMaxKP;
    A[q] = (l < s && m < s) ? G[l + m * s] : 0.0;
  }
  __syncthreads();
  const int fail = cta_cholesky(s, kMaxKP, A, &flag);
  for (int q = threadIdx.x; q < s * s; q += blockDim.x) {
    const int l = q % s, m = q / s;
    Z[q] = fail ? 0.0 : A[l + m * kMaxKP];
  }
  if (threadIdx.x == 0) *status = fail ? 6 : 0;
}

}  // namespace mbpcg
