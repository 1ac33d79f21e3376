// Internal interface between the host runtime (api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "mbpcg_device.cuh"

namespace mbpcg {

// Opt-in dynamic shared memory of a kernel: set when the kernel's attribute on the current device is
// below `bytes`. Checked on every launch -- the attribute belongs to the device's context, which
// another device, another thread's first launch or a device reset does not share with a flag.
template <typename K>
inline cudaError_t ensure_dynamic_smem(K* func, size_t bytes) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, (const void*)func);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute((const void*)func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}


// Host launchers of the row kernels for one padded width KP (defined in inst_kp*.cu).
struct RowOps {
  int kp;
  void (*spmm)(cudaStream_t, int nb, int n, const int* rp, const int* ci, const double* av, const double* P,
               double* Q, double* part, int pstride, const SolveState* st, int gram);
  void (*dense)(cudaStream_t, int nb, int n, const double* A, const double* P, double* Q, const SolveState* st,
                int* err);
  void (*gram)(cudaStream_t, int nb, int n, const double* X, const double* Y, double* part, int pstride,
               const SolveState* st);
  void (*axpy)(cudaStream_t, int nb, int n, const double* P, const double* Q, const double* W, double* R,
               double* Xt, double* V, const double* T, const double* Xi, const double* wdiag, double* part,
               int pstride, const SolveState* st, int rfree);
  void (*rsig)(cudaStream_t, int nb, int n, const double* V, const double* W, const double* Sigma, double* R,
               const SolveState* st);
  void (*pw)(cudaStream_t, int nb, int n, const double* V, double* W, double* P, const double* Zinv,
             const double* Z, const SolveState* st, int setp, int* emax);
  void (*setup_norms)(cudaStream_t, int nb, int n, const double* rhs, const double* d, double* bs,
                      const double* AU, double* part, int pstride);
  void (*init)(cudaStream_t, int nb, int n, int s, const double* U, const double* AU, const double* bs, double* X0,
               double* Xt, double* R, double* part, int pstride, const SolveState* st);
  void (*ls_gram)(cudaStream_t, int nb, int n, const double* R, const double* rhs, const double* sqd, double* part,
                  int pstride);
  void (*combine)(cudaStream_t, int nb, int n, int s, const double* Xt, const double* X0, const double* c,
                  const double* d, double* x);
  void (*gen_u)(cudaStream_t, int n, int s, unsigned long long seed, double* U);
  void (*from_colmajor)(cudaStream_t, int n, int s, const double* src, double* dst);
  void (*to_colmajor)(cudaStream_t, int n, int s, const double* src, double* dst);
  // the block update and the W/P update with their k x k-row products given (from rowprod_tc):
  // PT = P T, QT = (AP) T, QXi = (AP) Xi; VZi = V zeta^{-1}, PZt = P zeta^T
  void (*axpy_pre)(cudaStream_t, int nb, int n, const double* PT, const double* QT, const double* QXi,
                   const double* W, double* R, double* Xt, double* V, const double* wdiag, double* part, int pstride,
                   const SolveState* st);
  void (*pw_pre)(cudaStream_t, int n, const double* VZi, const double* PZt, double* W, double* P, const SolveState* st,
                 int* emax);
};

const RowOps* row_ops_kp1();
const RowOps* row_ops_kp2();
const RowOps* row_ops_kp4();
const RowOps* row_ops_kp8();
const RowOps* row_ops_kp16();
const RowOps* row_ops_kp32();

inline int padded_width(int s) {
  int kp = 1;
  while (kp < s) kp <<= 1;
  return kp;
}
inline const RowOps* row_ops(int kp) {
  switch (kp) {
    case 1: return row_ops_kp1();
    case 2: return row_ops_kp2();
    case 4: return row_ops_kp4();
    case 8: return row_ops_kp8();
    case 16: return row_ops_kp16();
    case 32: return row_ops_kp32();
    default: return nullptr;
  }
}

// Host launchers of the FP32 row kernels of the mixed-precision inner solve (inst_f32_kp*.cu).
struct RowOpsF {
  int kp;
  void (*spmm)(cudaStream_t, int nb, int n, const int* rp, const int* ci, const float* av, const float* P, float* Q,
               double* part, int pstride, const SolveState* st, int gram, int unroll);  // unroll 4 or 8 (no gram)
  void (*gram)(cudaStream_t, int nb, int n, const float* X, const float* Y, double* part, int pstride,
               const SolveState* st);
  void (*axpy)(cudaStream_t, int nb, int n, const float* P, const float* Q, const float* W, float* R, float* Xt,
               float* V, const double* T, const double* Xi, const float* wdiag, double* part, int pstride,
               const SolveState* st);
  void (*pw)(cudaStream_t, int nb, int n, const float* V, float* W, float* P, const double* Zinv, const double* Z,
             const SolveState* st, int setp);
  void (*setup_norms)(cudaStream_t, int nb, int n, const double* rhs, const double* d, double* bs, const float* AU,
                      double* part, int pstride);
  void (*init)(cudaStream_t, int nb, int n, int s, const float* U, const float* AU, const double* bs, float* X0,
               float* Xt, float* R, double* part, int pstride, const SolveState* st);
  void (*ls_gram)(cudaStream_t, int nb, int n, const float* R, const double* rhs, const double* sqd, double* part,
                  int pstride);
  void (*combine)(cudaStream_t, int nb, int n, int s, const float* Xt, const float* X0, const double* c,
                  const double* d, double* x);
  void (*gen_u)(cudaStream_t, int n, int s, unsigned long long seed, float* U);
  void (*from_colmajor)(cudaStream_t, int n, int s, const double* src, float* dst);
};

const RowOpsF* row_ops_f_kp1();
const RowOpsF* row_ops_f_kp2();
const RowOpsF* row_ops_f_kp4();
const RowOpsF* row_ops_f_kp8();
const RowOpsF* row_ops_f_kp16();
const RowOpsF* row_ops_f_kp32();

// rows of one CTA tile in the FP32 kernels (four threads per row above KP = 4)
inline int rows_per_tile_f(int kp) { return kp <= 4 ? 256 : 256 / (kp / 4); }

inline const RowOpsF* row_ops_f(int kp) {
  switch (kp) {
    case 1: return row_ops_f_kp1();
    case 2: return row_ops_f_kp2();
    case 4: return row_ops_f_kp4();
    case 8: return row_ops_f_kp8();
    case 16: return row_ops_f_kp16();
    case 32: return row_ops_f_kp32();
    default: return nullptr;
  }
}

// single-CTA and vector kernels (small_kernels.cu)
__global__ void k_to_f32(long long n, const double* __restrict__ src, float* __restrict__ dst);
__global__ void k_small_nu(SolveState* st, double* __restrict__ red, const double* __restrict__ Sigma, int kp,
                           int goff);
// out[e] = sum over p < nparts of part[p * pstride + e] for e < nent (fixed order; st may be NULL).
void launch_reduce(cudaStream_t s, const double* part, int nparts, int pstride, double* out, int nent,
                   const SolveState* st);
__global__ void k_params(SolveState* st, double tol_rel, int maxit, int no_test, int restart, int s, int stag);
__global__ void k_small_setup(SolveState* st, const double* red);
__global__ void k_small_ls(SolveState* st, const double* Mg, int kp, double* c_out);
__global__ void k_small_true(SolveState* st, const double* rr);
__global__ void k_small_cg_setup(SolveState* st, const double* red);
__global__ void k_small_cg(SolveState* st, const double* red, cudaGraphConditionalHandle cond, int use_cond);
__global__ void k_validate_csr(int n, long long nnz, const int* rp, const int* ci, int* flag);
__global__ void k_diag_csr(int n, const int* rp, const int* ci, const double* av, double* diag, int* flag);
__global__ void k_diag_dense(int n, const double* A, double* diag, int* flag);
__global__ void k_check_finite(long long count, const double* v, int* flag);
__global__ void k_make_scaling(int n, const double* diag, double* d, double* sqd);
__global__ void k_scale_csr(int n, const int* rp, const int* ci, double* av, const double* d);
__global__ void k_scale_dense(int n, double* A, const double* d);
__global__ void k_resid_csr(int n, const int* rp, const int* ci, const double* av, const double* sqd,
                            const double* b, const double* x, double* r, double* part, int pstride);
__global__ void k_resid_dense(int n, const double* A, const double* sqd, const double* b, const double* x,
                              double* r, double* part, int pstride);
__global__ void k_cg_init(int n, const double* rhs, const double* d, double* r, double* x, double* p, double* sv,
                          double* part, int pstride);
__global__ void k_cg_dots(int n, const double* r, const double* w, const double* wdiag, double* part, int pstride,
                          const SolveState* st);
__global__ void k_cg_update(int n, double* r, const double* w, double* x, double* p, double* sv,
                            const SolveState* st);
__global__ void k_cg_finish(int n, const double* xbar, const double* d, double* x);

// CSR product with the rows of P each tile needs staged in shared memory (spmm_tiled.cu). A plan
// cuts the rows into tiles of R rows; run q of tile t is rows [run_start[q], +run_len[q]) of P,
// runs run_ptr[t] .. run_ptr[t+1]-1; cl[p] is the position of nonzero p's column in its tile's
// window (wmax: the largest window, in rows).
struct SpmmPlan {
  int R, ntiles, wmax;
  const int* run_ptr;
  const int* run_start;
  const int* run_len;
  const uint16_t* cl;
};
struct SpmmPlanHost {
  int R = 0, ntiles = 0, wmax = 0;
  std::vector<int> run_ptr, run_start, run_len;
  std::vector<uint16_t> cl;
};
size_t spmm_plan_window_rows(int kp, size_t elem);
// Builds the plan from host CSR arrays (validated); 0 when no tile size lets every window fit.
int spmm_plan_build(int n, const int* rp, const int* ci, int kp, size_t elem, SpmmPlanHost* out);
size_t spmm_plan_smem(int kp, size_t elem, int wmax);
// The FP32 product with CTAs of `threads` (512 or 1024) threads (spmm_wide.cu): the same bits as
// the gather kernel.
void spmm_wide_f(cudaStream_t s, int kp, int threads, int nb, int n, const int* rp, const int* ci, const float* av,
                 const float* P, float* Q, const SolveState* st);
void spmm_tiled(cudaStream_t s, int kp, int nb, int n, const int* rp, const double* av, const SpmmPlan& pl,
                const double* P, double* Q, double* part, int pstride, const SolveState* st, int gram);
void spmm_tiled_f(cudaStream_t s, int kp, int nb, int n, const int* rp, const float* av, const SpmmPlan& pl,
                  const float* P, float* Q, const SolveState* st);

// Chronopoulos-Gear CG on a dense A, one launch per iteration (cg_dense.cu). r, w and s in two
// copies (by the parity of the iteration), p and x in one; counter: one zeroed unsigned int.
constexpr int kCgDenseMaxN = 16384;  // the whole vector r_j lives in each CTA's shared memory
struct CgVectors {
  double* r[2];
  double* w[2];
  double* s[2];
  double* p;
  double* x;
};
bool cg_dense_fused_ok(int n);  // n even and at most kCgDenseMaxN
int cg_dense_grid(int n, int sms);  // CTAs of the fused launch (one per SM)
__host__ __device__ int cg_dense_fragments(int n, int nb);
size_t cg_dense_smem_bytes(int n, int nb);
cudaError_t cg_dense_configure(int n, int nb);
void launch_cg_dense_iter(cudaStream_t s, int nb, int n, const double* A, const CgVectors& v, const double* wdiag,
                          double* part, int pstride, unsigned int* counter, SolveState* st,
                          cudaGraphConditionalHandle cond, int use_cond);

// FP32 dense product of the mixed-precision inner solve (dense_f32.cu): Q = A P with A in the FP32
// tiles k_dense_to_f32_tiles writes (dense_f32_tiles_bytes(n) bytes), P and Q row-major n x kp;
// st may be NULL.
size_t dense_f32_tiles_bytes(int n);
__global__ void k_dense_to_f32_tiles(int n, const double* A, float* At);
void dense_f32_product(cudaStream_t s, int kp, int n, int sms, const float* At, const float* P, float* Q,
                       const SolveState* st);

// FP64-accurate dense product on the BF16 tensor cores (ozaki_tc.cu)
size_t oz_a_tiles_bytes(int n);
size_t oz_p_chunks_bytes(int n, int kp);
int oz_ksplit(int n, int sms);  // partial slices of Q the product needs (Qpart holds this many n x kp blocks)
void oz_prepare_a(cudaStream_t s, int n, const double* A, int* emaxA, uint8_t* Atiles);
// part != NULL: also the CTA partials of P^T (A P) over nb balanced row ranges (stride pstride).
// exp_ready: the column exponents of P are already in emaxP (written by the W/P update).
// k x k-row products on the tensor cores (rowprod_tc.cu): Y = X M for up to three (X, M) pairs, one
// launch; X and Y row-major n x kp FP64, M column-major kp x kp (M^T with transM), kp = 16 or 32.
// Skipped when the solve is done (or, with skip_on_pw, when the W/P update is skipped).
struct RowProdJob {
  const double* X;
  const double* M;
  int transM;
  double* Y;
};
struct RowProdJobs {
  RowProdJob j[3];
};
void rowprod_tc(cudaStream_t s, int n, int kp, const RowProdJobs& jobs, int njobs, const SolveState* st,
                int skip_on_pw, int* err);

// The MMA kernel alone (k_dense_tc) on P digits already in Pchunks: partial slices into Qpart.
void oz_mma(cudaStream_t s, int n, int kp, int sms, const uint8_t* Atiles, const int* emaxA, const uint8_t* Pchunks,
            const int* emaxP, double* Qpart);
// The whole product: column exponents and digits of P (unless exp_ready), the MMA kernel, the split
// sum (with the Gram partials when part != NULL). once = 1: levels 5..8 exact too, the product
// rounded once at the end; 0: levels 5..8 carried in FP32 per window (the default).
void oz_product(cudaStream_t s, int n, int kp, int sms, const uint8_t* Atiles, const int* emaxA, const double* P,
                uint8_t* Pchunks, int* emaxP, double* Qpart, double* Q, int* err, const SolveState* st, double* part,
                int pstride, int nb, int exp_ready, int once);

// single-warp k x k steps of the loop (small_warp.cu)
void launch_small_sigma(cudaStream_t s, int kp, SolveState* st, const double* Gp, double* Sigma, double* SigmaInv);
void launch_small_xi(cudaStream_t s, int kp, SolveState* st, const double* G1p, const double* Sigma, double* Xi,
                     double* T);
void launch_small_zeta(cudaStream_t s, int kp, SolveState* st, const double* G2nu, double* Sigma, double* Zeta,
                       double* ZetaInv, cudaGraphConditionalHandle cond, int use_cond);
// the pivots' 1/d and 1/sqrt(d) of those steps, elementwise over n values (small_warp.cu)
void launch_pivot_recips(cudaStream_t s, int n, const double* d, double* inv, double* rsq);

// launch shape of the CSR product + Gram entry points, and the thread-local error message (api.cu)
void product_gram_shape(int n, int s, int* kp, int* nb, int* pstride);
int set_last_error(int code, const char* msg);

// kernel-level helpers for the component entry points (api.cu)
__global__ void k_unpack_full(const double* packed, int kp, int s, double* G);
__global__ void k_chol_only(const double* G, int s, double* Z, int* status);

}  // namespace mbpcg
