// mbpcg_k_spmm_gram_noalloc: the A P + P^T(A P) component entry point for callers that cannot
// allocate device memory.
//
// Who needs it: code that must not call cudaMalloc -- a host framework or plugin that owns every
// device allocation and hands out only input/output buffers, a real-time loop where cudaMalloc's
// implicit device synchronisation is not acceptable, or a process whose device memory is already
// committed. mbpcg_k_spmm_gram needs a scratch buffer for its per-CTA partial sums; this variant
// keeps that scratch in a fixed array compiled into the library instead.
//
// The array below is a host-side stand-in in host code, not a device address. Its device address is
// looked up (cudaGetSymbolAddress, with the caller's device current) on the first call in each CUDA
// context and cached under that context's unique id (cuCtxGetId, reached through the runtime's
// driver entry-point query, so the library does not link libcuda). A device reset creates a new
// context with a new id, so the next call looks the address up again; only looked-up addresses are
// passed to kernels.
#include <cuda.h>

#include <mutex>

#include "../../include/mbpcg.h"
#include "../../include/mbpcg_kernels.h"
#include "kernels.h"

namespace {

// Capacity: s <= 16 (partial-slot stride npack(16) + 16 + 1 = 153 -> 156 doubles) and up to 1216
// CTAs (a sparse product launches up to 8 per SM: 1216 on a 152-SM GB300), plus one slot for the
// reduced sums: 1217 * 156 doubles = 1 518 816 bytes, held by every GPU that loads the library
// until exit.
constexpr int kMaxS = 16;
constexpr int kMaxCtas = 1216;
constexpr int kSlot = 156;
constexpr size_t kScratchDoubles = (size_t)(kMaxCtas + 1) * kSlot;

static __device__ __align__(256) double g_spmm_gram_scratch[kScratchDoubles];

typedef CUresult(CUDAAPI* PfnCtxGetCurrent)(CUcontext*);
typedef CUresult(CUDAAPI* PfnCtxGetId)(CUcontext, unsigned long long*);

constexpr int kCacheSlots = 64;
struct CacheEntry {
  unsigned long long ctx_id;
  double* addr;
};
std::mutex g_mutex;
CacheEntry g_cache[kCacheSlots] = {};
int g_cache_next = 0;
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;

// Unique id of the current context (0 when none can be had).
unsigned long long current_context_id() {
  if (g_ctx_get_current == nullptr || g_ctx_get_id == nullptr) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return 0;
    }
    g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
    g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f2);
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the static scratch in the current context (looked up on first use there).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return mbpcg::set_last_error(MBPCG_ERR_CUDA, "mbpcg_k_spmm_gram_noalloc: no usable current device");
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  unsigned long long id = current_context_id();  // 0 before the runtime has made a context current
  for (int q = 0; id != 0 && q < kCacheSlots; ++q) {
    if (g_cache[q].ctx_id == id && g_cache[q].addr != nullptr) {
      *out = g_cache[q].addr;
      return MBPCG_OK;
    }
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_spmm_gram_scratch);  // makes the context current if needed
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return mbpcg::set_last_error(MBPCG_ERR_CUDA, "mbpcg_k_spmm_gram_noalloc: cudaGetSymbolAddress failed");
  }
  if (id == 0) id = current_context_id();
  if (id == 0) return mbpcg::set_last_error(MBPCG_ERR_CUDA, "mbpcg_k_spmm_gram_noalloc: no current CUDA context");
  g_cache[g_cache_next] = {id, static_cast<double*>(p)};
  g_cache_next = (g_cache_next + 1) % kCacheSlots;
  *out = static_cast<double*>(p);
  return MBPCG_OK;
}

}  // namespace

extern "C" int mbpcg_k_spmm_gram_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                         const double* vals, int32_t s, const double* P, double* AP, double* G,
                                         void* stream) {
  if (n < 1 || s < 1 || !row_ptr || !P || !AP || !G)
    return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_k_spmm_gram_noalloc: bad arguments");
  if (s > kMaxS)
    return mbpcg::set_last_error(MBPCG_ERR_INVALID,
                                 "mbpcg_k_spmm_gram_noalloc: s exceeds 16, the limit of its static scratch "
                                 "(use mbpcg_k_spmm_gram with caller-provided scratch)");
  int kp = 0, nb = 0, pstride = 0;
  mbpcg::product_gram_shape(n, s, &kp, &nb, &pstride);
  if (nb > kMaxCtas || pstride > kSlot)
    return mbpcg::set_last_error(MBPCG_ERR_INVALID,
                                 "mbpcg_k_spmm_gram_noalloc: launch needs more partial slots than its static "
                                 "scratch holds (more than 1216 CTAs)");
  double* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != MBPCG_OK) return rc;
  // Every partial slot the reduction reads (nb of them) is fully written by this call's product
  // kernel first, so nothing in the array has to start at zero.
  double* red = scratch + (size_t)kMaxCtas * kSlot;
  cudaStream_t st = (cudaStream_t)stream;
  mbpcg::row_ops(kp)->spmm(st, nb, n, row_ptr, col_idx, vals, P, AP, scratch, kSlot, nullptr, 1);
  mbpcg::launch_reduce(st, scratch, nb, kSlot, red, mbpcg::npack(kp), nullptr);
  mbpcg::k_unpack_full<<<1, 256, 0, st>>>(red, kp, s, G);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return mbpcg::set_last_error(MBPCG_ERR_CUDA, cudaGetErrorString(e));
  return MBPCG_OK;
}
