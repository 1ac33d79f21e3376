/*
 * mbpcg_kernels.h -- component entry points of the MBPCG library, for callers (and tests) that
 * drive single steps of Algorithm 1 on their own device buffers.
 *
 * All pointers are DEVICE pointers; calls are asynchronous on `stream` (a cudaStream_t, NULL =
 * legacy default stream) and return after enqueueing. Blocks are row-major n x kp with
 * kp = mbpcg_k_padded_width(s) (s rounded up to a power of two); columns s..kp-1 of P must be
 * zero. Small outputs are column-major s x s doubles. Errors: MBPCG_ERR_INVALID for bad
 * arguments, MBPCG_ERR_CUDA for a failed launch (mbpcg_last_error() has the message).
 */
#ifndef MBPCG_KERNELS_H
#define MBPCG_KERNELS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Padded row width used for s copies (1, 2, 4, 8, 16 or 32); 0 when s is outside [1, 32]. */
int32_t mbpcg_k_padded_width(int32_t s);

/* Bytes of device scratch the product+Gram entry points need (per-CTA partial sums). The caller
 * allocates it; contents need no initialisation and are overwritten. */
size_t mbpcg_k_scratch_bytes(int32_t n, int32_t s);

/*
 * The A P product of Algorithm 1 (the step that dominates Table 2 of the paper) fused with the
 * Gram matrix that defines Xi: AP = A P for CSR A (int32 row_ptr[n+1], int32 col_idx, double
 * vals), and G = P^T (A P) (s x s, symmetric; the upper triangle is accumulated and mirrored).
 * Summation order is fixed, so repeated calls give identical bits.
 */
int mbpcg_k_spmm_gram(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                      int32_t s, const double* P, double* AP, double* G, void* scratch,
                      size_t scratch_bytes, void* stream);

/*
 * mbpcg_k_spmm_gram without any device allocation. The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc (a host framework or plugin that owns all device memory,
 * a real-time loop that cannot afford cudaMalloc's device synchronisation, a process with no
 * device memory left to give). Its scratch is a fixed array of about 1.5 MB compiled into the
 * library, which every GPU that loads the library holds until the process exits; nothing is
 * allocated or freed. Limits: s <= 16 and at most 1216 CTAs of partial sums (a GB300 uses up to
 * 1216: 8 per SM);
 * larger requests return MBPCG_ERR_INVALID with a message. The first call in each CUDA context (per
 * device, and again after a device reset) looks up the array's device address, so make that first
 * call before any stream capture. All calls share
 * the one array: calls whose work overlaps on the GPU (e.g. on two streams) race and give wrong
 * results; serialise them. Inputs, outputs and errors are those of mbpcg_k_spmm_gram.
 */
int mbpcg_k_spmm_gram_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                              const double* vals, int32_t s, const double* P, double* AP,
                              double* G, void* stream);

/*
 * The FP32 form used by the mixed-precision inner solve (MBPCG_MIXED_FP32): vals, P and AP are
 * FP32 (P, AP row-major n x KP as above), AP = A P with FP32 accumulation, and G = P^T (A P) (s x s
 * FP64) accumulated from the FP32 values with compensated dot products (Ogita, Rump & Oishi 2005:
 * as accurate as a sum in twice FP32's precision). Scratch and errors as mbpcg_k_spmm_gram.
 * mbpcg_k_spmm_f32 is the product alone (no Gram, no scratch), in the solver's launch
 * configuration, for timing.
 */
int mbpcg_k_spmm_gram_f32(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const float* vals,
                          int32_t s, const float* P, float* AP, double* G, void* scratch,
                          size_t scratch_bytes, void* stream);
int mbpcg_k_spmm_f32(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const float* vals,
                     int32_t s, const float* P, float* AP, void* stream);

/*
 * The FP32 dense product of the mixed-precision inner solve on a dense A (MBPCG_MIXED_FP32 with
 * mbpcg_create_dense; the Xi step's A P of Algorithm 1), in two calls like the tensor-core product:
 *   mbpcg_k_dense_f32_bytes: size of the FP32 copy of A (tiles of 256 rows x 32 columns, zero
 *     past n; 0 for n < 1).
 *   mbpcg_k_dense_f32_prepare: writes that copy from A (device, column-major FP64 n x n, symmetric:
 *     row i is read as column i) into `tiles` (device, 16-byte aligned, tiles_bytes at least
 *     mbpcg_k_dense_f32_bytes(n)). Each entry is A rounded to FP32.
 *   mbpcg_k_dense_f32: AP = A P from the tiles, FP32 accumulation, in the solver's launch
 *     configuration. P, AP: device FP32 row-major n x KP (KP = mbpcg_k_padded_width(s)), P
 *     16-byte aligned; AP is written, columns s..KP-1 get A times P's (zero) padding. The order of
 *     accumulation is fixed for a given device (K split over a cluster of CTAs, summed in rank
 *     order), so repeated calls give identical bits; error <= n 2^-24 |A||P|. No scratch.
 * MBPCG_ERR_INVALID for bad sizes, pointers or alignment.
 */
size_t mbpcg_k_dense_f32_bytes(int32_t n);
int mbpcg_k_dense_f32_prepare(int32_t n, const double* A, void* tiles, size_t tiles_bytes, void* stream);
int mbpcg_k_dense_f32(int32_t n, const void* tiles, int32_t s, const float* P, float* AP, void* stream);

/* Same for dense symmetric A (column-major n x n; row i is read as column i). */
int mbpcg_k_dense_gram(int32_t n, const double* A, int32_t s, const double* P, double* AP,
                       double* G, void* scratch, size_t scratch_bytes, void* stream);

/* The product alone, in the launch configuration the solver uses inside its iteration loop:
 * AP = A P for CSR A (mbpcg_k_spmm) or dense symmetric column-major A (mbpcg_k_dense_product).
 * No scratch. Used to time the dominant kernel of an iteration in isolation. */
int mbpcg_k_spmm(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                 int32_t s, const double* P, double* AP, void* stream);
int mbpcg_k_dense_product(int32_t n, const double* A, int32_t s, const double* P, double* AP,
                          void* stream);

/* The tensor-core form of the dense product (precision MBPCG_FP64_TC), as accurate as an FP64
 * product. mbpcg_k_dense_tc_prepare writes the base-128 digits of A into `scratch` as bytes (8 per
 * entry; mbpcg_k_dense_tc_scratch_bytes(n, s) bytes of device memory, 256-byte aligned);
 * mbpcg_k_dense_tc_product then splits P into FP16 digits and computes AP = A P with tcgen05 MMAs
 * (the digits of A converted to FP16 operands on chip), reusing them. */
size_t mbpcg_k_dense_tc_scratch_bytes(int32_t n, int32_t s);
int mbpcg_k_dense_tc_prepare(int32_t n, const double* A, int32_t s, void* scratch,
                             size_t scratch_bytes, void* stream);
int mbpcg_k_dense_tc_product(int32_t n, int32_t s, const double* P, double* AP, void* scratch,
                             size_t scratch_bytes, void* stream);
/* The MMA kernel of the tensor-core product alone (k_dense_tc: the digit stream of A and the
 * tcgen05 MMAs; no splitting of P, no split sum), in the launch configuration of the product, on
 * the digits of P that the last mbpcg_k_dense_tc_product call left in `scratch`. It writes only
 * partial sums inside scratch -- never AP -- and they are not a product (that call's split sum
 * has already cleared the column exponents of P): it exists to time the dominant kernel of an
 * iteration in isolation. Arguments and errors as mbpcg_k_dense_tc_product. */
int mbpcg_k_dense_tc_mma(int32_t n, int32_t s, void* scratch, size_t scratch_bytes, void* stream);

/* The k x k-row products of the block update and of the W/P update of Algorithm 1 (P T, (AP) T,
 * (AP) Xi, V zeta^{-1}, P zeta^T) as the solver runs them for tensor-core handles at s > 8:
 * Y = X M on the FP16 tensor cores by exact digit splitting (X row by row, M column by column;
 * 8 base-128 digits each), with the accuracy of an FP64 product: error about 2^-53 times
 * (max_l |X_il|) (sum_l |M_lj|) per entry, against an FP64 product's w u sum_l |X_il||M_lj|.
 * width = 32 or 16 (the padded width KP). X, Y: device, row-major n x width FP64, 16-byte
 * aligned; M: device, column-major width x width FP64, used as M (transM = 0) or as its
 * transpose (transM = 1). Y is written. No scratch.
 * MBPCG_ERR_INVALID for bad sizes, width, pointers or alignment. */
int mbpcg_k_rowprod_tc(int32_t n, int32_t width, const double* X, const double* M, int32_t transM, double* Y,
                       void* stream);

/* Z = upper Cholesky factor of the SPD s x s matrix G (G = Z^T Z, positive diagonal), the k x k
 * factorisation used for Xi (Section 3) and for the Cholesky QR. *status_dev (device int) is set
 * to 0, or to 6 (MBPCG_BREAKDOWN) when a pivot is not finite or not above 64 eps max_j G_jj. */
int mbpcg_k_cholesky(int32_t s, const double* G, double* Z, int32_t* status_dev, void* stream);

/* The reciprocal 1/d and the inverse square root 1/sqrt(d) that the loop's k x k steps take of
 * their pivots (the LDL^T elimination behind Xi = (P^T A P)^{-1} and the Cholesky QR of V,
 * Section 3): the FP32 hardware approximation of d's leading 23 significand bits, rescaled by d's
 * exponent with integer operations, then one third-order Newton step in FP64. For a positive
 * normal d below 2^1000 (the only pivots those steps accept) inv is within 0.51 ulp of 1/d and rsq
 * within 1.01 ulp of 1/sqrt(d); other d give unspecified values, with no error. d, inv, rsq:
 * device, n doubles each; inv and rsq are written. MBPCG_ERR_INVALID for n < 1 or a NULL pointer. */
int mbpcg_k_pivot_reciprocals(int32_t n, const double* d, double* inv, double* rsq, void* stream);

#ifdef __cplusplus
}
#endif
#endif
