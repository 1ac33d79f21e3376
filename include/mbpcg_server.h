/*
 * mbpcg_server.h -- continuous-batching request server: many MBPCG / CG solves on one GPU.
 *
 * The paper solves one system at a time (Algorithm 1); this layer has no counterpart there. It
 * serves a stream of independent requests (A in CSR form, b, s) the way an inference server serves
 * requests: a request is admitted as soon as a solve slot is free AND its device footprint (the
 * handle's workspace, mbpcg_workspace_size_csr) fits in the remaining HBM budget, so requests
 * that arrive while others run are started without waiting for them. Every slot is a host worker
 * thread with its own CUDA stream; each admitted solve runs Algorithm 1 exactly as mbpcg_solve
 * does, with its loop launched from the slot's thread (MBPCG_LAUNCH_EAGER: per-request CUDA graph
 * instantiation waits for the other slots' device work), so the solves of different slots
 * overlap on the device. Admission is first come, first served.
 *
 * Determinism: every reduction of a solve has a fixed order and every solve has its own
 * workspace, so a request's result is bit-identical whether it runs alone or among others.
 *
 * Memory: workspaces come from the device's stream-ordered allocator (cudaMallocAsync /
 * cudaFreeAsync on the slot's stream), so finishing one request does not synchronise the device.
 *
 * Ownership: the server reads the request's arrays in place and writes x_out in place; the
 * caller keeps row_ptr, col_idx, vals, b and x_out valid and unchanged until mbpcg_server_wait
 * for that ticket has returned. All pointers are host pointers.
 *
 * Errors: int-returning functions return an mbpcg_status (include/mbpcg.h). A failed solve is
 * reported by mbpcg_server_wait (its status, and mbpcg_last_error() in the waiting thread).
 * Threading: submit, wait and get_stats may be called from any threads concurrently.
 */
#ifndef MBPCG_SERVER_H
#define MBPCG_SERVER_H

#include <stddef.h>
#include <stdint.h>

#include "mbpcg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbpcg_server* mbpcg_server_t;

typedef struct {
  int64_t submitted;     /* requests accepted by mbpcg_server_submit_csr */
  int64_t completed;     /* requests whose solve has ended (any status) */
  int64_t failed;        /* of those, status other than MBPCG_OK */
  int32_t active;        /* solves running now */
  int32_t peak_active;   /* most solves running at once so far */
  uint64_t used_bytes;   /* device footprint of the running solves */
  uint64_t peak_bytes;   /* largest footprint admitted at once so far */
  uint64_t budget_bytes; /* admission budget */
} mbpcg_server_stats;

/*
 * Start a server on the current CUDA device.
 *   slots            number of solves that may run at once (worker threads, streams), 1..64.
 *   hbm_budget_bytes device memory the running solves may hold together; 0 = 85 % of the
 *                    free device memory at this call.
 * MBPCG_ERR_INVALID for slots out of range, MBPCG_ERR_CUDA without a usable device.
 */
int mbpcg_server_create(mbpcg_server_t* out, int32_t slots, uint64_t hbm_budget_bytes);

/*
 * Queue one solve of A x = b (A: n x n CSR as in mbpcg_create_csr, host arrays; b and x_out: n
 * doubles). s, precond, algo, tol, maxit and seed mean what they mean for mbpcg_create_csr and
 * mbpcg_solve (U drawn on the device from seed; FP64 arithmetic). On success *ticket identifies
 * the request for mbpcg_server_wait. A request whose footprint exceeds the whole budget is
 * rejected with MBPCG_ERR_OOM; bad sizes give MBPCG_ERR_INVALID (the CSR contents are validated
 * when the solve starts and reported by mbpcg_server_wait).
 */
int mbpcg_server_submit_csr(mbpcg_server_t srv, int32_t n, int64_t nnz, const int32_t* row_ptr,
                            const int32_t* col_idx, const double* vals, const double* b, int32_t s,
                            int32_t precond, int32_t algo, double tol, int32_t maxit, uint64_t seed,
                            double* x_out, int64_t* ticket);

/*
 * Block until the request has finished, then release its ticket. Returns the solve's status;
 * info (may be NULL) as from mbpcg_solve; queue_seconds = submit to start of the solve,
 * run_seconds = start to end of the solve (host steady clock; either may be NULL).
 * MBPCG_ERR_INVALID for an unknown or already released ticket.
 */
int mbpcg_server_wait(mbpcg_server_t srv, int64_t ticket, mbpcg_info* info, double* queue_seconds,
                      double* run_seconds);

/* Counters of the server (see mbpcg_server_stats). */
int mbpcg_server_get_stats(mbpcg_server_t srv, mbpcg_server_stats* out);

/* Finish every queued request, stop the workers and free the server (NULL is ignored). Tickets
 * not yet waited for are released. */
void mbpcg_server_destroy(mbpcg_server_t srv);

#ifdef __cplusplus
}
#endif
#endif
