// Continuous-batching request server (include/mbpcg_server.h): worker threads, one CUDA stream
// each, admitting queued solves first come first served while a slot is free and the solve's
// workspace fits in the HBM budget. Each admitted solve is an ordinary handle (mbpcg_create_csr on
// a workspace from the stream-ordered allocator, mbpcg_solve, mbpcg_destroy) on the slot's stream.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "mbpcg.h"
#include "mbpcg_server.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kWsAlign = 256;  // workspace alignment the handle requires

struct Request {
  int64_t id = 0;
  int32_t n = 0;
  int64_t nnz = 0;
  const int32_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* vals = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  int32_t s = 1, precond = 0, algo = 0, maxit = 0;
  double tol = 0.0;
  uint64_t seed = 0;
  size_t ws_bytes = 0;  // workspace the handle needs
  size_t bytes = 0;     // admitted footprint (workspace + alignment slack)
  Clock::time_point t_submit, t_start, t_end;
  int status = MBPCG_OK;
  mbpcg_info info{};
  std::string error;
  bool done = false;
};

}  // namespace

struct mbpcg_server {
  int device = 0;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::mutex mu;
  std::condition_variable cv;  // queue changed, memory freed, a request finished, stop
  std::deque<Request*> queue;
  std::unordered_map<int64_t, Request*> live;
  int64_t next_id = 1;
  bool stop = false;
  mbpcg_server_stats stats{};
};

namespace {

// One solve on the slot's stream; fills status, info, error.
void run_request(Request* r, cudaStream_t stream) {
  void* raw = nullptr;
  if (cudaMallocAsync(&raw, r->bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    r->status = MBPCG_ERR_OOM;
    r->error = "cudaMallocAsync of the request's workspace failed";
    return;
  }
  void* ws = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(raw) + kWsAlign - 1) / kWsAlign * kWsAlign);
  mbpcg_handle h = nullptr;
  int st = mbpcg_create_csr(&h, r->n, r->nnz, r->rp, r->ci, r->vals, r->s, r->precond, r->algo, MBPCG_FP64,
                            r->seed, 0, ws, r->ws_bytes, stream);
  // Host-launched loop: building and instantiating a CUDA graph per request waits for the other
  // slots' device work (measured: 8 concurrent first solves 39 ms each against 8.7 ms alone), which
  // would serialise the slots; launching the same kernels from the slot's thread does not.
  if (st == MBPCG_OK) st = mbpcg_set_launch_mode(h, MBPCG_LAUNCH_EAGER);
  if (st == MBPCG_OK) st = mbpcg_solve(h, r->b, nullptr, r->tol, r->maxit, r->x, &r->info);
  if (st != MBPCG_OK) r->error = mbpcg_last_error();
  mbpcg_destroy(h);  // synchronises the slot's stream only
  cudaFreeAsync(raw, stream);
  if (cudaStreamSynchronize(stream) != cudaSuccess && st == MBPCG_OK) {
    st = MBPCG_ERR_CUDA;
    r->error = cudaGetErrorString(cudaGetLastError());
  }
  r->status = st;
}

void worker_main(mbpcg_server* S, int slot) {
  cudaSetDevice(S->device);
  cudaStream_t stream = S->streams[slot];
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] {
        if (S->queue.empty()) return S->stop;
        return S->stats.used_bytes + S->queue.front()->bytes <= S->stats.budget_bytes;
      });
      if (S->queue.empty()) return;  // stop requested and nothing left
      r = S->queue.front();
      S->queue.pop_front();
      S->stats.used_bytes += r->bytes;
      S->stats.active += 1;
      if (S->stats.active > S->stats.peak_active) S->stats.peak_active = S->stats.active;
      if (S->stats.used_bytes > S->stats.peak_bytes) S->stats.peak_bytes = S->stats.used_bytes;
    }
    r->t_start = Clock::now();
    run_request(r, stream);
    r->t_end = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stats.used_bytes -= r->bytes;
      S->stats.active -= 1;
      S->stats.completed += 1;
      if (r->status != MBPCG_OK) S->stats.failed += 1;
      r->done = true;
    }
    S->cv.notify_all();
  }
}

}  // namespace

extern "C" {

int mbpcg_server_create(mbpcg_server_t* out, int32_t slots, uint64_t hbm_budget_bytes) {
  if (out == nullptr) return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_server_create: out is NULL");
  *out = nullptr;
  if (slots < 1 || slots > 64)
    return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_server_create: slots must be in [1, 64]");
  int dev = 0;
  size_t free_b = 0, total_b = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return mbpcg::set_last_error(MBPCG_ERR_CUDA, "mbpcg_server_create: no usable CUDA device");
  }
  mbpcg_server* S = new (std::nothrow) mbpcg_server;
  if (S == nullptr) return mbpcg::set_last_error(MBPCG_ERR_OOM, "mbpcg_server_create: host allocation failed");
  S->device = dev;
  S->stats.budget_bytes = hbm_budget_bytes ? hbm_budget_bytes : (uint64_t)(0.85 * (double)free_b);
  // keep freed workspaces in the allocator's pool instead of returning them at every synchronisation
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  S->streams.resize(slots);
  for (int i = 0; i < slots; ++i) {
    if (cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < i; ++j) cudaStreamDestroy(S->streams[j]);
      delete S;
      return mbpcg::set_last_error(MBPCG_ERR_CUDA, "mbpcg_server_create: cudaStreamCreate failed");
    }
  }
  for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker_main, S, i);
  *out = S;
  return MBPCG_OK;
}

int mbpcg_server_submit_csr(mbpcg_server_t S, int32_t n, int64_t nnz, const int32_t* row_ptr,
                            const int32_t* col_idx, const double* vals, const double* b, int32_t s,
                            int32_t precond, int32_t algo, double tol, int32_t maxit, uint64_t seed,
                            double* x_out, int64_t* ticket) {
  const Clock::time_point now = Clock::now();
  if (S == nullptr || ticket == nullptr)
    return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_server_submit_csr: server or ticket is NULL");
  if (n < 1 || nnz < 0 || nnz >= (int64_t)1 << 31 || row_ptr == nullptr || b == nullptr || x_out == nullptr ||
      (nnz > 0 && (col_idx == nullptr || vals == nullptr)))
    return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_server_submit_csr: bad sizes or NULL arrays");
  if (algo == MBPCG_ALGO_MBPCG && (s < 1 || s > 32))
    return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_server_submit_csr: s must be in [1, 32]");
  if (!(tol > 0.0) || maxit < 1)
    return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_server_submit_csr: tol must be > 0, maxit >= 1");
  Request* r = new (std::nothrow) Request;
  if (r == nullptr) return mbpcg::set_last_error(MBPCG_ERR_OOM, "mbpcg_server_submit_csr: host allocation failed");
  r->n = n;
  r->nnz = nnz;
  r->rp = row_ptr;
  r->ci = col_idx;
  r->vals = vals;
  r->b = b;
  r->x = x_out;
  r->s = s;
  r->precond = precond;
  r->algo = algo;
  r->tol = tol;
  r->maxit = maxit;
  r->seed = seed;
  r->ws_bytes = mbpcg_workspace_size_csr(n, nnz, s, algo, MBPCG_FP64);
  r->bytes = r->ws_bytes + kWsAlign;
  r->t_submit = now;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->bytes > S->stats.budget_bytes) {
      delete r;
      return mbpcg::set_last_error(MBPCG_ERR_OOM, "mbpcg_server_submit_csr: the request needs more device memory "
                                                  "than the server's whole budget");
    }
    r->id = S->next_id++;
    S->live[r->id] = r;
    S->queue.push_back(r);
    S->stats.submitted += 1;
    *ticket = r->id;
  }
  S->cv.notify_all();
  return MBPCG_OK;
}

int mbpcg_server_wait(mbpcg_server_t S, int64_t ticket, mbpcg_info* info, double* queue_seconds,
                      double* run_seconds) {
  if (S == nullptr) return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_server_wait: server is NULL");
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->live.find(ticket);
    if (it == S->live.end()) return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_server_wait: unknown ticket");
    r = it->second;
    S->cv.wait(lk, [&] { return r->done; });
    S->live.erase(ticket);
  }
  if (info != nullptr) *info = r->info;
  if (queue_seconds != nullptr) *queue_seconds = std::chrono::duration<double>(r->t_start - r->t_submit).count();
  if (run_seconds != nullptr) *run_seconds = std::chrono::duration<double>(r->t_end - r->t_start).count();
  const int st = r->status;
  if (st != MBPCG_OK) mbpcg::set_last_error(st, r->error.c_str());
  delete r;
  return st;
}

int mbpcg_server_get_stats(mbpcg_server_t S, mbpcg_server_stats* out) {
  if (S == nullptr || out == nullptr)
    return mbpcg::set_last_error(MBPCG_ERR_INVALID, "mbpcg_server_get_stats: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  return MBPCG_OK;
}

void mbpcg_server_destroy(mbpcg_server_t S) {
  if (S == nullptr) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto& kv : S->live) delete kv.second;
    S->live.clear();
  }
  delete S;
}

}  // extern "C"
