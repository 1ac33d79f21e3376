"""GB300-native Multi-Basis Parallel Conjugate Gradient (MBPCG).

The solver is the CUDA library libmbpcg.so (C ABI in include/mbpcg.h); this package is its
binding. ``Solver`` wraps a handle: torch provides the device workspace and the stream, the library
does every step of the solve on the GPU (set-up, Algorithm 1 iterations, least-squares exit,
true-residual check). There is no CPU fallback: without a CUDA device creation raises.
"""
from __future__ import annotations

import numpy as np

from . import _native
from ._native import (  # noqa: F401  (re-exported C ABI names)
    Info, MBPCGError, lib, lib_path, mbpcg_create_csr, mbpcg_create_dense, mbpcg_destroy, mbpcg_k_cholesky, mbpcg_k_pivot_reciprocals,
    mbpcg_k_dense_gram, mbpcg_k_dense_product, mbpcg_k_dense_tc_prepare, mbpcg_k_dense_tc_product, mbpcg_k_dense_tc_mma, mbpcg_k_rowprod_tc, mbpcg_k_dense_tc_scratch_bytes, mbpcg_k_spmm, mbpcg_k_spmm_gram_noalloc, mbpcg_k_padded_width, mbpcg_k_scratch_bytes, mbpcg_k_spmm_gram, mbpcg_run_iterations_dev,
    mbpcg_set_launch_mode, mbpcg_solve, mbpcg_solve_dev, mbpcg_workspace_size_csr, mbpcg_workspace_size_dense, status_string, last_error,
    MBPCG_OK, MBPCG_NOT_CONVERGED, MBPCG_BREAKDOWN, MBPCG_PRECOND_NONE, MBPCG_PRECOND_JACOBI, MBPCG_ALGO_MBPCG,
    MBPCG_ALGO_CG, MBPCG_FP64, MBPCG_FP64_TC, MBPCG_MIXED_FP32, MBPCG_LAUNCH_GRAPH, MBPCG_LAUNCH_EAGER,
    mbpcg_k_spmm_gram_f32, mbpcg_k_spmm_f32, mbpcg_k_dense_f32, mbpcg_k_dense_f32_bytes, mbpcg_k_dense_f32_prepare,
    mbpcg_set_residual_mode, MBPCG_RESIDUAL_EXPLICIT,
    MBPCG_RESIDUAL_IMPLICIT, mbpcg_get_spmm_tuning, mbpcg_set_spmm_shape, mbpcg_apply_dev, mbpcg_get_product_kernel,
    mbpcg_set_product_kernel, MBPCG_PRODUCT_CSR_GATHER, MBPCG_PRODUCT_CSR_TILED, MBPCG_PRODUCT_CSR_WIDE, MBPCG_PRODUCT_DENSE,
    MBPCG_PRODUCT_DENSE_TC, MBPCG_PRODUCT_DENSE_FP32, mbpcg_set_product_rounding, MBPCG_ROUND_FP32_TAIL,
    MBPCG_ROUND_ONCE)

from ._native import (  # noqa: F401,E402
    mbpcg_server_create, mbpcg_server_destroy, mbpcg_server_get_stats, mbpcg_server_submit_csr, mbpcg_server_wait)

__all__ = ["Solver", "Server", "Info", "MBPCGError", "lib", "lib_path"]


class Server:
    """The library's continuous-batching request server (include/mbpcg_server.h): up to `slots`
    solves run at once, each on its own stream, admitted first come first served while a slot is
    free and its workspace fits in `hbm_budget_bytes` (0 = 85 % of the free device memory).
    ``submit`` returns a ticket at once; ``wait`` returns the result of a ticket. The arrays of a
    request are kept alive here until its ticket is waited for."""

    def __init__(self, slots: int = 8, hbm_budget_bytes: int = 0):
        self._srv = _native.mbpcg_server_create(slots, hbm_budget_bytes)
        self._keep = {}

    def submit(self, A, b, s: int = 4, precond: int = 0, algo: int = 0, tol: float = 1e-8, maxit: int = 100000,
               seed: int = 0) -> int:
        rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
        v = np.ascontiguousarray(A.val, dtype=np.float64)
        bb = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(int(A.n), dtype=np.float64)
        t = _native.mbpcg_server_submit_csr(self._srv, int(A.n), int(v.size), rp, ci, v, bb, s, precond, algo, tol,
                                            maxit, seed, x)
        self._keep[t] = (rp, ci, v, bb, x)
        return t

    def wait(self, ticket: int) -> dict:
        """{status, x, info, queue_s, run_s}: blocks until the request has finished."""
        st, info, q, r = _native.mbpcg_server_wait(self._srv, ticket)
        x = self._keep.pop(ticket)[4]
        return {"status": st, "x": x, "info": info.as_dict(), "queue_s": q, "run_s": r}

    def stats(self) -> dict:
        return _native.mbpcg_server_get_stats(self._srv)

    def close(self):
        if self._srv is not None:
            _native.mbpcg_server_destroy(self._srv)
            self._srv = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Several Solvers (any mix of matrices, sizes, s, algorithms and precisions, all in graph launch
    mode) whose inner solves run as independent chains of one CUDA graph, launched once per solve
    (mbpcg_batch_*). Each member's result is bit-identical to a solo solve of the same Solver."""

    def __init__(self, solvers):
        import torch
        self.solvers = list(solvers)
        self.stream = torch.cuda.Stream()
        self.b = _native.mbpcg_batch_create([sv.h for sv in self.solvers], self.stream.cuda_stream)

    def solve(self, bs, Us=None, tol: float = 1e-8, maxit: int = 100000):
        """bs (and Us, each None or n x s column-major): numpy arrays, one per member. Returns a
        list of (x, info dict)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        bd = [torch.as_tensor(np.ascontiguousarray(b, dtype=np.float64), device=dev) for b in bs]
        Ud = None
        if Us is not None:
            Ud = [None if U is None else torch.as_tensor(np.asarray(U, dtype=np.float64).T.copy(), device=dev)
                  for U in Us]  # row-major s x n = column-major n x s
        xs = [torch.empty(sv.n, dtype=torch.float64, device=dev) for sv in self.solvers]
        cur = torch.cuda.current_stream()
        for sv in self.solvers:
            sv.stream.wait_stream(cur)
        self.stream.wait_stream(cur)
        st, infos = _native.mbpcg_batch_solve_dev(self.b, bd, Ud, tol, maxit, xs)
        if st not in (MBPCG_OK, MBPCG_NOT_CONVERGED, MBPCG_BREAKDOWN):
            raise MBPCGError(st, "mbpcg_batch_solve_dev")
        return [(x.cpu().numpy(), info.as_dict()) for x, info in zip(xs, infos)]

    def close(self):
        if self.b is not None:
            _native.mbpcg_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Solver:
    """One handle of the library for a fixed matrix and number of copies s.

    A: an object with (n, row_ptr, col_idx, val) numpy arrays (CSR) or (n, a) with a column-major
       n x n array (dense), e.g. ``workloads.CSR`` / ``workloads.Dense``.
    The workspace is a torch uint8 CUDA tensor; calls run on a dedicated torch stream that first
    waits for the caller's current stream."""

    def __init__(self, A, s: int = 4, precond: int = 0, algo: int = 0, seed: int = 0,
                 launch_mode: int = MBPCG_LAUNCH_GRAPH, precision: int = MBPCG_FP64,
                 residual_mode: int = MBPCG_RESIDUAL_EXPLICIT):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("MBPCG needs a CUDA device (GB300, sm_103a); no CPU path exists")
        self.n = int(A.n)
        self.s = int(s) if algo == MBPCG_ALGO_MBPCG else 1
        self.algo = algo
        self.dense = not hasattr(A, "row_ptr")
        # a stream of our own, ordered after the caller's work before every call
        self.stream = torch.cuda.Stream()
        if self.dense:
            nbytes = mbpcg_workspace_size_dense(self.n, self.s, algo, precision)
        else:
            nbytes = mbpcg_workspace_size_csr(self.n, int(A.row_ptr[-1]), self.s, algo, precision)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        if self.dense:
            a = np.asfortranarray(A.a, dtype=np.float64)
            self.h = mbpcg_create_dense(self.n, a, self.s, precond, algo, precision, seed, 0, self.workspace, nbytes,
                                        self.stream.cuda_stream)
        else:
            rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
            ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
            v = np.ascontiguousarray(A.val, dtype=np.float64)
            self.h = mbpcg_create_csr(self.n, int(rp[-1]), rp, ci, v, self.s, precond, algo, precision, seed, 0,
                                      self.workspace, nbytes, self.stream.cuda_stream)
        if launch_mode != MBPCG_LAUNCH_GRAPH:
            st = mbpcg_set_launch_mode(self.h, launch_mode)
            if st != MBPCG_OK:
                raise MBPCGError(st, "mbpcg_set_launch_mode")
        if residual_mode != MBPCG_RESIDUAL_EXPLICIT:
            st = mbpcg_set_residual_mode(self.h, residual_mode)
            if st != MBPCG_OK:
                raise MBPCGError(st, "mbpcg_set_residual_mode")

    def solve(self, b, U=None, tol: float = 1e-8, maxit: int = 100000):
        """Solve A x = b. b (and U, n x s column-major) are numpy arrays (host path, mbpcg_solve)
        or torch CUDA tensors (device path, mbpcg_solve_dev). Returns (x, info dict)."""
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())
        if hasattr(b, "is_cuda") and b.is_cuda:
            x = torch.empty(self.n, dtype=torch.float64, device=b.device)
            Ud = None
            if U is not None:
                Ud = U.t().contiguous() if U.dim() == 2 else U  # column-major n x s == row-major s x n
            st, info = mbpcg_solve_dev(self.h, b, Ud, tol, maxit, x)
        else:
            b = np.ascontiguousarray(b, dtype=np.float64)
            Uh = None if U is None else np.asfortranarray(U, dtype=np.float64)
            x = np.zeros(self.n)
            st, info = mbpcg_solve(self.h, b, Uh, tol, maxit, x)
        if st not in (MBPCG_OK, MBPCG_NOT_CONVERGED, MBPCG_BREAKDOWN):
            raise MBPCGError(st, "mbpcg_solve")
        return x, info.as_dict()

    def spmm_tuning(self):
        """(unroll, ctas_per_sm, times_us) the autotuner chose for the FP32 product (mixed handles)."""
        return mbpcg_get_spmm_tuning(self.h)

    def set_spmm_shape(self, unroll: int, ctas_per_sm: int):
        st = mbpcg_set_spmm_shape(self.h, unroll, ctas_per_sm)
        if st != MBPCG_OK:
            raise MBPCGError(st, "mbpcg_set_spmm_shape")

    def product_kernel(self, fp32: bool = False):
        """(kernel, [gather_us, tiled_us]): the MBPCG_PRODUCT_* kernel of the FP64 (or FP32) product
        and the FP64 times measured at create."""
        return mbpcg_get_product_kernel(self.h, 1 if fp32 else 0)

    def set_product_rounding(self, mode: int):
        """MBPCG_ROUND_FP32_TAIL (default) or MBPCG_ROUND_ONCE for the tensor-core product."""
        st = mbpcg_set_product_rounding(self.h, mode)
        if st != MBPCG_OK:
            raise MBPCGError(st, "mbpcg_set_product_rounding")

    def set_product_kernel(self, kernel: int):
        st = mbpcg_set_product_kernel(self.h, kernel)
        if st != MBPCG_OK:
            raise MBPCGError(st, "mbpcg_set_product_kernel")

    def apply(self, X, fp32: bool = False):
        """A X for a device block X (n x w, w the padded width), by the handle's own product kernel.
        A is the stored operator (scaled under Jacobi). Waits for the result."""
        import torch
        Y = torch.empty_like(X)
        self.stream.wait_stream(torch.cuda.current_stream(X.device))
        st = mbpcg_apply_dev(self.h, 1 if fp32 else 0, X, Y)
        if st != MBPCG_OK:
            raise MBPCGError(st, "mbpcg_apply_dev")
        self.stream.synchronize()
        return Y

    def run_iterations(self, b, U, iters: int):
        """Diagnostic: the state of the scaled system after exactly `iters` iterations, as torch
        tensors (n x s blocks X0, Xt, R, W, P and Sigma s x s)."""
        import torch
        dev = torch.device("cuda")
        self.stream.wait_stream(torch.cuda.current_stream())
        bt = torch.as_tensor(np.ascontiguousarray(b, dtype=np.float64), device=dev)
        Ut = torch.as_tensor(np.ascontiguousarray(np.asarray(U, dtype=np.float64).T), device=dev)
        out = {k: torch.empty((self.s, self.n), dtype=torch.float64, device=dev) for k in ("X0", "Xt", "R", "W", "P")}
        out["Sigma"] = torch.empty((self.s, self.s), dtype=torch.float64, device=dev)
        self.stream.wait_stream(torch.cuda.current_stream())
        st = mbpcg_run_iterations_dev(self.h, bt, Ut, iters, out["X0"], out["Xt"], out["R"], out["W"], out["P"],
                                      out["Sigma"])
        res = {k: v.t().cpu().numpy() for k, v in out.items()}
        return res, st

    def close(self):
        if getattr(self, "h", None):
            mbpcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
