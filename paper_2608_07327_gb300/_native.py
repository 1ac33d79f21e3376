"""ctypes binding of libmbpcg.so: the C ABI of include/mbpcg.h and include/mbpcg_kernels.h under the
same names, with argument marshalling only (numpy arrays -> host pointers, torch CUDA tensors ->
device pointers). Every computation runs in the CUDA library; there is no Python or CPU path, and
loading fails loudly when the library cannot be built or loaded."""
from __future__ import annotations

import ctypes
import threading

from . import build as _build

MBPCG_OK = 0
MBPCG_ERR_INVALID = 1
MBPCG_ERR_OOM = 2
MBPCG_ERR_CUDA = 3
MBPCG_ERR_NOT_SPD = 4
MBPCG_NOT_CONVERGED = 5
MBPCG_BREAKDOWN = 6
MBPCG_ERR_TIMEOUT = 7
MBPCG_PRECOND_NONE = 0
MBPCG_PRECOND_JACOBI = 1
MBPCG_ALGO_MBPCG = 0
MBPCG_ALGO_CG = 1
MBPCG_FP64 = 0
MBPCG_MIXED_FP32 = 1
MBPCG_MIXED_BF16 = 2
MBPCG_FP64_TC = 3
MBPCG_LAUNCH_GRAPH = 0
MBPCG_LAUNCH_EAGER = 1
MBPCG_RESIDUAL_EXPLICIT = 0
MBPCG_RESIDUAL_IMPLICIT = 1
MBPCG_ROUND_FP32_TAIL = 0
MBPCG_ROUND_ONCE = 1
MBPCG_PRODUCT_CSR_GATHER = 0
MBPCG_PRODUCT_CSR_TILED = 1
MBPCG_PRODUCT_CSR_WIDE = 2
MBPCG_PRODUCT_DENSE = 3
MBPCG_PRODUCT_DENSE_TC = 4
MBPCG_PRODUCT_DENSE_FP32 = 5


class Info(ctypes.Structure):
    """mbpcg_info."""
    _fields_ = [
        ("iterations", ctypes.c_int32),
        ("restarts", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("best_col", ctypes.c_int32),
        ("ls_fallback", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("relres_recurrence", ctypes.c_double),
        ("relres_ls", ctypes.c_double),
        ("relres_true", ctypes.c_double),
        ("seconds", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class ServerStats(ctypes.Structure):
    """mbpcg_server_stats."""
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("failed", ctypes.c_int64),
        ("active", ctypes.c_int32),
        ("peak_active", ctypes.c_int32),
        ("used_bytes", ctypes.c_uint64),
        ("peak_bytes", ctypes.c_uint64),
        ("budget_bytes", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class MBPCGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status}): {last_error()}")


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_D = ctypes.c_double

_SIGS = {
    "mbpcg_workspace_size_csr": (_SZ, [_I32, _I64, _I32, _I32, _I32]),
    "mbpcg_workspace_size_dense": (_SZ, [_I32, _I32, _I32, _I32]),
    "mbpcg_create_csr": (ctypes.c_int, [ctypes.POINTER(_P), _I32, _I64, _P, _P, _P, _I32, _I32, _I32, _I32,
                                        ctypes.c_uint64, _I32, _P, _SZ, _P]),
    "mbpcg_create_dense": (ctypes.c_int, [ctypes.POINTER(_P), _I32, _P, _I32, _I32, _I32, _I32, ctypes.c_uint64,
                                          _I32, _P, _SZ, _P]),
    "mbpcg_solve": (ctypes.c_int, [_P, _P, _P, _D, _I32, _P, ctypes.POINTER(Info)]),
    "mbpcg_solve_dev": (ctypes.c_int, [_P, _P, _P, _D, _I32, _P, ctypes.POINTER(Info)]),
    "mbpcg_run_iterations_dev": (ctypes.c_int, [_P, _P, _P, _I32, _P, _P, _P, _P, _P, _P]),
    "mbpcg_destroy": (None, [_P]),
    "mbpcg_set_launch_mode": (ctypes.c_int, [_P, _I32]),
    "mbpcg_set_residual_mode": (ctypes.c_int, [_P, _I32]),
    "mbpcg_get_spmm_tuning": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                             ctypes.POINTER(ctypes.c_float)]),
    "mbpcg_set_spmm_shape": (ctypes.c_int, [_P, _I32, _I32]),
    "mbpcg_apply_dev": (ctypes.c_int, [_P, _I32, _P, _P]),
    "mbpcg_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), _I32, _P]),
    "mbpcg_batch_solve_dev": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I32,
                                             ctypes.POINTER(_P), ctypes.POINTER(Info)]),
    "mbpcg_batch_destroy": (None, [_P]),
    "mbpcg_get_product_kernel": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_float)]),
    "mbpcg_set_product_kernel": (ctypes.c_int, [_P, _I32]),
    "mbpcg_set_product_rounding": (ctypes.c_int, [_P, _I32]),
    "mbpcg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mbpcg_last_error": (ctypes.c_char_p, []),
    "mbpcg_k_padded_width": (_I32, [_I32]),
    "mbpcg_k_scratch_bytes": (_SZ, [_I32, _I32]),
    "mbpcg_k_spmm_gram": (ctypes.c_int, [_I32, _P, _P, _P, _I32, _P, _P, _P, _P, _SZ, _P]),
    "mbpcg_k_dense_gram": (ctypes.c_int, [_I32, _P, _I32, _P, _P, _P, _P, _SZ, _P]),
    "mbpcg_k_cholesky": (ctypes.c_int, [_I32, _P, _P, _P, _P]),
    "mbpcg_k_pivot_reciprocals": (ctypes.c_int, [_I32, _P, _P, _P, _P]),
    "mbpcg_k_dense_tc_scratch_bytes": (_SZ, [_I32, _I32]),
    "mbpcg_k_dense_tc_prepare": (ctypes.c_int, [_I32, _P, _I32, _P, _SZ, _P]),
    "mbpcg_k_dense_tc_product": (ctypes.c_int, [_I32, _I32, _P, _P, _P, _SZ, _P]),
    "mbpcg_k_dense_tc_mma": (ctypes.c_int, [_I32, _I32, _P, _SZ, _P]),
    "mbpcg_k_rowprod_tc": (ctypes.c_int, [_I32, _I32, _P, _P, _I32, _P, _P]),
    "mbpcg_k_spmm_gram_noalloc": (ctypes.c_int, [_I32, _P, _P, _P, _I32, _P, _P, _P, _P]),
    "mbpcg_k_spmm": (ctypes.c_int, [_I32, _P, _P, _P, _I32, _P, _P, _P]),
    "mbpcg_k_spmm_gram_f32": (ctypes.c_int, [_I32, _P, _P, _P, _I32, _P, _P, _P, _P, _SZ, _P]),
    "mbpcg_k_spmm_f32": (ctypes.c_int, [_I32, _P, _P, _P, _I32, _P, _P, _P]),
    "mbpcg_k_dense_f32_bytes": (ctypes.c_size_t, [_I32]),
    "mbpcg_k_dense_f32_prepare": (ctypes.c_int, [_I32, _P, _P, ctypes.c_size_t, _P]),
    "mbpcg_k_dense_f32": (ctypes.c_int, [_I32, _P, _I32, _P, _P, _P]),
    "mbpcg_k_dense_product": (ctypes.c_int, [_I32, _P, _I32, _P, _P, _P]),
    "mbpcg_server_create": (ctypes.c_int, [ctypes.POINTER(_P), _I32, ctypes.c_uint64]),
    "mbpcg_server_submit_csr": (ctypes.c_int, [_P, _I32, _I64, _P, _P, _P, _P, _I32, _I32, _I32, _D, _I32,
                                               ctypes.c_uint64, _P, ctypes.POINTER(_I64)]),
    "mbpcg_server_wait": (ctypes.c_int, [_P, _I64, ctypes.POINTER(Info), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "mbpcg_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "mbpcg_server_destroy": (None, [_P]),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libmbpcg.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def ptr(x):
    """Raw address of a numpy array / torch tensor / int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)!r}")


def status_string(status: int) -> str:
    return lib().mbpcg_status_string(status).decode()


def last_error() -> str:
    return lib().mbpcg_last_error().decode()


def mbpcg_workspace_size_csr(n, nnz, s, algo=MBPCG_ALGO_MBPCG, precision=MBPCG_FP64) -> int:
    return int(lib().mbpcg_workspace_size_csr(n, nnz, s, algo, precision))


def mbpcg_workspace_size_dense(n, s, algo=MBPCG_ALGO_MBPCG, precision=MBPCG_FP64) -> int:
    return int(lib().mbpcg_workspace_size_dense(n, s, algo, precision))


def mbpcg_create_csr(n, nnz, row_ptr, col_idx, vals, s, precond=0, algo=0, precision=0, seed=0, mem=0,
                     workspace=None, workspace_bytes=0, stream=None):
    h = _P()
    st = lib().mbpcg_create_csr(ctypes.byref(h), n, nnz, ptr(row_ptr), ptr(col_idx), ptr(vals), s, precond, algo,
                                precision, seed, mem, ptr(workspace), workspace_bytes, stream)
    if st != MBPCG_OK:
        raise MBPCGError(st, "mbpcg_create_csr")
    return h


def mbpcg_create_dense(n, A, s, precond=0, algo=0, precision=0, seed=0, mem=0, workspace=None, workspace_bytes=0,
                       stream=None):
    h = _P()
    st = lib().mbpcg_create_dense(ctypes.byref(h), n, ptr(A), s, precond, algo, precision, seed, mem,
                                  ptr(workspace), workspace_bytes, stream)
    if st != MBPCG_OK:
        raise MBPCGError(st, "mbpcg_create_dense")
    return h


def mbpcg_solve(h, b, U, tol, maxit, x_out):
    info = Info()
    st = lib().mbpcg_solve(h, ptr(b), ptr(U), tol, maxit, ptr(x_out), ctypes.byref(info))
    return st, info


def mbpcg_solve_dev(h, b, U, tol, maxit, x_out):
    info = Info()
    st = lib().mbpcg_solve_dev(h, ptr(b), ptr(U), tol, maxit, ptr(x_out), ctypes.byref(info))
    return st, info


def mbpcg_run_iterations_dev(h, b, U, iters, X0=None, Xt=None, R=None, W=None, P=None, Sigma=None):
    return lib().mbpcg_run_iterations_dev(h, ptr(b), ptr(U), iters, ptr(X0), ptr(Xt), ptr(R), ptr(W), ptr(P),
                                          ptr(Sigma))


def mbpcg_set_launch_mode(h, mode):
    return lib().mbpcg_set_launch_mode(h, mode)


def mbpcg_destroy(h):
    if h:
        lib().mbpcg_destroy(h)


def mbpcg_k_padded_width(s) -> int:
    return int(lib().mbpcg_k_padded_width(s))


def mbpcg_k_scratch_bytes(n, s) -> int:
    return int(lib().mbpcg_k_scratch_bytes(n, s))


def mbpcg_k_spmm_gram(n, row_ptr, col_idx, vals, s, P, AP, G, scratch, scratch_bytes, stream=None):
    return lib().mbpcg_k_spmm_gram(n, ptr(row_ptr), ptr(col_idx), ptr(vals), s, ptr(P), ptr(AP), ptr(G),
                                   ptr(scratch), scratch_bytes, stream)


def mbpcg_k_spmm_gram_noalloc(n, row_ptr, col_idx, vals, s, P, AP, G, stream=None):
    return lib().mbpcg_k_spmm_gram_noalloc(n, ptr(row_ptr), ptr(col_idx), ptr(vals), s, ptr(P), ptr(AP), ptr(G),
                                           stream)


def mbpcg_k_dense_gram(n, A, s, P, AP, G, scratch, scratch_bytes, stream=None):
    return lib().mbpcg_k_dense_gram(n, ptr(A), s, ptr(P), ptr(AP), ptr(G), ptr(scratch), scratch_bytes, stream)


def mbpcg_k_spmm(n, row_ptr, col_idx, vals, s, P, AP, stream=None):
    return lib().mbpcg_k_spmm(n, ptr(row_ptr), ptr(col_idx), ptr(vals), s, ptr(P), ptr(AP), stream)


def mbpcg_k_spmm_gram_f32(n, row_ptr, col_idx, vals, s, P, AP, G, scratch, scratch_bytes, stream=None):
    return lib().mbpcg_k_spmm_gram_f32(n, ptr(row_ptr), ptr(col_idx), ptr(vals), s, ptr(P), ptr(AP), ptr(G),
                                       ptr(scratch), scratch_bytes, stream)


def mbpcg_k_spmm_f32(n, row_ptr, col_idx, vals, s, P, AP, stream=None):
    return lib().mbpcg_k_spmm_f32(n, ptr(row_ptr), ptr(col_idx), ptr(vals), s, ptr(P), ptr(AP), stream)


def mbpcg_k_dense_f32_bytes(n):
    return lib().mbpcg_k_dense_f32_bytes(n)


def mbpcg_k_dense_f32_prepare(n, A, tiles, tiles_bytes, stream=None):
    return lib().mbpcg_k_dense_f32_prepare(n, ptr(A), ptr(tiles), tiles_bytes, stream)


def mbpcg_k_dense_f32(n, tiles, s, P, AP, stream=None):
    return lib().mbpcg_k_dense_f32(n, ptr(tiles), s, ptr(P), ptr(AP), stream)


def mbpcg_k_dense_product(n, A, s, P, AP, stream=None):
    return lib().mbpcg_k_dense_product(n, ptr(A), s, ptr(P), ptr(AP), stream)


def mbpcg_k_dense_tc_scratch_bytes(n, s) -> int:
    return int(lib().mbpcg_k_dense_tc_scratch_bytes(n, s))


def mbpcg_k_dense_tc_prepare(n, A, s, scratch, scratch_bytes, stream=None):
    return lib().mbpcg_k_dense_tc_prepare(n, ptr(A), s, ptr(scratch), scratch_bytes, stream)


def mbpcg_k_rowprod_tc(n, width, X, M, transM, Y, stream=None):
    return lib().mbpcg_k_rowprod_tc(n, width, ptr(X), ptr(M), transM, ptr(Y), stream)


def mbpcg_k_dense_tc_mma(n, s, scratch, scratch_bytes, stream=None):
    return lib().mbpcg_k_dense_tc_mma(n, s, ptr(scratch), scratch_bytes, stream)


def mbpcg_k_dense_tc_product(n, s, P, AP, scratch, scratch_bytes, stream=None):
    return lib().mbpcg_k_dense_tc_product(n, s, ptr(P), ptr(AP), ptr(scratch), scratch_bytes, stream)


def mbpcg_k_cholesky(s, G, Z, status_dev, stream=None):
    return lib().mbpcg_k_cholesky(s, ptr(G), ptr(Z), ptr(status_dev), stream)


def mbpcg_k_pivot_reciprocals(n, d, inv, rsq, stream=None):
    return lib().mbpcg_k_pivot_reciprocals(n, ptr(d), ptr(inv), ptr(rsq), stream)


def mbpcg_server_create(slots, hbm_budget_bytes=0):
    srv = _P()
    st = lib().mbpcg_server_create(ctypes.byref(srv), slots, hbm_budget_bytes)
    if st != MBPCG_OK:
        raise MBPCGError(st, "mbpcg_server_create")
    return srv


def mbpcg_server_submit_csr(srv, n, nnz, row_ptr, col_idx, vals, b, s, precond, algo, tol, maxit, seed, x_out):
    """Queue one solve; the arrays (host) must stay alive and unchanged until the ticket is waited for."""
    t = _I64()
    st = lib().mbpcg_server_submit_csr(srv, n, nnz, ptr(row_ptr), ptr(col_idx), ptr(vals), ptr(b), s, precond, algo,
                                       tol, maxit, seed, ptr(x_out), ctypes.byref(t))
    if st != MBPCG_OK:
        raise MBPCGError(st, "mbpcg_server_submit_csr")
    return int(t.value)


def mbpcg_server_wait(srv, ticket):
    """(status, Info, queue_seconds, run_seconds) of a finished request; blocks until it ends."""
    info = Info()
    q = _D()
    r = _D()
    st = lib().mbpcg_server_wait(srv, ticket, ctypes.byref(info), ctypes.byref(q), ctypes.byref(r))
    return st, info, q.value, r.value


def mbpcg_server_get_stats(srv) -> dict:
    out = ServerStats()
    st = lib().mbpcg_server_get_stats(srv, ctypes.byref(out))
    if st != MBPCG_OK:
        raise MBPCGError(st, "mbpcg_server_get_stats")
    return out.as_dict()


def mbpcg_server_destroy(srv):
    lib().mbpcg_server_destroy(srv)


def mbpcg_set_residual_mode(h, mode):
    return lib().mbpcg_set_residual_mode(h, mode)


def mbpcg_get_spmm_tuning(h):
    """(variant, ctas_per_sm, [eleven measured microseconds]) of a mixed-precision handle's FP32 A P
    (variant 4 or 8: the gather kernel; 0: the tiled kernel; 1, 2: the wide-CTA kernel with 1024 or
    512 threads; 0 us: not timed)."""
    u, c = _I32(), _I32()
    t = (ctypes.c_float * 11)()
    st = lib().mbpcg_get_spmm_tuning(h, ctypes.byref(u), ctypes.byref(c), t)
    if st != MBPCG_OK:
        raise MBPCGError(st, "mbpcg_get_spmm_tuning")
    return int(u.value), int(c.value), [float(x) for x in t]


def mbpcg_set_spmm_shape(h, unroll, ctas_per_sm):
    return lib().mbpcg_set_spmm_shape(h, unroll, ctas_per_sm)


def mbpcg_apply_dev(h, fp32, X, Y):
    return lib().mbpcg_apply_dev(h, fp32, ptr(X), ptr(Y))


def mbpcg_batch_create(handles, stream=None):
    arr = (_P * len(handles))(*handles)
    b = _P()
    st = lib().mbpcg_batch_create(ctypes.byref(b), arr, len(handles), stream)
    if st != MBPCG_OK:
        raise MBPCGError(st, "mbpcg_batch_create")
    return b


def mbpcg_batch_solve_dev(batch, bs, Us, tol, maxit, xs):
    """bs, xs: lists of device tensors; Us: None or a list of device tensors / None (column-major)."""
    k = len(bs)
    pb = (_P * k)(*[ptr(t) for t in bs])
    px = (_P * k)(*[ptr(t) for t in xs])
    pu = None if Us is None else (_P * k)(*[ptr(t) for t in Us])
    infos = (Info * k)()
    st = lib().mbpcg_batch_solve_dev(batch, pb, pu, tol, maxit, px, infos)
    return st, list(infos)


def mbpcg_batch_destroy(batch):
    lib().mbpcg_batch_destroy(batch)


def mbpcg_get_product_kernel(h, fp32=0):
    """(kernel, [gather_us, tiled_us]) of a handle's product (MBPCG_PRODUCT_* codes)."""
    k = _I32()
    t = (ctypes.c_float * 2)()
    st = lib().mbpcg_get_product_kernel(h, fp32, ctypes.byref(k), t)
    if st != MBPCG_OK:
        raise MBPCGError(st, "mbpcg_get_product_kernel")
    return int(k.value), [float(x) for x in t]


def mbpcg_set_product_kernel(h, kernel):
    return lib().mbpcg_set_product_kernel(h, kernel)


def mbpcg_set_product_rounding(h, mode):
    return lib().mbpcg_set_product_rounding(h, mode)
