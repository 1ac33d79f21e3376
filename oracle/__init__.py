"""MBPCG oracle -- TEST INFRASTRUCTURE ONLY.

A plain FP64 CPU implementation of the paper's Multi-Basis Parallel CG (Algorithm 1) and of the
Chronopoulos-Gear CG baseline, written in C (``mbpcg_oracle.c``) and loaded here with ctypes.
Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package. It shares no code with the CUDA library and never calls it.

Readings of the paper that the oracle fixes (where the paper is silent or garbled) are listed in
the header of ``mbpcg_oracle.c``'s functions and in the design notes; parity of every function is
pinned by ``tests/test_oracle_*.py`` against closed forms, LAPACK/scipy and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mbpcg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_OMP_PATH = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

STATUS = {0: "ok", 1: "invalid", 4: "not_spd", 5: "not_converged", 6: "breakdown"}


class OrcInfo(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32),
        ("restarts", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("best_col", ctypes.c_int32),
        ("ls_fallback", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("relres_recurrence", ctypes.c_double),
        ("relres_ls", ctypes.c_double),
        ("relres_true", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int32)
ITER_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                           _DP, _DP, _DP, _DP, _DP, _DP)


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc: oracle/_build/liboracle.so (plain -O2, single thread: the parity
    oracle), or with omp=True oracle/_build/liboracle_omp.so (-O3 -fopenmp: the same source with its
    independent loops shared among the host cores, for the timed CPU baseline; same results bit for
    bit)."""
    path = _OMP_PATH if omp else _LIB_PATH
    os.makedirs(os.path.dirname(path), exist_ok=True)
    if force or not os.path.exists(path) or os.path.getmtime(path) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mbpcg_oracle.h"))):
        tmp = path + f".tmp{os.getpid()}"
        flags = ["-O3", "-fopenmp"] if omp else ["-O2"]
        subprocess.check_call(["gcc", *flags, "-std=c99", "-Wall", "-Wextra", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def lib(omp: bool = False):
    with _lock:
        if omp not in _libs:
            path = build(omp=omp)
            L = ctypes.CDLL(path)
            L.orc_matmat.argtypes = [ctypes.c_int32, _IP, _IP, _DP, _DP, ctypes.c_int32, _DP, _DP]
            L.orc_mbpcg.argtypes = [ctypes.c_int32, _IP, _IP, _DP, _DP, _DP, _DP, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                    _DP, _DP, ctypes.POINTER(OrcInfo), ITER_CB, ctypes.c_void_p]
            L.orc_cg_cgear.argtypes = [ctypes.c_int32, _IP, _IP, _DP, _DP, _DP, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _DP,
                                       ctypes.POINTER(OrcInfo)]
            L.orc_mbpcg_state.argtypes = [ctypes.c_int32, _IP, _IP, _DP, _DP, _DP, _DP, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, _DP, _DP, _DP, _DP, _DP, _DP]
            for f in (L.orc_matmat, L.orc_mbpcg, L.orc_cg_cgear, L.orc_mbpcg_state):
                f.restype = ctypes.c_int
            _libs[omp] = L
    return _libs[omp]


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _ip(a):
    return None if a is None else a.ctypes.data_as(_IP)


def _mat_args(A):
    """(n, row_ptr, col_idx, val, dense) for a workloads.CSR / workloads.Dense, keeping refs alive."""
    if hasattr(A, "row_ptr"):
        rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
        v = np.ascontiguousarray(A.val, dtype=np.float64)
        return (A.n, rp, ci, v, None), (rp, ci, v)
    a = np.asfortranarray(A.a, dtype=np.float64)
    return (A.n, None, None, None, a), (a,)


def matmat(A, X: np.ndarray) -> np.ndarray:
    """Y = A X with X n x k (any layout); returns Y n x k (Fortran order)."""
    (n, rp, ci, v, dn), keep = _mat_args(A)
    X = np.asfortranarray(X.reshape(n, -1), dtype=np.float64)
    Y = np.zeros_like(X, order="F")
    st = lib().orc_matmat(n, _ip(rp), _ip(ci), _dp(v), _dp(dn), X.shape[1], _dp(X), _dp(Y))
    if st != 0:
        raise ValueError(f"orc_matmat: status {st}")
    return Y


def mbpcg(A, b, U, precond: int = 0, tol: float = 1e-8, maxit: int = 100000, max_restarts: int = 3,
          callback=None, omp: bool = False):
    """Algorithm 1 solve. Returns (x, c, info_dict). callback(iter, exiting, restart, state_dict)
    receives copies of X0, Xt, R, W, P (n x k) and Sigma (k x k) of the scaled system."""
    (n, rp, ci, v, dn), keep = _mat_args(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    U = np.asfortranarray(U, dtype=np.float64)
    k = U.shape[1]
    x = np.zeros(n)
    c = np.zeros(k)
    info = OrcInfo()
    if callback is not None:
        def _cb(user, it, exiting, restart, X0, Xt, R, W, P, S):
            def blk(p):
                return np.ctypeslib.as_array(p, shape=(k * n,)).reshape((n, k), order="F").copy()
            state = dict(X0=blk(X0), Xt=blk(Xt), R=blk(R), W=blk(W), P=blk(P),
                         Sigma=np.ctypeslib.as_array(S, shape=(k * k,)).reshape((k, k), order="F").copy())
            callback(it, exiting, restart, state)
        cb = ITER_CB(_cb)
    else:
        cb = ITER_CB()
    lib(omp).orc_mbpcg(n, _ip(rp), _ip(ci), _dp(v), _dp(dn), _dp(b), _dp(U), k, precond, tol, maxit,
                    max_restarts, _dp(x), _dp(c), ctypes.byref(info), cb, None)
    return x, c, info.as_dict()


def cg_cgear(A, b, precond: int = 0, tol: float = 1e-8, maxit: int = 100000, max_restarts: int = 3,
             omp: bool = False):
    """Chronopoulos-Gear CG from x0 = 0. Returns (x, info_dict)."""
    (n, rp, ci, v, dn), keep = _mat_args(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n)
    info = OrcInfo()
    lib(omp).orc_cg_cgear(n, _ip(rp), _ip(ci), _dp(v), _dp(dn), _dp(b), precond, tol, maxit, max_restarts,
                       _dp(x), ctypes.byref(info))
    return x, info.as_dict()


def mbpcg_state(A, b, U, iters: int, precond: int = 0, omp: bool = False):
    """Raw state after exactly `iters` iterations: dict(X0, Xt, R, W, P, Sigma) and the status."""
    (n, rp, ci, v, dn), keep = _mat_args(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    U = np.asfortranarray(U, dtype=np.float64)
    k = U.shape[1]
    out = {name: np.zeros((n, k), order="F") for name in ("X0", "Xt", "R", "W", "P")}
    out["Sigma"] = np.zeros((k, k), order="F")
    st = lib(omp).orc_mbpcg_state(n, _ip(rp), _ip(ci), _dp(v), _dp(dn), _dp(b), _dp(U), k, precond, iters,
                               _dp(out["X0"]), _dp(out["Xt"]), _dp(out["R"]), _dp(out["W"]), _dp(out["P"]),
                               _dp(out["Sigma"]))
    return out, st
