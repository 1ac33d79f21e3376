"""The C-ABI library builds and exports every function declared in include/*.h; the oracle and the
library share no code. No compute call is made (no GPU needed)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(mbpcg_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2608_07327_gb300 import build
    return build.build()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("mbpcg_create_csr", "mbpcg_create_dense", "mbpcg_solve", "mbpcg_solve_dev", "mbpcg_destroy",
                     "mbpcg_status_string", "mbpcg_k_spmm_gram"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(mbpcg_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_answers_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    L.mbpcg_status_string.restype = ctypes.c_char_p
    assert L.mbpcg_status_string(0) == b"ok"
    assert L.mbpcg_status_string(6) == b"breakdown"
    L.mbpcg_k_padded_width.restype = ctypes.c_int32
    assert [L.mbpcg_k_padded_width(s) for s in (1, 2, 3, 5, 9, 17, 32, 33)] == [1, 2, 4, 8, 16, 32, 32, 0]


def test_component_entries_reject_bad_arguments_without_gpu(libpath):
    """Argument checks of the component entries come before any device call, so they answer on a
    machine without a GPU: MBPCG_ERR_INVALID (1) for bad sizes, widths, NULL or misaligned pointers,
    and sizes of the FP32 copy of a dense A that follow its tiling (256 x 32 FP32 tiles)."""
    L = ctypes.CDLL(libpath)
    P, I32, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
    L.mbpcg_k_dense_f32_bytes.restype = SZ
    L.mbpcg_k_dense_f32_bytes.argtypes = [I32]
    tile = 256 * 32 * 4
    assert L.mbpcg_k_dense_f32_bytes(0) == 0
    assert L.mbpcg_k_dense_f32_bytes(1) == tile
    assert L.mbpcg_k_dense_f32_bytes(256) == 8 * tile
    assert L.mbpcg_k_dense_f32_bytes(257) == 2 * 9 * tile
    assert L.mbpcg_k_dense_f32_bytes(4096) == 4096 * 4096 * 4
    buf = ctypes.create_string_buffer(64)
    aligned = ctypes.addressof(buf) // 16 * 16 + 16  # inside buf, 16-byte aligned
    L.mbpcg_k_rowprod_tc.restype = ctypes.c_int
    L.mbpcg_k_rowprod_tc.argtypes = [I32, I32, P, P, I32, P, P]
    assert L.mbpcg_k_rowprod_tc(0, 32, aligned, aligned, 0, aligned, None) == 1  # n < 1
    assert L.mbpcg_k_rowprod_tc(4, 8, aligned, aligned, 0, aligned, None) == 1   # width not 16 or 32
    assert L.mbpcg_k_rowprod_tc(4, 32, aligned, aligned, 2, aligned, None) == 1  # transM not 0 or 1
    assert L.mbpcg_k_rowprod_tc(4, 32, None, aligned, 0, aligned, None) == 1     # NULL X
    assert L.mbpcg_k_rowprod_tc(4, 32, aligned + 8, aligned, 0, aligned, None) == 1  # X not 16-byte aligned
    L.mbpcg_k_dense_f32_prepare.restype = ctypes.c_int
    L.mbpcg_k_dense_f32_prepare.argtypes = [I32, P, P, SZ, P]
    assert L.mbpcg_k_dense_f32_prepare(8, aligned, aligned, tile - 1, None) == 1  # tiles too small
    assert L.mbpcg_k_dense_f32_prepare(8, None, aligned, tile, None) == 1         # NULL A
    assert L.mbpcg_k_dense_f32_prepare(8, aligned, aligned + 8, tile, None) == 1  # tiles misaligned
    L.mbpcg_k_dense_f32.restype = ctypes.c_int
    L.mbpcg_k_dense_f32.argtypes = [I32, P, I32, P, P, P]
    assert L.mbpcg_k_dense_f32(8, aligned, 33, aligned, aligned, None) == 1  # s > 32
    assert L.mbpcg_k_dense_f32(8, None, 4, aligned, aligned, None) == 1      # NULL tiles
    L.mbpcg_k_dense_tc_mma.restype = ctypes.c_int
    L.mbpcg_k_dense_tc_mma.argtypes = [I32, I32, P, SZ, P]
    assert L.mbpcg_k_dense_tc_mma(0, 32, aligned, 1 << 30, None) == 1  # n < 1
    assert L.mbpcg_k_dense_tc_mma(64, 0, aligned, 1 << 30, None) == 1  # s < 1
    L.mbpcg_k_pivot_reciprocals.restype = ctypes.c_int
    L.mbpcg_k_pivot_reciprocals.argtypes = [I32, P, P, P, P]
    assert L.mbpcg_k_pivot_reciprocals(0, aligned, aligned, aligned, None) == 1  # n < 1
    assert L.mbpcg_k_pivot_reciprocals(4, aligned, None, aligned, None) == 1     # NULL inv


def test_binding_names_match_the_abi():
    import paper_2608_07327_gb300 as pkg
    for name in declared_functions():
        if name in ("mbpcg_status_string", "mbpcg_last_error"):
            continue
        assert hasattr(pkg._native, name), name


def test_oracle_and_library_share_no_code():
    for f in glob.glob(os.path.join(ROOT, "paper_2608_07327_gb300", "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".inc")):
            txt = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
            assert "mbpcg_oracle" not in txt, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if os.path.isfile(f):
            txt = open(f).read()
            assert "paper_2608_07327_gb300" not in txt and "csrc" not in txt, f


def test_no_cpu_fallback_without_a_device(libpath):
    """Without a CUDA device the library refuses to solve instead of computing on the host:
    mbpcg_create_csr with host arrays returns MBPCG_ERR_CUDA (3) and no handle, and the Python
    Solver raises before any arithmetic."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import numpy as np

    import workloads as wl
    A = wl.poisson2d(4)
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(A.val, dtype=np.float64)
    L = ctypes.CDLL(libpath)
    P, I32 = ctypes.c_void_p, ctypes.c_int32
    L.mbpcg_create_csr.restype = ctypes.c_int
    L.mbpcg_create_csr.argtypes = [ctypes.POINTER(P), I32, ctypes.c_int64, P, P, P, I32, I32, I32, I32,
                                   ctypes.c_uint64, I32, P, ctypes.c_size_t, P]
    h = P(None)
    st = L.mbpcg_create_csr(ctypes.byref(h), A.n, int(rp[-1]), rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 2, 0, 0,
                            0, 1, 0, None, 0, None)
    assert st == 3 and not h.value
    import paper_2608_07327_gb300 as mb
    with pytest.raises(Exception):
        mb.Solver(A, s=2)
