"""The mixed-precision inner solve (MBPCG_MIXED_FP32), CSR and dense, against the FP64 oracle.

Kernel level: the FP32 product A P is within FP32 rounding of the oracle's product of the same
FP32 data, |AP - AP_o| <= 1e-6 |A||P| (nnz_row <= 8 terms, unit roundoff 2^-24); the Gram P^T (A P)
is accumulated with compensated dot products and must agree with the exact Gram of the same FP32
P and AP to 1e-12 of |P|^T |AP| -- an FP32-accumulated Gram would miss this by about 1e6.

Solve level: the FP64 true residual reaches the requested 1e-10 through the FP64 refinement loop,
the error against the FP64 oracle's solution is bounded by 2 kappa tol (two solutions with
relative residual tol differ by at most that much), and the result is bit-repeatable."""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_07327_gb300 as mb
    mb.lib()
    return mb


def random_csr(n, seed, max_per_row=7, empty_every=5):
    cnt = (wl.uniform01(seed, 5000, n) * (max_per_row + 1)).astype(np.int64)
    cnt[::empty_every] = 0
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(cnt, out=rp[1:])
    nnz = int(rp[-1])
    cols = (wl.uniform01(seed, 5001, max(nnz, 1))[:nnz] * n).astype(np.int64)
    vals = wl.uniform_pm1(seed, 5002, max(nnz, 1))[:nnz]
    return wl.CSR(n, rp.astype(np.int32), cols.astype(np.int32), vals)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 8, 13, 16, 32])
@pytest.mark.parametrize("n", [1, 33, 1000, 4099])
def test_spmm_gram_f32_matches_oracle(mb, orc, n, s):
    A = random_csr(n, n + 3 * s)
    kp = int(mb.mbpcg_k_padded_width(s))
    P = np.zeros((n, kp), np.float32)
    P[:, :s] = wl.initial_block(n, s, 9).astype(np.float32)
    v32 = A.val.astype(np.float32)
    A32 = wl.CSR(n, A.row_ptr, A.col_idx, v32.astype(np.float64))  # the FP32 values, exactly, in FP64
    dev = torch.device("cuda")
    rp = torch.as_tensor(A.row_ptr, device=dev)
    ci = torch.as_tensor(A.col_idx if A.nnz else np.zeros(1, np.int32), device=dev)
    av = torch.as_tensor(v32 if A.nnz else np.zeros(1, np.float32), device=dev)
    Pd = torch.as_tensor(P, device=dev)
    AP = torch.full_like(Pd, float("nan"))
    G = torch.empty((s, s), dtype=torch.float64, device=dev)
    nbytes = mb.mbpcg_k_scratch_bytes(n, s)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    assert mb.mbpcg_k_spmm_gram_f32(n, rp, ci, av, s, Pd, AP, G, scratch, nbytes, None) == 0, mb.last_error()
    torch.cuda.synchronize()
    got = AP.cpu().numpy()
    ref = orc.matmat(A32, P.astype(np.float64))
    scale = np.abs(A32.to_scipy()) @ np.abs(P.astype(np.float64))
    assert np.all(np.abs(got - ref) <= 1e-6 * scale + 1e-30)
    assert np.all(got[:, s:] == 0.0)
    Pg, APg = P[:, :s].astype(np.float64), got[:, :s].astype(np.float64)
    exact = Pg.T @ APg  # products of FP32 numbers are exact in FP64
    bound = np.abs(Pg).T @ np.abs(APg)
    Gh = G.cpu().numpy().T
    Gu = np.triu(exact) + np.triu(exact, 1).T
    assert np.all(np.abs(Gh - Gu) <= 1e-12 * (np.triu(bound) + np.triu(bound, 1).T) + 1e-300)


@pytest.mark.parametrize("s", [1, 2, 3, 8, 13, 16, 32])
@pytest.mark.parametrize("n", [1, 33, 300, 1031, 4099])
def test_dense_f32_matches_oracle(mb, orc, n, s):
    """The FP32 dense product of the mixed inner solve on a dense A against the oracle's product of
    the same FP32 values: FP32 accumulation of n terms is within n 2^-24 |A||P| of the exact sum
    (any order). The tiles hold A rounded to FP32 and zeros past n (n = 4099: a ragged row tile
    and a ragged last chunk). The K split of a row tile over a cluster is summed in rank order:
    two calls give identical bits."""
    D = wl.dense_spd(n, 11, 0.0, 4.0)
    kp = int(mb.mbpcg_k_padded_width(s))
    P = np.zeros((n, kp), np.float32)
    P[:, :s] = wl.initial_block(n, s, 4).astype(np.float32)
    dev = torch.device("cuda")
    Ad = torch.as_tensor(np.asfortranarray(D.a).ravel(order="F"), device=dev)
    nb = mb.mbpcg_k_dense_f32_bytes(n)
    tiles = torch.full((nb // 4,), float("nan"), dtype=torch.float32, device=dev)
    assert mb.mbpcg_k_dense_f32_prepare(n, Ad, tiles, nb, None) == 0, mb.last_error()
    Pd = torch.as_tensor(P, device=dev)
    AP = torch.full_like(Pd, float("nan"))
    AP2 = torch.full_like(Pd, float("nan"))
    assert mb.mbpcg_k_dense_f32(n, tiles, s, Pd, AP, None) == 0, mb.last_error()
    assert mb.mbpcg_k_dense_f32(n, tiles, s, Pd, AP2, None) == 0, mb.last_error()
    torch.cuda.synchronize()
    got = AP.cpu().numpy()
    A32 = np.asarray(D.a, dtype=np.float64).astype(np.float32).astype(np.float64)  # the FP32 values, exactly
    ref = orc.matmat(wl.Dense(n, np.asfortranarray(A32)), P.astype(np.float64))
    scale = np.abs(A32) @ np.abs(P.astype(np.float64))
    assert np.all(np.abs(got - ref) <= (n + 2) * 2.0 ** -24 * scale + 1e-30)
    assert np.all(got[:, s:] == 0.0)
    assert np.array_equal(got, AP2.cpu().numpy())


def test_dense_f32_rejects_bad_arguments(mb):
    dev = torch.device("cuda")
    A = torch.zeros(64, dtype=torch.float64, device=dev)
    nb = mb.mbpcg_k_dense_f32_bytes(8)
    assert nb == 256 * 32 * 4 and mb.mbpcg_k_dense_f32_bytes(0) == 0
    tiles = torch.zeros(nb // 4, dtype=torch.float32, device=dev)
    P = torch.zeros((8, 4), dtype=torch.float32, device=dev)
    Q = torch.zeros_like(P)
    assert mb.mbpcg_k_dense_f32_prepare(8, A, tiles, nb - 4, None) == mb._native.MBPCG_ERR_INVALID  # too small
    assert mb.mbpcg_k_dense_f32_prepare(0, A, tiles, nb, None) == mb._native.MBPCG_ERR_INVALID
    assert mb.mbpcg_k_dense_f32(8, tiles, 33, P, Q, None) == mb._native.MBPCG_ERR_INVALID  # s > 32
    assert mb.mbpcg_k_dense_f32(8, None, 4, P, Q, None) == mb._native.MBPCG_ERR_INVALID


MIXED_CASES = [
    # (name, matrix factory, s, precond) -- shapes of the mixed-precision configuration (27-point
    # stencil, s = 16) and of the other sparse families, at sizes the oracle finishes quickly
    ("stencil27_16_s16", lambda: wl.stencil27(16, 0), 16, 0),
    ("stencil27_12_s8", lambda: wl.stencil27(12, 1), 8, 0),
    ("poisson64_s4", lambda: wl.poisson2d(64), 4, 0),
    ("diffusion16_s4_jacobi", lambda: wl.diffusion3d(16, 2), 4, 1),
    ("poisson3d_20_s1", lambda: wl.poisson3d(20), 1, 0),
    ("diffusion12_s32_jacobi", lambda: wl.diffusion3d(12, 3), 32, 1),
    # dense SPD A = Q diag(10^U[0,hi]) Q^T (the dense configuration's family), FP32 copy of A
    ("dense300_k1e6_s8", lambda: wl.dense_spd(300, 0, 0.0, 6.0), 8, 0),
    ("dense257_k1e4_s32_jacobi", lambda: wl.dense_spd(257, 1, 0.0, 4.0), 32, 1),
    ("dense1031_k1e4_s16", lambda: wl.dense_spd(1031, 2, 0.0, 4.0), 16, 0),
    ("dense64_k1e3_s1", lambda: wl.dense_spd(64, 3, 0.0, 3.0), 1, 0),
]


def kappa(A, precond):
    M = np.asarray(A.a, dtype=np.float64) if not hasattr(A, "row_ptr") else A.to_scipy().toarray()
    if precond:
        d = 1.0 / np.sqrt(np.diag(M))
        M = d[:, None] * M * d[None, :]
    ev = np.linalg.eigvalsh(M)
    return ev[-1] / ev[0]


@pytest.mark.parametrize("name,factory,s,precond", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_mixed_solve_against_fp64_oracle(mb, orc, name, factory, s, precond):
    A = factory()
    n = A.n
    b = wl.rhs(n, 0)
    U = wl.initial_block(n, s, 1)
    tol = 1e-10
    sv = mb.Solver(A, s=s, precond=precond, precision=mb.MBPCG_MIXED_FP32)
    try:
        x, info = sv.solve(b, U, tol=tol, maxit=200000)
        x2, info2 = sv.solve(b, U, tol=tol, maxit=200000)
    finally:
        sv.close()
    assert info["status"] == 0, info
    r = b - (np.asarray(A.a) @ x if not hasattr(A, "row_ptr") else A.to_scipy() @ x)
    relres = np.linalg.norm(r) / np.linalg.norm(b)
    assert relres <= tol and info["relres_true"] <= tol
    assert info["restarts"] >= 1  # FP32 inner solves need the FP64 refinement for 1e-10
    assert np.array_equal(x, x2) and info["iterations"] == info2["iterations"]
    xo, _, io = orc.mbpcg(A, b, U, precond=precond, tol=tol)
    assert io["status"] == 0
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    assert err <= 2 * kappa(A, precond) * tol, (err, info, io)


def test_mixed_precision_is_refused_where_it_does_not_apply(mb):
    with pytest.raises(mb.MBPCGError):
        mb.Solver(wl.poisson2d(8), s=4, algo=mb.MBPCG_ALGO_CG, precision=mb.MBPCG_MIXED_FP32)
    sv = mb.Solver(wl.poisson2d(8), s=4, precision=mb.MBPCG_MIXED_FP32)
    try:
        _, st = sv.run_iterations(wl.rhs(64, 0), wl.initial_block(64, 4, 1), 2)
        assert st == mb._native.MBPCG_ERR_INVALID
    finally:
        sv.close()


def test_spmm_autotuner_picks_the_fastest_shape_and_never_changes_results(mb):
    A = wl.stencil27(24, 5)
    n, s = A.n, 16
    b = wl.rhs(n, 0)
    U = wl.initial_block(n, s, 1)
    sv = mb.Solver(A, s=s, precision=mb.MBPCG_MIXED_FP32)
    try:
        unroll, cps, times = sv.spmm_tuning()
        order = [(4, 4), (4, 8), (4, 16), (8, 4), (8, 8), (8, 16), (0, 2), (1, 1), (1, 2), (2, 2), (2, 4)]
        assert (unroll, cps) in order and len(times) == 11
        assert times[6] == 0.0  # 13,824 rows: no tiling plan
        timed = [t for t in times if t > 0.0]
        assert len(timed) == 10 and times[order.index((unroll, cps))] == min(timed)
        x0, i0 = sv.solve(b, U, tol=1e-10, maxit=100000)
        for shape in ((4, 4), (8, 16), (1, 2), (2, 2)):
            sv.set_spmm_shape(*shape)
            x, info = sv.solve(b, U, tol=1e-10, maxit=100000)
            assert np.array_equal(x, x0) and info["iterations"] == i0["iterations"]
        for bad in ((3, 8), (0, 2)):  # an unknown shape; the tiled kernel without a plan
            with pytest.raises(mb.MBPCGError):
                sv.set_spmm_shape(*bad)
    finally:
        sv.close()
    for other in (mb.Solver(A, s=s), mb.Solver(wl.dense_spd(64, 0), s=4, precision=mb.MBPCG_MIXED_FP32)):
        try:
            with pytest.raises(mb.MBPCGError):  # FP64 handles and the dense FP32 product have no shapes
                other.spmm_tuning()
        finally:
            other.close()
