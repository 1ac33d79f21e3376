"""The tiled CSR product (the rows of P a tile of A reads staged once in shared memory, nonzeros
addressing them by 16-bit local indices) and the wide-CTA FP32 product against the oracle's product
and the gather kernel.

All kernels sum each row in CSR order, so their A P agree bit for bit; against the oracle's FP64
product the difference is within the rounding of a row sum, |AP - AP_o| <= 2 nnz_row u |A||P| with
u = 2^-53 (2^-24 for the FP32 product, against the oracle's product of the same FP32 data).
Matrices: 3D diffusion 41^3 (n = 68,921, odd: the last tile is ragged), a random banded pattern
(n = 70,001, columns within +-200 of the diagonal), the 27-point stencil 41^3 (the FP32 product of
the mixed inner solve); an arrow matrix whose dense first row fits no tile window and a random
pattern without locality keep the gather kernel."""
import numpy as np
import pytest

import oracle
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


def spd_from_pairs(n, r, c, v):
    """Symmetric, diagonally dominant CSR from off-diagonal entries (r, c, v) (duplicates summed)."""
    keep = r != c
    r, c, v = r[keep], c[keep], v[keep]
    rows, cols, vals = np.concatenate([r, c]), np.concatenate([c, r]), np.concatenate([v, v])
    key, inv = np.unique(rows * n + cols, return_inverse=True)
    acc = np.zeros(len(key))
    np.add.at(acc, inv, vals)
    rows, cols = key // n, key % n
    diag = np.ones(n)
    np.add.at(diag, rows, np.abs(acc))
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([acc, diag])
    order = np.lexsort((cols, rows))
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return wl.CSR(n, rp.astype(np.int32), cols[order].astype(np.int32), vals[order])


def banded_spd(n, seed, band=200, per_row=4):
    """About 8 off-diagonal entries per row at random columns within +-band of the diagonal: the
    window of a tile is its rows plus 2 band, partly filled (a pattern that is not a stencil)."""
    cnt = per_row * n
    r = (wl.uniform01(seed, 3100, cnt) * n).astype(np.int64)
    c = np.clip(r + np.rint((2.0 * wl.uniform01(seed, 3101, cnt) - 1.0) * band).astype(np.int64), 0, n - 1)
    return spd_from_pairs(n, r, c, -wl.uniform01(seed, 3102, cnt))


def scattered_spd(n, seed):
    """About 8 off-diagonal entries per row at uniformly random columns (no locality: about one run
    of staged rows per nonzero, beyond the plan's budget of runs)."""
    cnt = 4 * n
    r = (wl.uniform01(seed, 3100, cnt) * n).astype(np.int64)
    c = (wl.uniform01(seed, 3101, cnt) * n).astype(np.int64)
    return spd_from_pairs(n, r, c, -wl.uniform01(seed, 3102, cnt))


def arrow_spd(n):
    """Row and column 0 full, plus the diagonal: row 0 alone holds n columns, more than any window."""
    rows = np.concatenate([np.zeros(n - 1, np.int64), np.arange(1, n), np.arange(n)])
    cols = np.concatenate([np.arange(1, n), np.zeros(n - 1, np.int64), np.arange(n)])
    off = -1e-3 * np.ones(n - 1)
    diag = 2.0 + np.zeros(n)
    diag[0] = 2.0 + 1e-3 * (n - 1)
    vals = np.concatenate([off, off, diag])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return wl.CSR(n, rp.astype(np.int32), cols.astype(np.int32), vals)


MATRICES = {
    "diffusion41": lambda: wl.diffusion3d(41, 0),
    "banded70001": lambda: banded_spd(70001, 2),
}
_cache = {}


def matrix(name):
    if name not in _cache:
        _cache[name] = MATRICES[name]()
    return _cache[name]


def row_bound(A, X, u):
    """2 nnz_row u (|A| |X|) row by row: the rounding of a row sum of nnz_row products."""
    absA = A.to_scipy().copy()
    absA.data = np.abs(absA.data)
    nrow = np.diff(A.row_ptr).astype(np.float64)[:, None]
    return 2.0 * nrow * u * (absA @ np.abs(X)) + 1e-300


@pytest.mark.parametrize("name", sorted(MATRICES))
@pytest.mark.parametrize("s,algo", [(1, 1), (1, 0), (4, 0), (16, 0)])
def test_fp64_tiled_product_matches_the_oracle_and_the_gather_kernel(mb, name, s, algo):
    A = matrix(name)
    sv = mb.Solver(A, s=s, algo=algo)
    try:
        kernel, times = sv.product_kernel()
        assert kernel == mb.MBPCG_PRODUCT_CSR_GATHER  # the loop's FP64 product never depends on a timing
        assert times[0] > 0.0 and times[1] == 0.0  # the plan is built when the tiled kernel is imposed
        kp = 1 if algo == 1 else mb.mbpcg_k_padded_width(s)
        X = torch.as_tensor(wl.initial_block(A.n, kp, 3)).reshape(A.n, kp).contiguous().cuda()
        sv.set_product_kernel(mb.MBPCG_PRODUCT_CSR_TILED)
        kernel, times = sv.product_kernel()
        assert kernel == mb.MBPCG_PRODUCT_CSR_TILED and times[1] > 0.0, "a plan is expected for this matrix"
        Yt = sv.apply(X)
        sv.set_product_kernel(mb.MBPCG_PRODUCT_CSR_GATHER)
        Yg = sv.apply(X)
        assert torch.equal(Yt, Yg)
        Xh = X.cpu().numpy()
        Yo = oracle.matmat(A, Xh)
        err = np.abs(Yt.cpu().numpy() - Yo)
        assert np.all(err <= row_bound(A, Xh, 2.0 ** -53)), float(err.max())
    finally:
        sv.close()


def test_fp64_solve_with_the_tiled_product(mb):
    """Diffusion 41^3, Jacobi, s = 4, tol 1e-8: the solve through either kernel converges with the
    same iteration count up to the rounding of the Gram (a few iterations), the tiled solve is
    bit-repeatable, and both solutions have a true residual (recomputed here in FP64 on the host)
    at the requested level."""
    A = matrix("diffusion41")
    b = wl.rhs(A.n, 0)
    U = wl.initial_block(A.n, 4, 1)
    sv = mb.Solver(A, s=4, precond=mb.MBPCG_PRECOND_JACOBI)
    try:
        sv.set_product_kernel(mb.MBPCG_PRODUCT_CSR_TILED)
        xt, it = sv.solve(b, U, tol=1e-8, maxit=100000)
        xt2, it2 = sv.solve(b, U, tol=1e-8, maxit=100000)
        assert np.array_equal(xt, xt2) and it["iterations"] == it2["iterations"]
        sv.set_product_kernel(mb.MBPCG_PRODUCT_CSR_GATHER)
        xg, ig = sv.solve(b, U, tol=1e-8, maxit=100000)
    finally:
        sv.close()
    for info in (it, ig):
        assert info["status"] == 0 and info["relres_true"] <= 1e-8
    assert abs(it["iterations"] - ig["iterations"]) <= max(3, ig["iterations"] // 50)
    S = A.to_scipy()
    for x in (xt, xg):
        assert np.linalg.norm(b - S @ x) <= 1.1e-8 * np.linalg.norm(b)


def test_fp32_tiled_product_and_mixed_solve(mb):
    """27-point stencil 41^3, s = 16, mixed precision: the autotuner times the tiled kernel as a
    seventh shape; the tiled and the gather FP32 products are the same bits, within FP32 rounding of
    the oracle's product of the same FP32 data, and a solve through either gives the same bits."""
    A = wl.stencil27(41, 5)
    n, s = A.n, 16
    sv = mb.Solver(A, s=s, precision=mb.MBPCG_MIXED_FP32)
    try:
        unroll, cps, times = sv.spmm_tuning()
        assert len(times) == 11 and min(times) > 0.0
        order = [(4, 4), (4, 8), (4, 16), (8, 4), (8, 8), (8, 16), (0, 2), (1, 1), (1, 2), (2, 2), (2, 4)]
        assert times[order.index((unroll, cps))] == min(times)
        codes = {0: mb.MBPCG_PRODUCT_CSR_TILED, 1: mb.MBPCG_PRODUCT_CSR_WIDE, 2: mb.MBPCG_PRODUCT_CSR_WIDE}
        assert sv.product_kernel(fp32=True)[0] == codes.get(unroll, mb.MBPCG_PRODUCT_CSR_GATHER)
        assert sv.product_kernel() == (mb.MBPCG_PRODUCT_CSR_GATHER, [0.0, 0.0])  # FP64 of a mixed handle
        X = torch.as_tensor(wl.initial_block(n, s, 3)).reshape(n, s).to(torch.float32).contiguous().cuda()
        sv.set_spmm_shape(0, 2)
        Yt = sv.apply(X, fp32=True)
        sv.set_spmm_shape(1, 2)
        Ys = sv.apply(X, fp32=True)
        sv.set_spmm_shape(8, 8)
        Yg = sv.apply(X, fp32=True)
        assert torch.equal(Yt, Yg) and torch.equal(Ys, Yg)
        A32 = wl.CSR(n, A.row_ptr, A.col_idx, A.val.astype(np.float32).astype(np.float64))
        Xh = X.cpu().numpy().astype(np.float64)
        err = np.abs(Yt.cpu().numpy().astype(np.float64) - oracle.matmat(A32, Xh))
        assert np.all(err <= row_bound(A32, Xh, 2.0 ** -24)), float(err.max())
        b = wl.rhs(n, 0)
        U = wl.initial_block(n, s, 1)
        x0, i0 = sv.solve(b, U, tol=1e-10, maxit=100000)
        assert i0["status"] == 0
        for shape in ((0, 2), (1, 1), (2, 4)):
            sv.set_spmm_shape(*shape)
            x1, i1 = sv.solve(b, U, tol=1e-10, maxit=100000)
            assert np.array_equal(x0, x1) and i0["iterations"] == i1["iterations"]
    finally:
        sv.close()


@pytest.mark.parametrize("name", ["arrow", "scattered"])
def test_patterns_without_a_plan_keep_the_gather_kernel(mb, name):
    """The arrow matrix's first row fits no window; the scattered pattern needs more runs than the
    plan's budget. Both keep the gather kernel, whose product still matches the oracle."""
    A = arrow_spd(70000) if name == "arrow" else scattered_spd(70001, 2)
    sv = mb.Solver(A, s=4)
    try:
        kernel, times = sv.product_kernel()
        assert kernel == mb.MBPCG_PRODUCT_CSR_GATHER and times[1] == 0.0
        with pytest.raises(mb.MBPCGError):
            sv.set_product_kernel(mb.MBPCG_PRODUCT_CSR_TILED)
        kp = mb.mbpcg_k_padded_width(4)
        X = torch.as_tensor(wl.initial_block(A.n, kp, 3)).reshape(A.n, kp).contiguous().cuda()
        Y = sv.apply(X).cpu().numpy()
        Xh = X.cpu().numpy()
        assert np.all(np.abs(Y - oracle.matmat(A, Xh)) <= row_bound(A, Xh, 2.0 ** -53))
    finally:
        sv.close()


def test_small_systems_have_no_plan_and_dense_handles_one_product(mb):
    sv = mb.Solver(wl.poisson2d(64), s=4)
    try:
        kernel, times = sv.product_kernel()
        assert kernel == mb.MBPCG_PRODUCT_CSR_GATHER and times[0] > 0.0 and times[1] == 0.0
        with pytest.raises(mb.MBPCGError):
            sv.product_kernel(fp32=True)
    finally:
        sv.close()
    sv = mb.Solver(wl.dense_spd(256, 0), s=4)
    try:
        assert sv.product_kernel()[0] == mb.MBPCG_PRODUCT_DENSE
        with pytest.raises(mb.MBPCGError):
            sv.set_product_kernel(mb.MBPCG_PRODUCT_CSR_GATHER)
    finally:
        sv.close()


@pytest.mark.parametrize("form", ["fp64", "tc", "tc_once", "mixed"])
def test_dense_apply_matches_the_oracle(mb, form):
    """mbpcg_apply_dev on dense handles: the FP64 product (rounding of an FP64 row sum), the
    tensor-core product in both rounding modes (1e-14 |A||P|, the bound of the digit-split product)
    and the FP32 product of a mixed handle (FP32 rounding of the oracle's product of the same FP32 data); n = 1031 spans several
    128-row tiles and a ragged last one."""
    A = wl.dense_spd(1031, 3, 0.0, 4.0)
    n, s = A.n, 16
    prec = {"fp64": mb.MBPCG_FP64, "tc": mb.MBPCG_FP64_TC, "tc_once": mb.MBPCG_FP64_TC,
            "mixed": mb.MBPCG_MIXED_FP32}[form]
    sv = mb.Solver(A, s=s, precision=prec)
    try:
        if form == "tc_once":
            sv.set_product_rounding(mb.MBPCG_ROUND_ONCE)
        elif form != "tc":
            with pytest.raises(mb.MBPCGError):  # the rounding mode belongs to tensor-core handles
                sv.set_product_rounding(mb.MBPCG_ROUND_ONCE)
        kernel = sv.product_kernel(fp32=form == "mixed")[0]
        assert kernel == {"fp64": mb.MBPCG_PRODUCT_DENSE, "tc": mb.MBPCG_PRODUCT_DENSE_TC,
                          "tc_once": mb.MBPCG_PRODUCT_DENSE_TC, "mixed": mb.MBPCG_PRODUCT_DENSE_FP32}[form]
        X = torch.as_tensor(wl.initial_block(n, s, 4)).reshape(n, s).contiguous().cuda()
        absA = np.abs(np.asarray(A.a))
        if form == "mixed":
            Xf = X.to(torch.float32).contiguous()
            Y = sv.apply(Xf, fp32=True).cpu().numpy().astype(np.float64)
            A32 = wl.Dense(n, np.asfortranarray(np.asarray(A.a).astype(np.float32).astype(np.float64)))
            Xh = Xf.cpu().numpy().astype(np.float64)
            ref = oracle.matmat(A32, Xh)
            bound = 2.0 * n * 2.0 ** -24 * (absA @ np.abs(Xh)) + 1e-300
        else:
            Y = sv.apply(X).cpu().numpy()
            Xh = X.cpu().numpy()
            ref = oracle.matmat(A, Xh)
            u = 2.0 ** -53 if form == "fp64" else 1e-14 / (2.0 * n)
            bound = 2.0 * n * u * (absA @ np.abs(Xh)) + 1e-300
        err = np.abs(Y - ref)
        assert np.all(err <= bound), float((err / bound).max())
    finally:
        sv.close()


@pytest.mark.parametrize("s", [1, 4])
def test_full_size_diffusion_product_matches_the_oracle(mb, s):
    """The product the bench's SpMM roofline times (diffusion 128^3, Jacobi-scaled, the handle's own
    kernel through mbpcg_apply_dev) against the oracle's product of the same scaled matrix, every
    entry, at the rounding of a row sum."""
    A = wl.diffusion3d(128, 0)
    n = A.n
    sv = mb.Solver(A, s=s, precond=mb.MBPCG_PRECOND_JACOBI)
    try:
        kp = mb.mbpcg_k_padded_width(s)
        X = torch.as_tensor(wl.initial_block(n, kp, 5)).reshape(n, kp).contiguous().cuda()
        Y = sv.apply(X).cpu().numpy()
    finally:
        sv.close()
    d = 1.0 / np.sqrt(A.diagonal())
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    As = wl.CSR(n, A.row_ptr, A.col_idx, A.val * d[rows] * d[A.col_idx])  # D^-1/2 A D^-1/2
    Xh = X.cpu().numpy()
    err = np.abs(Y - oracle.matmat(As, Xh))
    # the GPU scales the values itself (one rounding per value): bound the product of either scaling
    assert np.all(err <= row_bound(As, Xh, 2.0 ** -52) + 4 * 2.0 ** -53 * (np.abs(As.to_scipy()) @ np.abs(Xh))), \
        float(err.max())
