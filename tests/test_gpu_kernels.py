"""Component kernels through the C ABI (include/mbpcg_kernels.h) against the oracle / numpy on the
same seeded inputs: the A P product fused with P^T (A P), for CSR (empty rows, a single row, ragged
tails, every padded width) and dense A, and the k x k Cholesky with its breakdown test.

Tolerances: the product sums each row in CSR order with FMAs (the oracle rounds twice per term),
so |AP - AP_oracle| <= 2 nnz_row eps sum|a||p|, bounded here by 1e-13 * max|AP|-scale; the Gram
sums n terms in a different (tree) order: |dG| <= n eps ||P|| ||AP||, bounded by 1e-12 relative.
"""
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
    """Random (not necessarily symmetric) CSR with some empty rows and duplicate-free columns."""
    cnt = (wl.uniform01(seed, 5000, n) * (max_per_row + 1)).astype(np.int64)
    cnt[::empty_every] = 0
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(cnt, out=rp[1:])
    nnz = int(rp[-1])
    cols = (wl.uniform01(seed, 5001, max(nnz, 1))[:nnz] * n).astype(np.int64)
    vals = wl.uniform_pm1(seed, 5002, max(nnz, 1))[:nnz]
    return wl.CSR(n, rp.astype(np.int32), cols.astype(np.int32), vals)


def padded_block(n, s, seed):
    kp = int(2 ** np.ceil(np.log2(s))) if s > 1 else 1
    P = np.zeros((n, kp))
    P[:, :s] = wl.initial_block(n, s, seed)
    return P, kp


def run_spmm_gram(mb, A, P, s):
    n = A.n
    dev = torch.device("cuda")
    rp = torch.as_tensor(A.row_ptr, device=dev)
    ci = torch.as_tensor(A.col_idx if A.nnz else np.zeros(1, np.int32), device=dev)
    av = torch.as_tensor(A.val if A.nnz else np.zeros(1), device=dev)
    Pd = torch.as_tensor(np.ascontiguousarray(P), device=dev)
    AP = torch.full_like(Pd, float("nan"))
    G = torch.empty((s, s), dtype=torch.float64, device=dev)
    nbytes = mb.mbpcg_k_scratch_bytes(n, s)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    st = mb.mbpcg_k_spmm_gram(n, rp, ci, av, s, Pd, AP, G, scratch, nbytes, None)
    assert st == 0, mb.last_error()
    torch.cuda.synchronize()
    return AP.cpu().numpy(), G.cpu().numpy().T  # column-major s x s


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 8, 13, 16, 32])
@pytest.mark.parametrize("n", [1, 7, 33, 1000, 4099])
def test_spmm_gram_matches_oracle(mb, orc, n, s):
    A = random_csr(n, n + s)
    P, kp = padded_block(n, s, 7)
    AP, G = run_spmm_gram(mb, A, P, s)
    ref = orc.matmat(A, P)
    scale = (np.abs(A.to_scipy()) @ np.abs(P)).max() + 1e-300
    assert np.abs(AP - ref).max() <= 1e-13 * scale
    assert np.all(AP[:, s:] == 0.0)
    Gref = P[:, :s].T @ ref[:, :s]
    Gref_u = np.triu(Gref) + np.triu(Gref, 1).T  # the library accumulates the upper triangle
    assert np.abs(G - Gref_u).max() <= 1e-12 * (np.abs(P).sum(0).max() * np.abs(ref).sum(0).max() + 1e-300) + 1e-300
    assert np.array_equal(G, G.T)


def test_spmm_gram_empty_matrix_and_determinism(mb, orc):
    A = wl.CSR(9, np.zeros(10, np.int32), np.zeros(0, np.int32), np.zeros(0))
    P, kp = padded_block(9, 4, 1)
    AP, G = run_spmm_gram(mb, A, P, 4)
    assert np.all(AP == 0.0) and np.all(G == 0.0)
    B = wl.poisson2d(40)
    P, kp = padded_block(B.n, 8, 2)
    r1 = run_spmm_gram(mb, B, P, 8)
    r2 = run_spmm_gram(mb, B, P, 8)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


@pytest.mark.parametrize("s", [1, 2, 4, 6, 8, 16, 32])
@pytest.mark.parametrize("n", [5, 300, 1031])
def test_dense_gram_matches_oracle(mb, orc, n, s):
    D = wl.dense_spd(n, 3, 0.0, 3.0)
    P, kp = padded_block(n, s, 4)
    dev = torch.device("cuda")
    Ad = torch.as_tensor(np.asfortranarray(D.a).ravel(order="F"), device=dev)
    Pd = torch.as_tensor(np.ascontiguousarray(P), device=dev)
    AP = torch.empty_like(Pd)
    G = torch.empty((s, s), dtype=torch.float64, device=dev)
    nbytes = mb.mbpcg_k_scratch_bytes(n, s)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    assert mb.mbpcg_k_dense_gram(n, Ad, s, Pd, AP, G, scratch, nbytes, None) == 0, mb.last_error()
    torch.cuda.synchronize()
    ref = orc.matmat(D, P)
    scale = (np.abs(D.a) @ np.abs(P)).max()
    assert np.abs(AP.cpu().numpy() - ref).max() <= 1e-13 * scale
    Gref = P[:, :s].T @ ref[:, :s]
    Gref_u = np.triu(Gref) + np.triu(Gref, 1).T
    assert np.abs(G.cpu().numpy().T - Gref_u).max() <= 1e-12 * np.abs(Gref).max() * 10


@pytest.mark.parametrize("s", [1, 2, 7, 16, 32])
def test_cholesky_kernel(mb, s):
    rng_m = wl.uniform_pm1(s, 6000, s * s).reshape(s, s)
    G = rng_m @ rng_m.T + s * np.eye(s)
    dev = torch.device("cuda")
    Gd = torch.as_tensor(np.asfortranarray(G).ravel(order="F"), device=dev)
    Z = torch.empty(s * s, dtype=torch.float64, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    assert mb.mbpcg_k_cholesky(s, Gd, Z, status, None) == 0
    torch.cuda.synchronize()
    Zh = Z.cpu().numpy().reshape(s, s, order="F")
    assert int(status.item()) == 0
    assert np.allclose(np.tril(Zh, -1), 0.0)
    assert np.abs(Zh - np.linalg.cholesky(G).T).max() <= 1e-12 * np.abs(G).max()


def test_cholesky_kernel_breakdown(mb):
    s = 6
    v = wl.uniform_pm1(1, 6001, s)
    G = np.outer(v, v) + np.diag([1.0] * (s - 1) + [0.0]) * 0.0  # rank one
    dev = torch.device("cuda")
    Gd = torch.as_tensor(np.asfortranarray(G).ravel(order="F"), device=dev)
    Z = torch.empty(s * s, dtype=torch.float64, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    assert mb.mbpcg_k_cholesky(s, Gd, Z, status, None) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 6


def _ulp_error(y, ref):
    """|y - ref| in units of the FP64 ulp of ref (2^(floor(log2 ref) - 52)), in extended precision."""
    _, ex = np.frexp(ref)
    ulp = np.ldexp(np.longdouble(1.0), (ex - 53).astype(np.int64))
    return np.abs(y.astype(np.longdouble) - ref) / ulp


def test_pivot_reciprocals_within_their_error_bounds(mb):
    """The pivots' 1/d and 1/sqrt(d) of the k x k steps (FP32 hardware seed + one third-order Newton
    step in FP64) against the exact values, computed in extended precision: within 0.51 ulp and
    1.01 ulp (the bounds the error analysis of the Newton step gives: the seed's relative error is
    below 2^-22, so the truncated series adds below 2^-64; the inverse square root takes one more
    rounding, of d y0, worth half an ulp), over the whole accepted range 2^-1022 <= d < 2^1000."""
    if np.finfo(np.longdouble).nmant < 63:
        pytest.skip("no extended-precision long double for the exact reference")
    m = 200_003  # ragged against the 256-thread CTAs
    sig = 1.0 + wl.uniform01(3, 7000, m)
    ex = np.floor(-1022 + 2022 * wl.uniform01(3, 7001, m)).astype(np.int64)
    top = np.nextafter(2.0 ** 1000, 0.0)
    edges = np.array([1.0, 2.0, np.nextafter(2.0, 0.0), np.nextafter(1.0, 2.0), 2.0 ** -1022, top, 3.0, 0.75,
                      np.nextafter(4.0, 0.0), 2.0 ** 999, 2.0 ** -1021 * 1.5])
    pw2 = np.ldexp(1.0, np.arange(-1022, 1000))  # powers of two: both results are exact for even exponents
    d = np.concatenate([np.minimum(np.ldexp(sig, ex), top), edges, pw2])
    assert np.all(d >= 2.0 ** -1022) and np.all(d < 2.0 ** 1000)
    dev = torch.device("cuda")
    dd = torch.as_tensor(d, device=dev)
    inv = torch.full_like(dd, float("nan"))
    rsq = torch.full_like(dd, float("nan"))
    assert mb.mbpcg_k_pivot_reciprocals(d.size, dd, inv, rsq, None) == 0
    torch.cuda.synchronize()
    inv_h, rsq_h = inv.cpu().numpy(), rsq.cpu().numpy()
    dl = d.astype(np.longdouble)
    e_inv = _ulp_error(inv_h, 1 / dl)
    e_rsq = _ulp_error(rsq_h, 1 / np.sqrt(dl))
    assert np.all(np.isfinite(inv_h)) and np.all(np.isfinite(rsq_h))
    assert e_inv.max() <= 0.51, (float(e_inv.max()), d[np.argmax(e_inv)])
    assert e_rsq.max() <= 1.01, (float(e_rsq.max()), d[np.argmax(e_rsq)])
    k = d.size - pw2.size
    assert np.array_equal(inv_h[k:], 1.0 / pw2)  # 1 / 2^j is exact
    even = (np.arange(-1022, 1000) % 2) == 0
    assert np.array_equal(rsq_h[k:][even], 1.0 / np.sqrt(pw2[even]))  # 2^(-j/2) is exact for even j


@pytest.mark.parametrize("s", [1, 4, 9, 16, 32])
@pytest.mark.parametrize("n", [64, 300, 1031, 2049])
def test_dense_tc_product_matches_oracle(mb, orc, n, s):
    """The tensor-core (exact digit splitting) product against the FP64 oracle: the error must be at
    the FP64 rounding level of |A||P| entry by entry (an FP64 GEMM's own bound is n eps |A||P|).
    On 152 SMs, n = 1031 splits 153 one-chunk windows over 144 CTAs and n = 2049 splits 289
    two-chunk windows (the last of each tile one chunk) over 136 CTAs: CTA ranges cross row tiles."""
    D = wl.dense_spd(n, 5, 0.0, 6.0)
    P, kp = padded_block(n, s, 6)
    P[:, :s] *= 10.0 ** (3 * wl.uniform_pm1(9, 77, s))[None, :]  # columns of very different scales
    dev = torch.device("cuda")
    Ad = torch.as_tensor(np.asfortranarray(D.a).ravel(order="F"), device=dev)
    Pd = torch.as_tensor(np.ascontiguousarray(P), device=dev)
    AP = torch.full_like(Pd, float("nan"))
    nbytes = mb.mbpcg_k_dense_tc_scratch_bytes(n, s)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    assert mb.mbpcg_k_dense_tc_prepare(n, Ad, s, scratch, nbytes, None) == 0, mb.last_error()
    assert mb.mbpcg_k_dense_tc_product(n, s, Pd, AP, scratch, nbytes, None) == 0, mb.last_error()
    torch.cuda.synchronize()
    got = AP.cpu().numpy()
    ref = orc.matmat(D, P)
    scale = np.abs(np.asarray(D.a)) @ np.abs(P)
    assert np.all(np.isfinite(got[:, :s]))
    assert np.all(np.abs(got[:, :s] - ref[:, :s]) <= 1e-14 * scale[:, :s] + 1e-300)


@pytest.mark.parametrize("w", [16, 32])
@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("n", [1, 127, 128, 300, 4099])
def test_rowprod_tc_matches_oracle(mb, orc, n, trans, w):
    """The k x k-row products on the tensor cores (Y = X M, X n x w, M w x w, digit splitting)
    against the oracle's FP64 product of the same data. Columns of X and entries of M spread over
    several orders of magnitude, as in the loop (T = Xi Sigma). Bound: the digits keep 56 bits of
    each row scale of X and column scale of M, so the error is a few 2^-53 of
    max_l |X_il| sum_l |M_lj| + sum_l |X_il| max_l |M_lj|; the oracle's own FP64 sum adds w u of
    sum_l |X_il||M_lj|."""
    X = wl.initial_block(n, w, 12) * 10.0 ** (2 * wl.uniform_pm1(3, 91, w))[None, :]
    M = (wl.uniform_pm1(5, 92, w * w) * 10.0 ** (3 * wl.uniform_pm1(5, 93, w * w))).reshape(w, w, order="F")
    M[5, :] = 0.0  # a zero row and column
    M[:, 7] = 0.0
    X[::7, :] = 0.0  # zero rows of X
    dev = torch.device("cuda")
    Xd = torch.as_tensor(np.ascontiguousarray(X), device=dev)
    Md = torch.as_tensor(np.asfortranarray(M).ravel(order="F"), device=dev)
    Yd = torch.full_like(Xd, float("nan"))
    assert mb.mbpcg_k_rowprod_tc(n, w, Xd, Md, trans, Yd, None) == 0, mb.last_error()
    torch.cuda.synchronize()
    got = Yd.cpu().numpy()
    Mu = M.T if trans else M  # the matrix used
    # the oracle's product: Y^T = Mu^T X^T, Mu^T as a 32 x 32 dense matrix
    ref = orc.matmat(wl.Dense(w, np.asfortranarray(Mu.T)), np.asfortranarray(X.T)).T
    aX, aM = np.abs(X), np.abs(Mu)
    bound = aX.max(axis=1)[:, None] * aM.sum(axis=0)[None, :] + aX.sum(axis=1)[:, None] * aM.max(axis=0)[None, :]
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= 2.0 ** -48 * bound + 1e-300)
    zero_col = 5 if trans else 7  # the zero column of the matrix used
    assert np.all(got[::7, :] == 0.0) and np.all(got[:, zero_col] == 0.0)
    assert mb.mbpcg_k_rowprod_tc(n, w, Xd, Md, 2, Yd, None) == mb._native.MBPCG_ERR_INVALID
    assert mb.mbpcg_k_rowprod_tc(n, 8, Xd, Md, 0, Yd, None) == mb._native.MBPCG_ERR_INVALID


def test_dense_tc_mma_alone_leaves_the_product_untouched(mb):
    """The timing entry for the MMA kernel alone runs on the digits a product call left in scratch
    and writes only inside scratch: AP from the product stays as it was."""
    n, s = 300, 32
    D = wl.dense_spd(n, 5, 0.0, 3.0)
    P, kp = padded_block(n, s, 6)
    dev = torch.device("cuda")
    Ad = torch.as_tensor(np.asfortranarray(D.a).ravel(order="F"), device=dev)
    Pd = torch.as_tensor(np.ascontiguousarray(P), device=dev)
    AP = torch.full_like(Pd, float("nan"))
    nbytes = mb.mbpcg_k_dense_tc_scratch_bytes(n, s)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    assert mb.mbpcg_k_dense_tc_mma(n, s, scratch, nbytes - 1, None) == mb._native.MBPCG_ERR_INVALID
    assert mb.mbpcg_k_dense_tc_prepare(n, Ad, s, scratch, nbytes, None) == 0, mb.last_error()
    assert mb.mbpcg_k_dense_tc_product(n, s, Pd, AP, scratch, nbytes, None) == 0, mb.last_error()
    before = AP.clone()
    assert mb.mbpcg_k_dense_tc_mma(n, s, scratch, nbytes, None) == 0, mb.last_error()
    torch.cuda.synchronize()
    assert torch.equal(AP, before)
