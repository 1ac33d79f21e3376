"""Pins for the oracle: each check compares the oracle with something other than itself --
LAPACK/scipy solvers, the textbook CG of scipy, closed forms, and invariants that Algorithm 1 and
Proposition 1 of the paper fix. No GPU needed."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def spd_with_spectrum(n, lam, seed):
    g = wl.uniform_pm1(seed, 4000, n * n).reshape(n, n)
    Q, _ = np.linalg.qr(g)
    A = (Q * lam) @ Q.T
    return wl.Dense(n, np.asfortranarray(0.5 * (A + A.T)))


def dense_to_csr(D):
    S = sp.csr_matrix(np.asarray(D.a))
    S.sort_indices()
    return wl.CSR(D.n, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def amul(A, X):
    if isinstance(A, wl.Dense):
        return np.asarray(A.a) @ X
    return A.to_scipy() @ X


# ------------------------------------------------------------------------------ generators


def test_splitmix_matches_published_outputs():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    gamma = np.uint64(int(g["gamma"], 16))
    with np.errstate(over="ignore"):
        got = [int(wl._mix(np.uint64(i) * gamma)) for i in (1, 2, 3)]
    assert got == [int(h, 16) for h in g["outputs"]]


def test_generator_structure_closed_forms():
    assert wl.poisson2d(64).nnz == 5 * 64 * 64 - 4 * 64 == 20224
    assert wl.diffusion3d(8, 0).nnz == 7 * 8 ** 3 - 6 * 8 ** 2
    assert wl.stencil27(6, 0).nnz == (3 * 6 - 2) ** 3
    # Poisson eigenvalues: 4 - 2 cos(i pi/(m+1)) - 2 cos(j pi/(m+1))
    m = 12
    ev = np.linalg.eigvalsh(wl.poisson2d(m).to_scipy().toarray())
    t = 2 - 2 * np.cos(np.arange(1, m + 1) * np.pi / (m + 1))
    assert np.allclose(np.sort(ev), np.sort((t[:, None] + t[None, :]).ravel()), atol=1e-12)
    for A in (wl.diffusion3d(6, 3), wl.stencil27(5, 3)):
        S = A.to_scipy()
        assert abs(S - S.T).max() == 0.0
        assert np.linalg.eigvalsh(S.toarray()).min() > 0


# ------------------------------------------------------------------------------ matmat


@pytest.mark.parametrize("k", [1, 3, 8])
def test_matmat_matches_scipy(orc, k):
    A = wl.random_spd_csr(37, 5, density=0.08)
    X = wl.initial_block(37, k, 9)
    assert np.allclose(orc.matmat(A, X), A.to_scipy() @ X, rtol=0, atol=1e-13)
    D = spd_with_spectrum(19, np.linspace(1, 3, 19), 2)
    X = wl.initial_block(19, k, 9)
    assert np.allclose(orc.matmat(D, X), np.asarray(D.a) @ X, rtol=0, atol=1e-13)


def test_matmat_empty_rows(orc):
    # rows 1 and 3 empty
    A = wl.CSR(4, np.array([0, 1, 1, 3, 3], np.int32), np.array([0, 0, 2], np.int32), np.array([2.0, 1.0, 5.0]))
    X = np.arange(8.0).reshape(4, 2, order="F")
    assert np.array_equal(orc.matmat(A, X), A.to_scipy() @ X)


# ------------------------------------------------------------------------------ whole solver


@pytest.mark.parametrize("n,k,sparse", [(8, 1, False), (16, 2, True), (64, 4, False), (64, 8, True), (48, 3, True)])
def test_solution_matches_cholesky_solve(orc, n, k, sparse):
    D = spd_with_spectrum(n, np.linspace(1.0, 50.0, n), n + k)
    A = dense_to_csr(D) if sparse else D
    b = wl.rhs(n, 11)
    U = wl.initial_block(n, k, 12)
    x, c, info = orc.mbpcg(A, b, U, precond=0, tol=1e-12)
    xs = sla.cho_solve(sla.cho_factor(np.asarray(D.a)), b)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-10


def test_golden_two_by_two(orc):
    g = json.load(open(os.path.join(GOLDEN, "tiny_2x2.json")))
    A = wl.Dense(2, np.asfortranarray(np.array(g["A"])))
    x, c, info = orc.mbpcg(A, np.array(g["b"]), np.asfortranarray(np.array(g["U"])), tol=1e-12)
    assert info["iterations"] == g["iterations"]
    assert info["ls_fallback"] == 1
    assert np.allclose(x, np.array(g["x_num"]) / g["x_den"], rtol=0, atol=1e-14)


@pytest.mark.parametrize("n,k", [(64, 8), (64, 4), (60, 6), (32, 16)])
def test_block_krylov_termination(orc, n, k):
    """Block CG over a k-dimensional block spans n dimensions after ceil(n/k) steps (exact
    arithmetic). With kappa <= 10 FP64 rounding does not delay it: the oracle must stop within
    ceil(n/k) iterations. (At kappa = 1e2 loss of orthogonality adds a few steps, n=64, k=4 takes
    20 in any FP64 implementation, so that case is not a termination pin.)"""
    D = spd_with_spectrum(n, np.geomspace(1.0, 10.0, n), 3)
    b = wl.rhs(n, 1)
    U = wl.initial_block(n, k, 2)
    x, c, info = orc.mbpcg(D, b, U, tol=1e-10)
    assert info["status"] == 0
    assert info["iterations"] <= -(-n // k)


def _textbook_cg(A, b, x0, tol, M=None):
    its = []
    x, flag = spla.cg(A, b, x0=x0, rtol=tol, atol=0.0, maxiter=100000, M=M, callback=lambda xk: its.append(1))
    return x, len(its), flag


def test_k1_equals_textbook_cg_same_start(orc):
    """Section 5 / Section 4: MBPCG with k = 1 follows CG; in exact arithmetic it IS CG started
    from X0. scipy's textbook CG from the oracle's X0 must take the same steps."""
    A = wl.poisson2d(32)
    n = A.n
    b = wl.rhs(n, 0)
    U = wl.initial_block(n, 1, 1)
    states = []
    x, c, info = orc.mbpcg(A, b, U, tol=1e-8, callback=lambda it, ex, rs, s: states.append(s) if it == 0 else None)
    X0 = states[0]["X0"][:, 0]
    # the paper's normalisation of the random start: ||A X0||_F = ||B||_F
    assert np.isclose(np.linalg.norm(A.to_scipy() @ X0), np.linalg.norm(b), rtol=1e-13)
    xr, its, flag = _textbook_cg(A.to_scipy(), b, X0, 1e-8)
    assert flag == 0
    assert abs(info["iterations"] - its) <= 1
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-8


def test_k1_jacobi_equals_textbook_pcg(orc):
    """Diagonal scaling (Section 1) with k = 1 is Jacobi-preconditioned CG in exact arithmetic."""
    A = wl.diffusion3d(10, 4)
    n = A.n
    b = wl.rhs(n, 0)
    U = wl.initial_block(n, 1, 1)
    states = []
    x, c, info = orc.mbpcg(A, b, U, precond=1, tol=1e-8,
                           callback=lambda it, ex, rs, s: states.append(s) if it == 0 else None)
    dg = A.diagonal()
    x0 = states[0]["X0"][:, 0] / np.sqrt(dg)  # x = D^{-1} xbar
    Minv = spla.LinearOperator((n, n), matvec=lambda v: v / dg)
    xr, its, flag = _textbook_cg(A.to_scipy(), b, x0, 1e-8, M=Minv)
    assert flag == 0
    assert abs(info["iterations"] - its) <= 1
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-8


def test_cgear_equals_textbook_cg(orc):
    """Chronopoulos-Gear CG is CG in exact arithmetic (Section 1); zero start (Section 4)."""
    for A, pre in ((wl.poisson2d(40), 0), (wl.diffusion3d(9, 1), 1)):
        b = wl.rhs(A.n, 3)
        x, info = orc.cg_cgear(A, b, precond=pre, tol=1e-8)
        dg = A.diagonal()
        M = spla.LinearOperator((A.n, A.n), matvec=lambda v: v / dg) if pre else None
        xr, its, flag = _textbook_cg(A.to_scipy(), b, np.zeros(A.n), 1e-8, M=M)
        assert info["status"] == 0 and flag == 0
        assert abs(info["iterations"] - its) <= 1
        assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-7


# ------------------------------------------------------------------------------ invariants


def _scaled(A, precond):
    S = A.to_scipy()
    d = 1.0 / np.sqrt(A.diagonal()) if precond else np.ones(A.n)
    return sp.diags(d) @ S @ sp.diags(d), d


@pytest.mark.parametrize("precond", [0, 1])
def test_proposition1_and_R_equals_W_Sigma(orc, precond):
    """Proposition 1: A X~^i + R^i = B~ for every i; and R^i = W^i Sigma^i (the QR of the
    residual block carried through the zeta updates of Algorithm 1)."""
    A = wl.poisson2d(64) if precond == 0 else wl.diffusion3d(12, 2)
    n, k = A.n, 4
    b = wl.rhs(n, 0)
    U = wl.initial_block(n, k, 1)
    As, d = _scaled(A, precond)
    Bbar = np.outer(d * b, np.ones(k))
    worst = [0.0, 0.0]

    def cb(it, exiting, restart, s):
        if restart or it > 200:
            return
        Bt = Bbar - As @ s["X0"]
        worst[0] = max(worst[0], np.linalg.norm(As @ s["Xt"] + s["R"] - Bt) / np.linalg.norm(Bt))
        if not exiting:
            worst[1] = max(worst[1], np.linalg.norm(s["R"] - s["W"] @ s["Sigma"]) / np.linalg.norm(s["R"]))
    x, c, info = orc.mbpcg(A, b, U, precond=precond, tol=1e-8, callback=cb)
    assert info["status"] == 0
    assert worst[0] <= 1e-10
    assert worst[1] <= 1e-6


def test_cholqr_orthonormal_and_sigma_upper(orc):
    A = wl.poisson2d(24)
    n, k = A.n, 6
    b = wl.rhs(n, 0)
    U = wl.initial_block(n, k, 1)
    errs = []

    def cb(it, exiting, restart, s):
        if exiting or it > 20:
            return
        W, Sg = s["W"], s["Sigma"]
        errs.append(np.linalg.norm(W.T @ W - np.eye(k)))
        assert np.allclose(np.tril(Sg, -1), 0.0)
        assert np.all(np.diag(Sg) > 0)
    orc.mbpcg(A, b, U, tol=1e-8, callback=cb)
    assert max(errs) <= 1e-8


def test_block_a_conjugacy(orc):
    """Consecutive search blocks are A-conjugate: P^{i,T} A P^{i-1} = 0 (block CG)."""
    A = wl.poisson2d(32)
    n, k = A.n, 4
    S = A.to_scipy()
    b = wl.rhs(n, 0)
    U = wl.initial_block(n, k, 1)
    Ps = []
    orc.mbpcg(A, b, U, tol=1e-8, callback=lambda it, ex, rs, s: Ps.append(s["P"]) if (not ex and it <= 6) else None)
    for P1, P0 in zip(Ps[1:], Ps[:-1]):
        cross = P1.T @ (S @ P0)
        nrm = np.sqrt(np.linalg.norm(P1.T @ (S @ P1)) * np.linalg.norm(P0.T @ (S @ P0)))
        assert np.linalg.norm(cross) / nrm <= 1e-8


@pytest.mark.parametrize("precond", [0, 1])
def test_least_squares_exit_matches_lstsq(orc, precond):
    """The exit combination c = argmin ||b - Bhat c|| with Bhat = B - R = A X (Proposition 1), in
    the original-system metric; and ||b - Bhat c|| <= min_j ||R_j|| (Bhat e_h = b - R_h)."""
    A = wl.poisson2d(40) if precond == 0 else wl.diffusion3d(10, 1)
    n, k = A.n, 4
    b = wl.rhs(n, 0)
    U = wl.initial_block(n, k, 1)
    d = 1.0 / np.sqrt(A.diagonal()) if precond else np.ones(n)
    final = {}
    x, c, info = orc.mbpcg(A, b, U, precond=precond, tol=1e-8,
                           callback=lambda it, ex, rs, s: final.update(s) if ex else None)
    R_orig = final["R"] / d[:, None]
    Bhat = b[:, None] - R_orig
    c_ref, *_ = np.linalg.lstsq(Bhat, b, rcond=None)
    r_ref = np.linalg.norm(b - Bhat @ c_ref)
    r_got = np.linalg.norm(b - Bhat @ c)
    assert info["ls_fallback"] == 0
    assert r_got <= np.linalg.norm(R_orig, axis=0).min() * (1 + 1e-12)
    assert r_got <= r_ref * (1 + 1e-6)
    # same minimiser: x from the oracle's c vs x from lstsq's c
    X = (final["Xt"] + final["X0"]) * d[:, None]
    assert np.linalg.norm(X @ c - X @ c_ref) / np.linalg.norm(X @ c_ref) <= 1e-6
    assert np.allclose(x, X @ c, rtol=0, atol=1e-12 * np.abs(x).max())


def test_true_residual_restart_reaches_tol(orc):
    """A recurrence residual below tol does not bound the true residual (ill-conditioned dense
    system); the restart rule must bring the recomputed ||b - A x|| / ||b|| under tol."""
    A = wl.dense_spd(256, 0)
    b = wl.rhs(256, 0)
    for k in (4, 8):
        U = wl.initial_block(256, k, 1)
        x, c, info = orc.mbpcg(A, b, U, tol=1e-8)
        true = np.linalg.norm(b - np.asarray(A.a) @ x) / np.linalg.norm(b)
        assert info["status"] == 0
        assert true <= 1e-8
        assert np.isclose(true, info["relres_true"], rtol=1e-6)


def test_cg_true_residual(orc):
    A = wl.dense_spd(128, 1)
    b = wl.rhs(128, 0)
    x, info = orc.cg_cgear(A, b, tol=1e-8)
    assert info["status"] == 0
    assert np.linalg.norm(b - np.asarray(A.a) @ x) / np.linalg.norm(b) <= 1e-8


# ------------------------------------------------------------------------------ errors


def test_invalid_inputs(orc):
    A = wl.poisson2d(4)
    b = wl.rhs(A.n, 0)
    U = wl.initial_block(A.n, 2, 1)
    bad = wl.CSR(A.n, A.row_ptr.copy(), A.col_idx.copy(), A.val.copy())
    bad.col_idx[3] = A.n + 5
    assert orc.mbpcg(bad, b, U)[2]["status"] == 1
    neg = wl.CSR(A.n, A.row_ptr.copy(), A.col_idx.copy(), -A.val)
    assert orc.mbpcg(neg, b, U, precond=1)[2]["status"] == 4
    assert orc.mbpcg(A, b, U, tol=0.0)[2]["status"] == 1


def test_maxit_not_converged_returns_best_column(orc):
    A = wl.poisson2d(32)
    b = wl.rhs(A.n, 0)
    U = wl.initial_block(A.n, 4, 1)
    x, c, info = orc.mbpcg(A, b, U, tol=1e-8, maxit=5, max_restarts=0)
    assert info["status"] == 5 and info["iterations"] == 5
    true = np.linalg.norm(b - A.to_scipy() @ x) / np.linalg.norm(b)
    assert np.isclose(true, info["relres_recurrence"], rtol=1e-6)


def test_state_matches_full_solve_prefix(orc):
    A = wl.poisson2d(16)
    b = wl.rhs(A.n, 0)
    U = wl.initial_block(A.n, 3, 1)
    seen = {}
    orc.mbpcg(A, b, U, tol=1e-8, callback=lambda it, ex, rs, s: seen.__setitem__(it, s) if not ex else None)
    st, status = orc.mbpcg_state(A, b, U, 5)
    assert status == 0
    for name in ("Xt", "R", "W", "P", "Sigma", "X0"):
        assert np.array_equal(st[name], seen[5][name])


# ------------------------------------------------------------------------------ breakdown


def one_block_step(A, r, U):
    """One step of textbook block CG from X0 = c U on A e = r, written from its closed form: with
    R0 = r 1^T - A X0, the first block iterate is the A-orthogonal (Galerkin) correction over
    span(R0), X1 = X0 + R0 (R0^T A R0)^{-1} R0^T R0 (Algorithm 1 reaches the same X1, since P0 spans
    R0). c = ||r 1^T||_F / ||A U||_F as in the set-up of Algorithm 1. Returns X1 and the residual
    norms of its columns."""
    M = np.asarray(A.a)
    s = U.shape[1]
    c = np.sqrt(s) * np.linalg.norm(r) / np.linalg.norm(M @ U)
    X0 = c * U
    R0 = r[:, None] - M @ X0
    X1 = X0 + R0 @ np.linalg.solve(R0.T @ M @ R0, R0.T @ R0)
    return X1, np.linalg.norm(r[:, None] - M @ X1, axis=0)


def breakdown_system(n=6, s=4):
    # a well-conditioned SPD 6 x 6 with s = 4 copies: after one block step the residual block lies in
    # the 2-dimensional A-orthogonal complement of span(R0), so V (whose column space is that of the
    # new residual block) has rank 2 < 4 and the Cholesky QR of V meets a zero pivot: breakdown
    A = spd_with_spectrum(n, np.linspace(1.0, 4.0, n), 11)
    return A, wl.rhs(n, 3), wl.initial_block(n, s, 5)


def test_breakdown_when_block_krylov_space_is_exhausted(orc):
    """Cholesky breakdown (pivot not above 64 eps max G_jj) in the Cholesky QR of V after the first
    iteration: status BREAKDOWN after exactly one iteration, x = the best column of the first block
    iterate (Algorithm 1's best-basis choice h = argmin_j ||R_j||), checked against the closed form."""
    A, b, U = breakdown_system()
    x, c, info = orc.mbpcg(A, b, U, tol=1e-12, max_restarts=0)
    assert info["status"] == 6 and info["iterations"] == 1, info
    X1, res = one_block_step(A, b, U)
    h = int(np.argmin(res))
    assert info["best_col"] == h
    assert np.array_equal(c, np.eye(U.shape[1])[h])
    assert np.linalg.norm(x - X1[:, h]) <= 1e-12 * np.linalg.norm(X1[:, h])
    assert np.isclose(info["relres_recurrence"], res[h] / np.linalg.norm(b), rtol=1e-8)


def test_breakdown_then_restarts_follow_the_same_rule(orc):
    """With the true-residual restarts on, each correction solve breaks down the same way and adds
    the best column of its own first block iterate (same U, right-hand side b - A x); the solve ends
    with status BREAKDOWN after max_restarts restarts unless the true residual reaches tol first."""
    A, b, U = breakdown_system()
    tol = 1e-12
    x, c, info = orc.mbpcg(A, b, U, tol=tol, max_restarts=3)
    M = np.asarray(A.a)
    xr = np.zeros_like(b)
    rounds = 0
    while True:
        r = b - M @ xr
        X1, res = one_block_step(A, r, U)
        xr = xr + X1[:, int(np.argmin(res))]
        rounds += 1
        if np.linalg.norm(b - M @ xr) <= tol * np.linalg.norm(b) or rounds == 4:
            break
    assert info["iterations"] == rounds and info["restarts"] == rounds - 1, info
    assert info["status"] == (0 if np.linalg.norm(b - M @ xr) <= tol * np.linalg.norm(b) else 6), info
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)


def test_breakdown_at_setup_when_s_exceeds_n(orc):
    """s > n: R0 (n x s) has rank n < s, so the set-up Cholesky QR breaks down before the first
    iteration; x = c U_h, the best column of X0 (h = argmin_j ||b - c A U_j||)."""
    A = spd_with_spectrum(3, np.array([1.0, 2.0, 3.0]), 12)
    b = wl.rhs(3, 4)
    U = wl.initial_block(3, 4, 6)
    x, c, info = orc.mbpcg(A, b, U, tol=1e-12, max_restarts=0)
    assert info["status"] == 6 and info["iterations"] == 0, info
    M = np.asarray(A.a)
    cs = np.sqrt(4) * np.linalg.norm(b) / np.linalg.norm(M @ U)
    res = np.linalg.norm(b[:, None] - cs * (M @ U), axis=0)
    h = int(np.argmin(res))
    assert info["best_col"] == h
    assert np.linalg.norm(x - cs * U[:, h]) <= 1e-14 * np.linalg.norm(cs * U[:, h])


# ------------------------------------------------------------------------------ OpenMP build


@pytest.mark.parametrize("dense", [True, False])
def test_openmp_build_gives_the_same_bits(orc, dense):
    """The timed CPU baseline runs the same oracle source built with OpenMP: it only shares
    independent loop iterations among threads, so solution, coefficients and counts are the
    parity build's, bit for bit."""
    A = wl.dense_spd(96, 2, 0.0, 3.0) if dense else wl.poisson2d(12)
    b = wl.rhs(A.n, 0)
    U = wl.initial_block(A.n, 8, 1)
    x1, c1, i1 = orc.mbpcg(A, b, U, tol=1e-10)
    x2, c2, i2 = orc.mbpcg(A, b, U, tol=1e-10, omp=True)
    assert np.array_equal(x1, x2) and np.array_equal(c1, c2) and i1 == i2
    s1, _ = orc.mbpcg_state(A, b, U, 4)
    s2, _ = orc.mbpcg_state(A, b, U, 4, omp=True)
    for key in s1:
        assert np.array_equal(s1[key], s2[key]), key
